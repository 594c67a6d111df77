// mk_ctx.h -- the library context (host state of one mk_ctx) and the host
// helpers shared by the host translation units (mk_host.cpp, mk_server.cpp).
// Not part of the public ABI.
#pragma once
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "mk_internal.h"

namespace mk {

// ------------------------------------------------------------ host Goldilocks NTT
constexpr uint64_t P = kGoldilocks;

inline uint64_t hadd(uint64_t a, uint64_t b) {
    unsigned __int128 s = (unsigned __int128)a + b;
    if (s >= P) s -= P;
    return (uint64_t)s;
}
inline uint64_t hsub(uint64_t a, uint64_t b) { return a >= b ? a - b : a + (P - b); }
inline uint64_t hmul(uint64_t a, uint64_t b) {
    const unsigned __int128 x = (unsigned __int128)a * b;
    const uint64_t lo = (uint64_t)x, hi = (uint64_t)(x >> 64);
    const uint64_t eps = 0xFFFFFFFFull;  // 2^64 mod p
    const uint64_t hh = hi >> 32, hl = hi & eps;
    // x = lo + hl * 2^64 + hh * 2^96 = lo + hl * (2^32 - 1) - hh  (mod p)
    uint64_t t0 = lo - hh;
    if (lo < hh) t0 -= eps;
    const uint64_t t1 = hl * eps;
    uint64_t r = t0 + t1;
    if (r < t1) r += eps;
    return r >= P ? r - P : r;
}
inline uint64_t hpow(uint64_t b, uint64_t e) {
    uint64_t r = 1;
    while (e) {
        if (e & 1) r = hmul(r, b);
        b = hmul(b, b);
        e >>= 1;
    }
    return r;
}

struct HostNtt {
    uint32_t N = 0, logN = 0;
    std::vector<uint64_t> psi_rev, psi_inv_rev;
    uint64_t n_inv = 0;
    bool init(uint32_t n_) {
        N = n_;
        logN = 0;
        while ((1u << logN) < N) ++logN;
        // 7 generates the multiplicative group of the Goldilocks field.
        const uint64_t psi = hpow(7, (P - 1) / (2ull * N));
        if (hpow(psi, N) != P - 1) return false;  // psi must be a primitive 2N-th root
        const uint64_t psi_inv = hpow(psi, P - 2);
        psi_rev.assign(N, 0);
        psi_inv_rev.assign(N, 0);
        for (uint32_t m = 0; m < N; ++m) {
            uint32_t r = 0;
            for (uint32_t b = 0; b < logN; ++b)
                if (m & (1u << b)) r |= 1u << (logN - 1 - b);
            psi_rev[m] = hpow(psi, r);
            psi_inv_rev[m] = hpow(psi_inv, r);
        }
        n_inv = hpow(N, P - 2);
        return true;
    }
    // Cooley-Tukey, natural order in, bit-reversed order out.
    void forward(uint64_t *a) const {
        uint32_t t = N;
        for (uint32_t m = 1; m < N; m <<= 1) {
            t >>= 1;
            for (uint32_t i = 0; i < m; ++i) {
                const uint32_t j1 = 2 * i * t;
                const uint64_t S = psi_rev[m + i];
                for (uint32_t j = j1; j < j1 + t; ++j) {
                    const uint64_t U = a[j], V = hmul(a[j + t], S);
                    a[j] = hadd(U, V);
                    a[j + t] = hsub(U, V);
                }
            }
        }
    }
    // Gentleman-Sande, bit-reversed in, natural out, including 1/N.
    void inverse(uint64_t *a) const {
        uint32_t t = 1;
        for (uint32_t m = N; m > 1; m >>= 1) {
            uint32_t j1 = 0;
            const uint32_t h = m >> 1;
            for (uint32_t i = 0; i < h; ++i) {
                const uint64_t S = psi_inv_rev[h + i];
                for (uint32_t j = j1; j < j1 + t; ++j) {
                    const uint64_t U = a[j], V = a[j + t];
                    a[j] = hadd(U, V);
                    a[j + t] = hmul(hsub(U, V), S);
                }
                j1 += 2 * t;
            }
            t <<= 1;
        }
        for (uint32_t j = 0; j < N; ++j) a[j] = hmul(a[j], n_inv);
    }
    // Torus32 polynomial (coefficients taken in [0, 2^32)) to the NTT domain.
    void to_ntt(const uint32_t *src, uint64_t *dst, bool negate, bool scale_inv_n) const {
        for (uint32_t j = 0; j < N; ++j) dst[j] = negate ? hsub(0, src[j]) : (uint64_t)src[j];
        forward(dst);
        if (scale_inv_n)
            for (uint32_t j = 0; j < N; ++j) dst[j] = hmul(dst[j], n_inv);
    }
    // out = binary * q (negacyclic, mod 2^32).  The integer result lies in
    // (-N*2^32, N*2^32), far inside (-p/2, p/2): lift the field value to that
    // integer (p = 1 mod 2^32, so a negative x maps to (uint32)(x + p) - 1).
    void mul_binary(const uint64_t *bin_hat, const uint32_t *q, uint32_t *out, std::vector<uint64_t> &tmp) const {
        tmp.resize(N);
        for (uint32_t j = 0; j < N; ++j) tmp[j] = q[j];
        forward(tmp.data());
        for (uint32_t j = 0; j < N; ++j) tmp[j] = hmul(tmp[j], bin_hat[j]);
        inverse(tmp.data());
        for (uint32_t j = 0; j < N; ++j) out[j] = (uint32_t)tmp[j] - (tmp[j] > (P >> 1) ? 1u : 0u);
    }
};

// Negacyclic NTT modulo a 30-bit prime (the two primes of MK_FORM_NTT2),
// same index conventions as HostNtt.
struct HostNtt32 {
    uint32_t p = 0, N = 0, logN = 0;
    std::vector<uint32_t> psi_rev, psi_inv_rev;
    uint32_t n_inv = 0;
    static uint32_t mulm(uint32_t a, uint32_t b, uint32_t p) { return (uint32_t)((uint64_t)a * b % p); }
    static uint32_t powm(uint64_t b, uint64_t e, uint32_t p) {
        uint64_t r = 1;
        b %= p;
        while (e) {
            if (e & 1) r = r * b % p;
            b = b * b % p;
            e >>= 1;
        }
        return (uint32_t)r;
    }
    bool init(uint32_t prime, uint32_t n_) {
        p = prime;
        N = n_;
        logN = 0;
        while ((1u << logN) < N) ++logN;
        if ((p - 1) % (2 * N) != 0) return false;
        // g^((p-1)/2N) for a quadratic non-residue g is a primitive 2N-th root
        // of unity (2N is a power of two dividing p - 1).
        uint32_t g = 2;
        while (g < 1000 && powm(g, (p - 1) / 2, p) != p - 1) ++g;
        const uint32_t psi = powm(g, (p - 1) / (2 * N), p);
        if (powm(psi, N, p) != p - 1) return false;
        const uint32_t psi_inv = powm(psi, p - 2, p);
        psi_rev.assign(N, 0);
        psi_inv_rev.assign(N, 0);
        for (uint32_t m = 0; m < N; ++m) {
            uint32_t r = 0;
            for (uint32_t b = 0; b < logN; ++b)
                if (m & (1u << b)) r |= 1u << (logN - 1 - b);
            psi_rev[m] = powm(psi, r, p);
            psi_inv_rev[m] = powm(psi_inv, r, p);
        }
        n_inv = powm(N, p - 2, p);
        return true;
    }
    void forward(uint32_t *a) const {
        uint32_t t = N;
        for (uint32_t m = 1; m < N; m <<= 1) {
            t >>= 1;
            for (uint32_t i = 0; i < m; ++i) {
                const uint32_t j1 = 2 * i * t;
                const uint32_t S = psi_rev[m + i];
                for (uint32_t j = j1; j < j1 + t; ++j) {
                    const uint32_t U = a[j], V = mulm(a[j + t], S, p);
                    a[j] = (U + V) % p;
                    a[j + t] = (U + p - V) % p;
                }
            }
        }
    }
    // Device form of a key polynomial: NTT of its coefficients taken as
    // signed 32-bit integers (the same values mod 2^32; |c| <= 2^31 keeps the
    // product sums within the CRT range), times N^-1, in Montgomery form
    // (times 2^32 mod p).
    void to_device(const uint32_t *src, uint32_t *dst, bool negate) const {
        std::vector<uint32_t> a(N);
        for (uint32_t j = 0; j < N; ++j) {
            int64_t v = (int32_t)src[j];
            if (negate) v = -v;
            int64_t r = v % (int64_t)p;
            if (r < 0) r += p;
            a[j] = (uint32_t)r;
        }
        forward(a.data());
        const uint32_t scale = (uint32_t)(((uint64_t)n_inv << 32) % p);
        for (uint32_t j = 0; j < N; ++j) dst[j] = mulm(a[j], scale, p);
    }
};

// Host side of the FP64 FFT form: negacyclic transform of size M = N/2 over C
// (Cooley-Tukey with psi = exp(i pi / M) in bit-reversed powers), after folding
// (c_j + i c_{j+M}) and twisting by theta^j = exp(-i pi j / N).
struct HostFft {
    uint32_t N = 0, M = 0, logM = 0;
    std::vector<std::complex<double>> psi_rev, psi_inv_rev, theta;
    void init(uint32_t n_) {
        N = n_;
        M = N / 2;
        logM = 0;
        while ((1u << logM) < M) ++logM;
        psi_rev.resize(M);
        psi_inv_rev.resize(M);
        theta.resize(M);
        const double pi = 3.14159265358979323846;
        for (uint32_t m = 0; m < M; ++m) {
            uint32_t r = 0;
            for (uint32_t b = 0; b < logM; ++b)
                if (m & (1u << b)) r |= 1u << (logM - 1 - b);
            psi_rev[m] = std::polar(1.0, pi * r / M);
            psi_inv_rev[m] = std::conj(psi_rev[m]);
            theta[m] = std::polar(1.0, -pi * m / N);
        }
    }
    void forward(std::complex<double> *a) const {
        uint32_t t = M;
        for (uint32_t m = 1; m < M; m <<= 1) {
            t >>= 1;
            for (uint32_t i = 0; i < m; ++i) {
                const uint32_t j1 = 2 * i * t;
                const std::complex<double> S = psi_rev[m + i];
                for (uint32_t j = j1; j < j1 + t; ++j) {
                    const std::complex<double> U = a[j], V = a[j + t] * S;
                    a[j] = U + V;
                    a[j + t] = U - V;
                }
            }
        }
    }
    // Device form of a key polynomial: fold, twist, transform, times 1/M;
    // coefficients taken as signed 32-bit integers (same value mod 2^32).
    void to_device(const uint32_t *src, double *dst, bool negate) const {
        std::vector<std::complex<double>> z(M);
        for (uint32_t j = 0; j < M; ++j) {
            double lo = (double)(int32_t)src[j], hi = (double)(int32_t)src[j + M];
            if (negate) lo = -lo, hi = -hi;
            z[j] = std::complex<double>(lo, hi) * theta[j];
        }
        forward(z.data());
        for (uint32_t j = 0; j < M; ++j) {
            dst[2 * j] = z[j].real() / M;
            dst[2 * j + 1] = z[j].imag() / M;
        }
    }
};

}  // namespace mk

using namespace mk;

struct PartyKeys {
    bool has_public = false, has_secret = false;
    std::vector<uint32_t> s, z, pk, bk, ks;
};

// A k-bit operator prepared for `pairs` operand pairs: the levelised gate
// descriptors (all levels concatenated, gate-major then pair), the wire
// buffer and the per-level scratch.
struct CircuitPlan {
    Netlist net;
    uint32_t pairs = 0, n_wires = 0, max_level = 0;
    std::vector<uint32_t> level_off;  // descriptor offset of each level, size levels + 1
    GateDesc *d_desc = nullptr;
    uint32_t *d_pool = nullptr;
    uint32_t *d_ext = nullptr;
    int32_t *d_outs = nullptr;
    // persistent execution: a ready word per pool row, {item counter, abort}
    uint32_t *d_ready = nullptr;
    uint32_t *d_ctl = nullptr;
    uint32_t epoch = 0;
    uint32_t levels = 0;
    // The level loop captured as a CUDA graph, and what it was captured with.
    cudaGraphExec_t graph = nullptr;
    int graph_form = -1, graph_variant = -1;
    uint32_t graph_cluster = 0;
    DeviceKeys graph_keys{};
    ~CircuitPlan() {
        if (graph) cudaGraphExecDestroy(graph);
        cudaFree(d_desc);
        cudaFree(d_pool);
        cudaFree(d_ext);
        cudaFree(d_outs);
        cudaFree(d_ready);
        cudaFree(d_ctl);
    }
};

struct mk_ctx {
    mk_params P{};
    uint32_t logN = 0;
    uint64_t crs_seed = 0;
    int device = -1;
    cudaStream_t stream = nullptr;
    int form = MK_FORM_NTT2;
    int variant = 2;
    uint32_t max_batch = 4096;
    std::vector<uint32_t> crs;
    std::vector<PartyKeys> party;
    HostNtt ntt;
    HostNtt32 ntt_p1, ntt_p2;
    HostFft fft;
    // device state
    bool dev_keys_valid = false;
    void *d_tw = nullptr;       // [2][N] twiddles (8 or 16 bytes each)
    uint64_t *d_bk = nullptr;   // [k][n][3][d][N]
    uint64_t *d_keyA = nullptr; // [(k+1)][d][N]
    uint32_t *d_ks = nullptr;   // [k][N][t][B'-1][n+1]
    uint32_t *d_status = nullptr;  // status word of the kernels' bounded waits (bit 0: one ran out)
    uint64_t wait_ns = 1000000000ull;  // bound on each such wait (1 s)
    int64_t debug_skip_key_step = -1;  // test hook of the staged kernel (see LaunchShape)
    void *d_tcws = nullptr;     // MK_FORM_TC wave workspace for tc_ws_gates gates
    uint32_t tc_ws_gates = 0;
    uint32_t *d_ext = nullptr;  // scratch [scratch_gates][k*N+1]
    GateDesc *d_desc = nullptr; // scratch [scratch_gates]
    uint32_t scratch_gates = 0;
    std::string err;
    // measurement: event pairs around launches, per kernel class
    bool timing = false;
    bool use_graphs = true;               // circuits replay their level loop as a CUDA graph
    int circuit_style = MK_CIRCUIT_ARRAY;  // netlist family of the operators
    int cluster_mode = MK_CLUSTER_AUTO;   // latency (cluster) kernel for small batches
    int circuit_exec = MK_EXEC_AUTO;      // operators: one launch pair per level, or one persistent launch
    int64_t debug_skip_item = -1;         // test hook of the persistent launch (mk_debug_fault)
    uint32_t sm_count = 0;
    uint32_t cluster_cap = 0;  // resident clusters of the latency form for the keys' form (0: none)
    cudaStream_t capture_stream = nullptr;  // non-default stream the graphs are captured on
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[2];
    std::vector<cudaEvent_t> ev_pool;
    std::map<std::tuple<int, uint32_t, uint32_t, int>, std::unique_ptr<CircuitPlan>> plans;  // op, k, pairs, style

    size_t W() const { return (size_t)P.k * P.n + 1; }
    size_t E() const { return (size_t)P.k * P.N + 1; }
    size_t pk_words() const { return (size_t)P.d * P.N; }
    size_t bk_words() const { return (size_t)P.n * 3 * P.d * P.N; }
    size_t ks_words() const { return (size_t)P.N * P.t * ((1u << P.ks_bit) - 1) * (P.n + 1); }
    LaunchShape shape() const {
        // AUTO: the cluster kernel while the launch's gates fit in max(1,
        // floor(k/2)) waves of resident clusters (cluster_cap, queried from
        // the device for the form's kernel); beyond that the batched kernel's
        // throughput wins.  One gate runs 2-4 times faster in the cluster
        // form (GB300: 16.1 vs 31.3 ms at k = 2, 34.9 vs 99.0 at k = 4, 76.3
        // vs 306 at k = 7), and the measured crossovers sit at one to two,
        // two and three to four waves.  A capacity of 0 (other forms, k > 7,
        // or a shape whose CTA does not fit in shared memory) keeps it off.
        const uint32_t waves = P.k >= 4 ? P.k / 2 : 1u;
        const uint32_t cmax = cluster_mode == MK_CLUSTER_ON    ? 0xFFFFFFFFu
                              : cluster_mode == MK_CLUSTER_OFF ? 0u
                                                               : waves * cluster_cap;
        return LaunchShape{P.n, P.N, logN, P.k, P.d, P.bg_bit, P.ks_bit, P.t, variant, form, cmax, wait_ns,
                           debug_skip_key_step};
    }
    DeviceKeys dkeys() const {
        // twiddles: [2][N] of 8-byte (NTT) or 16-byte (NTT2) entries; FFT: one [3][N/2] table
        const size_t half = (form == MK_FORM_NTT2 ? 16 : (form == MK_FORM_FFT ? 0 : 8)) * (size_t)P.N;
        const void *split = form == MK_FORM_NTT2 ? (const unsigned char *)d_tw + 32 * (size_t)P.N : nullptr;
        return DeviceKeys{d_tw, (const unsigned char *)d_tw + half, d_bk, d_keyA, d_ks, d_tcws, tc_ws_gates, d_status,
                          split};
    }
};


namespace mk {
// Record a failure message on the context and return `code`.
int fail(mk_ctx *c, int code, const std::string &msg);
int cuda_fail(mk_ctx *c, cudaError_t e, const char *where);
// Build (if needed) and upload the device keys of the context's form.
int ensure_device_keys(mk_ctx *c);
cudaEvent_t take_event(mk_ctx *c);
// Launch `fn` and, when timing is on, bracket it with events on the stream.
template <class F>
cudaError_t timed(mk_ctx *c, int kind, F &&fn) {
    if (!c->timing) return fn();
    cudaEvent_t a = take_event(c), b = take_event(c);
    cudaEventRecord(a, c->stream);
    cudaError_t e = fn();
    cudaEventRecord(b, c->stream);
    c->ev[kind].emplace_back(a, b);
    return e;
}
}  // namespace mk

#define MK_CUDA(c, expr)                                               \
    do {                                                               \
        cudaError_t e__ = (expr);                                      \
        if (e__ != cudaSuccess) return mk::cuda_fail((c), e__, #expr); \
    } while (0)
