// mk_host.cpp -- host runtime of the multi-key TFHE library: parameters,
// counter-based randomness, key generation (MKTFHE.Setup / KeyGen, Sec. 3.2
// of arXiv 2205.05825), SymEnc / SymDec, key layout and upload for the
// kernels, and the C ABI declared in include/mk_tfhe.h.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <tuple>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "mk_ctx.h"

namespace mk {
namespace {

// ------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC 2011).  Stream (seed, tag) is the sequence of 32-bit words
//   word(q) = Philox4x32-10(ctr = (q/4 lo, q/4 hi, tag, 0), key = (seed lo, seed hi))[q % 4].
struct Philox {
    static void block(uint32_t c[4], uint32_t k0, uint32_t k1) {
        for (int r = 0; r < 10; ++r) {
            const uint64_t m0 = (uint64_t)0xD2511F53u * c[0];
            const uint64_t m1 = (uint64_t)0xCD9E8D57u * c[2];
            const uint32_t x0 = (uint32_t)(m1 >> 32) ^ c[1] ^ k0;
            const uint32_t x2 = (uint32_t)(m0 >> 32) ^ c[3] ^ k1;
            c[1] = (uint32_t)m1;
            c[3] = (uint32_t)m0;
            c[0] = x0;
            c[2] = x2;
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
    }
    uint64_t seed;
    uint32_t tag;
    Philox(uint64_t s, uint32_t t) : seed(s), tag(t) {}
    uint32_t word(uint64_t q) const {
        const uint64_t blk = q >> 2;
        uint32_t c[4] = {(uint32_t)blk, (uint32_t)(blk >> 32), tag, 0u};
        block(c, (uint32_t)seed, (uint32_t)(seed >> 32));
        return c[q & 3];
    }
    // Standard normal number q: Box-Muller (cosine branch) on words 2q, 2q+1,
    // u1 = (w0 + 1) / 2^32, u2 = w1 / 2^32.
    double normal(uint64_t q) const {
        const double u1 = ((double)word(2 * q) + 1.0) / 4294967296.0;
        const double u2 = (double)word(2 * q + 1) / 4294967296.0;
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * 3.14159265358979323846 * u2);
    }
    // Torus32 Gaussian noise: round((sigma * 2^32) * g), wrapping.
    uint32_t gauss32(uint64_t q, double sigma) const {
        if (sigma == 0.0) return 0u;
        const double g = normal(q);
        return (uint32_t)(uint64_t)std::llround(sigma * 4294967296.0 * g);
    }
};

enum : uint32_t {
    kTagCrs = 0x01, kTagS = 0x10, kTagZ = 0x11, kTagPkE = 0x12,
    kTagBkR = 0x20, kTagBkF1 = 0x21, kTagBkE1 = 0x22, kTagBkE2 = 0x23,
    kTagKsA = 0x30, kTagKsE = 0x31, kTagEncA = 0x40, kTagEncE = 0x41
};

template <class F>
void parallel_for(size_t count, F &&fn) {
    unsigned nt = std::thread::hardware_concurrency();
    if (nt == 0) nt = 1;
    if (nt > 64) nt = 64;
    if (count < 2 || nt == 1) {
        for (size_t i = 0; i < count; ++i) fn(i);
        return;
    }
    if (nt > count) nt = (unsigned)count;
    std::vector<std::thread> th;
    for (unsigned w = 0; w < nt; ++w)
        th.emplace_back([&, w]() {
            for (size_t i = w; i < count; i += nt) fn(i);
        });
    for (auto &x : th) x.join();
}

uint64_t fnv1a64(const unsigned char *p, size_t n, uint64_t h = 0xcbf29ce484222325ull) {
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

}  // namespace
}  // namespace mk

using namespace mk;

namespace mk {
int fail(mk_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_fail(mk_ctx *c, cudaError_t e, const char *where) {
    return fail(c, MK_EDEVICE, std::string(where) + ": " + cudaGetErrorString(e));
}
}  // namespace mk

namespace {


bool params_supported(const mk_params &p, std::string &why) {
    if (p.k < 1 || p.k > 8) { why = "k must be in [1, 8]"; return false; }
    if (p.N != 256 && p.N != 1024) { why = "N must be 256 or 1024"; return false; }
    if (p.n < 1 || p.n > 4096) { why = "n must be in [1, 4096]"; return false; }
    if (p.d != 3) { why = "the kernels decompose with d = 3 gadget digits"; return false; }
    if (p.bg_bit < 1 || p.bg_bit * p.d > 32 || p.bg_bit > 10) { why = "need 1 <= bg_bit <= 10 and bg_bit*d <= 32"; return false; }
    if (p.ks_bit < 1 || p.t < 1 || p.ks_bit * p.t > 31 || p.ks_bit > 8) { why = "need ks_bit*t <= 31, ks_bit <= 8"; return false; }
    if (!(p.sigma_lwe >= 0) || !(p.sigma_rlwe >= 0)) { why = "sigmas must be >= 0"; return false; }
    return true;
}

}  // namespace
namespace mk {
cudaEvent_t take_event(mk_ctx *c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

}  // namespace mk
namespace {
void release_timing(mk_ctx *c) {
    for (auto &v : c->ev)
        for (auto &pr : v) {
            c->ev_pool.push_back(pr.first);
            c->ev_pool.push_back(pr.second);
        }
    c->ev[0].clear();
    c->ev[1].clear();
}

void free_device(mk_ctx *c) {
    if (c->device < 0) return;
    cudaSetDevice(c->device);
    release_timing(c);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    c->ev_pool.clear();
    cudaFree(c->d_tw);
    cudaFree(c->d_bk);
    cudaFree(c->d_keyA);
    cudaFree(c->d_ks);
    cudaFree(c->d_status);
    c->d_status = nullptr;
    cudaFree(c->d_ext);
    cudaFree(c->d_desc);
    cudaFree(c->d_tcws);
    c->d_tcws = nullptr;
    c->plans.clear();  // graphs and plan buffers go before the capture stream
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    c->capture_stream = nullptr;
    c->tc_ws_gates = 0;
    c->d_tw = nullptr;
    c->d_bk = c->d_keyA = nullptr;
    c->d_ks = c->d_ext = nullptr;
    c->d_desc = nullptr;
    c->scratch_gates = 0;
    c->dev_keys_valid = false;
}

int check_party_public(mk_ctx *c) {
    for (uint32_t i = 0; i < c->P.k; ++i)
        if (!c->party[i].has_public) return fail(c, MK_ESTATE, "public keys of party " + std::to_string(i) + " missing");
    return MK_OK;
}

int check_all_secret(mk_ctx *c) {
    for (uint32_t i = 0; i < c->P.k; ++i)
        if (!c->party[i].has_secret) return fail(c, MK_ESTATE, "secret key of party " + std::to_string(i) + " missing");
    return MK_OK;
}

}  // namespace
namespace mk {
// Build the NTT-domain bootstrapping keys and upload everything the kernels read.
int ensure_device_keys(mk_ctx *c) {
    if (c->device < 0) return fail(c, MK_EDEVICE, "host-only context (device = -1)");
    int rc = check_party_public(c);
    if (rc) return rc;
    if (c->dev_keys_valid) return MK_OK;
    MK_CUDA(c, cudaSetDevice(c->device));
    const uint32_t N = c->P.N, n = c->P.n, k = c->P.k, d = c->P.d;
    const size_t bk_entries = (size_t)k * n * 3 * d;  // polynomials
    const size_t keyA_entries = (size_t)(k + 1) * d;
    // Both forms store 8 bytes per NTT-domain coefficient.
    // 8 bytes per NTT-domain coefficient (NTT forms) or per folded coefficient
    // pair half (FFT form: N/2 double2 = 8 N bytes): the same sizes.
    std::vector<uint64_t> h_bk(bk_entries * N), h_keyA(keyA_entries * N);
    // The largest twiddle tables of the forms: NTT2's [2][N] uint4 plus the
    // per-prime tables [2 directions][2 primes][N] uint2 of the split kernel.
    std::vector<unsigned char> h_tw(4 * (size_t)N * 16);
    // src polynomial of BK entry e and of keyA entry r (negated for the CRS)
    auto bk_src = [&](size_t e) {
        const uint32_t i = (uint32_t)(e / ((size_t)n * 3 * d));
        return c->party[i].bk.data() + (e % ((size_t)n * 3 * d)) * N;
    };
    auto keyA_src = [&](size_t r) {
        const uint32_t jj = (uint32_t)(r / d), l = (uint32_t)(r % d);
        return jj == 0 ? c->crs.data() + (size_t)l * N : c->party[jj - 1].pk.data() + (size_t)l * N;
    };
    if (c->form == MK_FORM_NTT) {
        uint64_t *tw = reinterpret_cast<uint64_t *>(h_tw.data());
        for (uint32_t m = 0; m < N; ++m) {
            tw[m] = c->ntt.psi_rev[m];
            tw[N + m] = c->ntt.psi_inv_rev[m];
        }
        parallel_for(bk_entries, [&](size_t e) { c->ntt.to_ntt(bk_src(e), h_bk.data() + e * N, false, true); });
        for (size_t r = 0; r < keyA_entries; ++r) c->ntt.to_ntt(keyA_src(r), h_keyA.data() + r * N, r < d, true);
    } else if (c->form == MK_FORM_FFT) {
        if (!c->fft.N) c->fft.init(N);
        const uint32_t M = N / 2;
        double *tw = reinterpret_cast<double *>(h_tw.data());  // [3][M] double2: forward, inverse, twist
        for (uint32_t m = 0; m < M; ++m) {
            tw[2 * m] = c->fft.psi_rev[m].real(), tw[2 * m + 1] = c->fft.psi_rev[m].imag();
            tw[2 * (M + m)] = c->fft.psi_inv_rev[m].real(), tw[2 * (M + m) + 1] = c->fft.psi_inv_rev[m].imag();
            tw[2 * (2 * M + m)] = c->fft.theta[m].real(), tw[2 * (2 * M + m) + 1] = c->fft.theta[m].imag();
        }
        parallel_for(bk_entries, [&](size_t e) {
            c->fft.to_device(bk_src(e), reinterpret_cast<double *>(h_bk.data() + e * N), false);
        });
        for (size_t r = 0; r < keyA_entries; ++r)
            c->fft.to_device(keyA_src(r), reinterpret_cast<double *>(h_keyA.data() + r * N), r < d);
    } else if (c->form == MK_FORM_TC) {
        // torus32 words, 4 bytes per coefficient in the same order; [0] = -a
        uint32_t *bk32 = reinterpret_cast<uint32_t *>(h_bk.data());
        uint32_t *kA32 = reinterpret_cast<uint32_t *>(h_keyA.data());
        parallel_for(bk_entries, [&](size_t e) { std::memcpy(bk32 + e * N, bk_src(e), (size_t)N * 4); });
        for (size_t r = 0; r < keyA_entries; ++r) {
            const uint32_t *src = keyA_src(r);
            for (uint32_t m = 0; m < N; ++m) kA32[r * N + m] = r < d ? 0u - src[m] : src[m];
        }
    } else {
        if (!c->ntt_p1.N && !(c->ntt_p1.init(kP1, N) && c->ntt_p2.init(kP2, N)))
            return fail(c, MK_EPARAMS, "ring dimension not supported by the two-prime NTT");
        // Exactness: every product sum, at most (k+1) d N 2^(bg_bit-1) 2^31 in
        // magnitude, must lie inside the CRT range (-p1 p2 / 2, p1 p2 / 2).
        const long double bound = (long double)(k + 1) * d * N * std::ldexp(1.0L, (int)c->P.bg_bit - 1) *
                                  std::ldexp(1.0L, 31);
        if (2.0L * bound >= (long double)kP1 * (long double)kP2)
            return fail(c, MK_EPARAMS, "product sums exceed the two-prime NTT's exact range");
        uint32_t *tw = reinterpret_cast<uint32_t *>(h_tw.data());  // [2][N] of {w1, w2, w1', w2'}
        auto comp = [](uint32_t w, uint32_t p) { return (uint32_t)(((uint64_t)w << 32) / p); };  // Shoup
        for (uint32_t m = 0; m < N; ++m) {
            uint32_t *ef = tw + 4 * (size_t)m, *ei = tw + 4 * ((size_t)N + m);
            const uint32_t f1 = c->ntt_p1.psi_rev[m], f2 = c->ntt_p2.psi_rev[m];
            const uint32_t i1 = c->ntt_p1.psi_inv_rev[m], i2 = c->ntt_p2.psi_inv_rev[m];
            ef[0] = f1, ef[1] = f2, ef[2] = comp(f1, kP1), ef[3] = comp(f2, kP2);
            ei[0] = i1, ei[1] = i2, ei[2] = comp(i1, kP1), ei[3] = comp(i2, kP2);
            uint32_t *sp = tw + 8 * (size_t)N;  // split tables: {w, w'} at ((dir * 2 + prime) * N + m)
            sp[2 * (0 * (size_t)N + m)] = f1, sp[2 * (0 * (size_t)N + m) + 1] = comp(f1, kP1);
            sp[2 * (1 * (size_t)N + m)] = f2, sp[2 * (1 * (size_t)N + m) + 1] = comp(f2, kP2);
            sp[2 * (2 * (size_t)N + m)] = i1, sp[2 * (2 * (size_t)N + m) + 1] = comp(i1, kP1);
            sp[2 * (3 * (size_t)N + m)] = i2, sp[2 * (3 * (size_t)N + m) + 1] = comp(i2, kP2);
        }
        auto dual = [&](const uint32_t *src, uint64_t *dst, bool negate) {
            std::vector<uint32_t> r1(N), r2(N);
            c->ntt_p1.to_device(src, r1.data(), negate);
            c->ntt_p2.to_device(src, r2.data(), negate);
            uint32_t *o = reinterpret_cast<uint32_t *>(dst);  // uint2 {r1, r2} per coefficient
            for (uint32_t j = 0; j < N; ++j) {
                o[2 * j] = r1[j];
                o[2 * j + 1] = r2[j];
            }
        };
        parallel_for(bk_entries, [&](size_t e) { dual(bk_src(e), h_bk.data() + e * N, false); });
        for (size_t r = 0; r < keyA_entries; ++r) dual(keyA_src(r), h_keyA.data() + r * N, r < d);
    }
    if (c->form == MK_FORM_NTT || c->form == MK_FORM_NTT2) {
        // The kernels' key layouts (key_unit_pos, plane_unit_pos).
        //  NTT: 16-byte unit u (elements 2u, 2u + 1) goes to (u % 4) * (N / 8) + u / 4.
        //  NTT2: the {r1, r2} pairs split into a plane of r1 and a plane of r2;
        //  in each, the 16-byte unit u (elements 4u .. 4u + 3) goes to
        //  (u % 2) * (N / 8) + u / 2.
        const bool planes = c->form == MK_FORM_NTT2;
        auto interleave = [N, planes](uint64_t *poly, std::vector<uint64_t> &tmp) {
            tmp.assign(poly, poly + N);
            const uint32_t stride = N / 8;
            if (planes) {
                const uint32_t *src = reinterpret_cast<const uint32_t *>(tmp.data());  // {r1, r2} per element
                uint32_t *dst = reinterpret_cast<uint32_t *>(poly);
                for (uint32_t pl = 0; pl < 2; ++pl)
                    for (uint32_t u = 0; u < N / 4; ++u) {
                        const uint32_t pos = (u & 1) * stride + (u >> 1);
                        for (uint32_t e = 0; e < 4; ++e) dst[pl * N + 4 * pos + e] = src[2 * (4 * u + e) + pl];
                    }
                return;
            }
            for (uint32_t u = 0; u < N / 2; ++u) {
                const uint32_t pos = (u & 3) * stride + (u >> 2);
                poly[2 * pos] = tmp[2 * u];
                poly[2 * pos + 1] = tmp[2 * u + 1];
            }
        };
        parallel_for(bk_entries, [&](size_t e) {
            std::vector<uint64_t> tmp;
            interleave(h_bk.data() + e * N, tmp);
        });
        std::vector<uint64_t> tmp;
        for (size_t r = 0; r < keyA_entries; ++r) interleave(h_keyA.data() + r * N, tmp);
    }
    if (!c->d_tw) MK_CUDA(c, cudaMalloc(&c->d_tw, h_tw.size()));
    if (!c->d_bk) MK_CUDA(c, cudaMalloc(&c->d_bk, h_bk.size() * 8));
    if (!c->d_keyA) MK_CUDA(c, cudaMalloc(&c->d_keyA, h_keyA.size() * 8));
    if (!c->d_ks) MK_CUDA(c, cudaMalloc(&c->d_ks, (size_t)k * c->ks_words() * 4));
    if (!c->d_status) {
        MK_CUDA(c, cudaMalloc(&c->d_status, 16));
        MK_CUDA(c, cudaMemset(c->d_status, 0, 16));
    }
    if (c->form == MK_FORM_TC && !c->d_tcws) {
        const uint32_t gates = kTcWaveGates;
        MK_CUDA(c, cudaMalloc(&c->d_tcws, tc_workspace_bytes(c->shape(), gates)));
        c->tc_ws_gates = gates;
    }
    // Work already enqueued may still read the previous keys.
    MK_CUDA(c, cudaStreamSynchronize(c->stream));
    MK_CUDA(c, cudaMemcpy(c->d_tw, h_tw.data(), h_tw.size(), cudaMemcpyHostToDevice));
    const size_t coef_bytes = c->form == MK_FORM_TC ? 4 : 8;
    MK_CUDA(c, cudaMemcpy(c->d_bk, h_bk.data(), h_bk.size() * coef_bytes, cudaMemcpyHostToDevice));
    MK_CUDA(c, cudaMemcpy(c->d_keyA, h_keyA.data(), h_keyA.size() * coef_bytes, cudaMemcpyHostToDevice));
    for (uint32_t i = 0; i < k; ++i)
        MK_CUDA(c, cudaMemcpy(c->d_ks + (size_t)i * c->ks_words(), c->party[i].ks.data(), c->ks_words() * 4,
                              cudaMemcpyHostToDevice));
    c->cluster_cap = (uint32_t)cluster_capacity(c->shape());
    (void)cudaGetLastError();  // a shape the device cannot host only leaves the capacity at 0
    c->dev_keys_valid = true;
    return MK_OK;
}

}  // namespace mk
namespace {
int ensure_scratch(mk_ctx *c, uint32_t gates) {
    if (gates <= c->scratch_gates) return MK_OK;
    MK_CUDA(c, cudaSetDevice(c->device));
    // Work already enqueued may still read the old buffers.
    MK_CUDA(c, cudaStreamSynchronize(c->stream));
    cudaFree(c->d_ext);
    cudaFree(c->d_desc);
    c->d_ext = nullptr;
    c->d_desc = nullptr;
    c->scratch_gates = 0;
    MK_CUDA(c, cudaMalloc(&c->d_ext, (size_t)gates * c->E() * 4));
    MK_CUDA(c, cudaMalloc(&c->d_desc, (size_t)gates * sizeof(GateDesc)));
    c->scratch_gates = gates;
    return MK_OK;
}

int device_ready(mk_ctx *c, size_t count) {
    int rc = ensure_device_keys(c);
    if (rc) return rc;
    const uint32_t chunk = (uint32_t)std::min<size_t>(count, c->max_batch);
    rc = ensure_scratch(c, chunk ? chunk : 1);
    if (rc) return rc;
    MK_CUDA(c, cudaSetDevice(c->device));
    return MK_OK;
}

enum DescKind { kDescTypes, kDescLin, kDescUniform };

int run_gates(mk_ctx *c, DescKind kind, const void *src, int type, const uint32_t *d_a, const uint32_t *d_b,
              uint32_t *d_out, size_t count) {
    if (count == 0) return MK_OK;
    if (!d_a || !d_b || !d_out) return fail(c, MK_EINVAL, "null ciphertext pointer");
    if (count > 0xFFFFFFFFull / 2) return fail(c, MK_EINVAL, "count too large");
    int rc = device_ready(c, count);
    if (rc) return rc;
    const LaunchShape S = c->shape();
    const DeviceKeys K = c->dkeys();
    for (size_t start = 0; start < count; start += c->max_batch) {
        const uint32_t cnt = (uint32_t)std::min<size_t>(c->max_batch, count - start);
        cudaError_t e;
        if (kind == kDescTypes) e = launch_desc_from_types((const uint8_t *)src, c->d_desc, (uint32_t)start, cnt, c->stream);
        else if (kind == kDescLin) e = launch_desc_from_lin((const mk_lin *)src, c->d_desc, (uint32_t)start, cnt, c->stream);
        else e = launch_desc_uniform(type, c->d_desc, (uint32_t)start, cnt, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "descriptor kernel");
        e = timed(c, MK_KERNEL_BOOTSTRAP,
                  [&] { return launch_bootstrap_ntt(S, K, c->d_desc, d_a, d_b, c->d_ext, cnt, c->stream); });
        if (e != cudaSuccess) return cuda_fail(c, e, "bootstrap kernel");
        e = timed(c, MK_KERNEL_KEYSWITCH,
                  [&] { return launch_keyswitch(S, K, c->d_desc, c->d_ext, d_out, cnt, c->stream); });
        if (e != cudaSuccess) return cuda_fail(c, e, "keyswitch kernel");
    }
    return MK_OK;
}

int get_plan(mk_ctx *c, int op, uint32_t k, uint32_t pairs, CircuitPlan **out) {
    auto key = std::make_tuple(op, k, pairs, c->circuit_style);
    auto it = c->plans.find(key);
    if (it != c->plans.end()) {
        *out = it->second.get();
        return MK_OK;
    }
    auto plan = std::make_unique<CircuitPlan>();
    if (!build_netlist(op, k, c->circuit_style, plan->net)) return fail(c, MK_EINVAL, "unsupported operator or kbits");
    const Netlist &net = plan->net;
    const std::vector<uint32_t> lev = netlist_levels(net);
    const uint32_t L = lev.empty() ? 0 : *std::max_element(lev.begin(), lev.end());
    const uint32_t base = 2 + net.ka + net.kb;
    plan->pairs = pairs;
    plan->n_wires = base + (uint32_t)net.gates.size();
    std::vector<std::vector<uint32_t>> by_level(L + 1);
    for (uint32_t g = 0; g < net.gates.size(); ++g) by_level[lev[g]].push_back(g);
    std::vector<GateDesc> desc;
    desc.reserve((size_t)net.gates.size() * pairs);
    plan->level_off.push_back(0);
    for (uint32_t l = 1; l <= L; ++l) {
        for (uint32_t g : by_level[l]) {
            const mk_gate_rec &r = net.gates[g];
            const mk_lin lin = gate_lin(r);
            for (uint32_t p = 0; p < pairs; ++p)
                desc.push_back(GateDesc{(uint32_t)r.a * pairs + p, (uint32_t)r.b * pairs + p, lin.cst, lin.s1, lin.s2,
                                        (base + g) * pairs + p});
        }
        plan->level_off.push_back((uint32_t)desc.size());
        plan->max_level = std::max<uint32_t>(plan->max_level, (uint32_t)(by_level[l].size() * pairs));
    }
    std::vector<int32_t> outs;
    for (const Wire &w : net.outputs) outs.push_back(w.w * 2 + w.neg);
    MK_CUDA(c, cudaSetDevice(c->device));
    MK_CUDA(c, cudaMalloc(&plan->d_desc, std::max<size_t>(desc.size(), 1) * sizeof(GateDesc)));
    MK_CUDA(c, cudaMalloc(&plan->d_pool, (size_t)plan->n_wires * pairs * c->W() * 4));
    MK_CUDA(c, cudaMalloc(&plan->d_ext, (size_t)std::max<uint32_t>(plan->max_level, 1) * c->E() * 4));
    MK_CUDA(c, cudaMalloc(&plan->d_outs, outs.size() * sizeof(int32_t)));
    MK_CUDA(c, cudaMalloc(&plan->d_ready, (size_t)plan->n_wires * pairs * sizeof(uint32_t)));
    MK_CUDA(c, cudaMemset(plan->d_ready, 0, (size_t)plan->n_wires * pairs * sizeof(uint32_t)));
    MK_CUDA(c, cudaMalloc(&plan->d_ctl, 4 * sizeof(uint32_t)));
    plan->levels = L;
    MK_CUDA(c, cudaMemcpy(plan->d_desc, desc.data(), desc.size() * sizeof(GateDesc), cudaMemcpyHostToDevice));
    MK_CUDA(c, cudaMemcpy(plan->d_outs, outs.data(), outs.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    *out = plan.get();
    c->plans[key] = std::move(plan);
    return MK_OK;
}

// Capture the level loop of a plan on the context's capture stream.  On any
// failure the plan keeps no graph and the caller launches directly.
void capture_levels(mk_ctx *c, CircuitPlan *pl, const LaunchShape &S, const DeviceKeys &K) {
    if (!c->capture_stream && cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
        c->capture_stream = nullptr;
        return;
    }
    cudaStream_t cs = c->capture_stream;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) return;
    cudaError_t e = cudaSuccess;
    for (size_t l = 0; e == cudaSuccess && l + 1 < pl->level_off.size(); ++l) {
        const uint32_t off = pl->level_off[l], cnt = pl->level_off[l + 1] - off;
        e = launch_bootstrap_ntt(S, K, pl->d_desc + off, pl->d_pool, pl->d_pool, pl->d_ext, cnt, cs);
        if (e == cudaSuccess) e = launch_keyswitch(S, K, pl->d_desc + off, pl->d_ext, pl->d_pool, cnt, cs);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess && ee == cudaSuccess && g) {
        if (cudaGraphInstantiate(&pl->graph, g, 0) != cudaSuccess) pl->graph = nullptr;
    }
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();  // a failed capture leaves no sticky error: the caller launches directly
    if (pl->graph) {
        pl->graph_form = c->form;
        pl->graph_variant = c->variant;
        pl->graph_cluster = S.cluster_max;
        pl->graph_keys = K;
    }
}

// Evaluate operator `op` on `pairs` operand pairs; outputs [pairs][n_outputs],
// or, with d_out2, the first half of the outputs into d_out and the second
// half into d_out2 (quotient and remainder).
int run_circuit(mk_ctx *c, int op, uint32_t k, const uint32_t *d_a, const uint32_t *d_b, uint32_t *d_out,
                size_t pairs, uint32_t *d_out2 = nullptr) {
    if (pairs == 0) return MK_OK;
    if (!d_a || !d_b || !d_out) return fail(c, MK_EINVAL, "null pointer");
    if (k < 2 || k > 64) return fail(c, MK_EINVAL, "kbits must be in [2, 64]");
    if (pairs > (1u << 20)) return fail(c, MK_EINVAL, "too many pairs");
    int rc = ensure_device_keys(c);
    if (rc) return rc;
    CircuitPlan *pl = nullptr;
    rc = get_plan(c, op, k, (uint32_t)pairs, &pl);
    if (rc) return rc;
    const uint32_t P = (uint32_t)pairs, W = (uint32_t)c->W();
    const LaunchShape S = c->shape();
    const DeviceKeys K = c->dkeys();
    cudaError_t e = launch_circuit_consts(pl->d_pool, P, W, c->stream);
    if (e == cudaSuccess) e = launch_circuit_inputs(pl->d_pool, d_a, k, P, 2, W, c->stream);
    if (e == cudaSuccess) e = launch_circuit_inputs(pl->d_pool, d_b, k, P, 2 + k, W, c->stream);
    // One persistent launch over every (gate, pair) item (NTT forms), or one
    // launch pair per level.  AUTO takes the level loop: on these netlists
    // every pair advances through the levels in step, so the persistent
    // launch overlaps little that the level barriers hold back, and its
    // per-gate key switch (each gate reads its own key-switch rows) costs more
    // than the batched one (measured slower for every operator and width).
    const uint32_t items = (uint32_t)pl->net.gates.size() * P;
    const bool ntt_form = c->form == MK_FORM_NTT || c->form == MK_FORM_NTT2;
    const bool persistent = ntt_form && c->circuit_exec == MK_EXEC_PERSISTENT;
    bool replayed = false;
    if (e == cudaSuccess && persistent) {
        if (++pl->epoch == 0) ++pl->epoch;  // 0 marks rows never written
        NetlistArgs A{pl->d_desc, items, pl->d_pool, (2 + pl->net.ka + pl->net.kb) * P, pl->d_ready, pl->epoch,
                      pl->d_ctl, pl->d_ctl + 1, pl->d_ctl + 2, c->debug_skip_item};
        e = cudaMemsetAsync(pl->d_ctl, 0, 3 * sizeof(uint32_t), c->stream);
        if (e == cudaSuccess)
            e = timed(c, MK_KERNEL_BOOTSTRAP, [&] { return launch_netlist(S, K, A, c->sm_count, c->stream); });
        replayed = true;
    }
    // The level loop reads and writes only the plan's own buffers, so it is
    // captured once as a CUDA graph (per form, variant and key buffers) and
    // replayed; the tensor form (thousands of launches per level) and timed
    // runs launch directly.
    if (e == cudaSuccess && !replayed && c->use_graphs && !c->timing && c->form != MK_FORM_TC) {
        if (pl->graph && (pl->graph_form != c->form || pl->graph_variant != c->variant ||
                          pl->graph_cluster != S.cluster_max ||
                          std::memcmp(&pl->graph_keys, &K, sizeof(K)) != 0)) {
            cudaGraphExecDestroy(pl->graph);
            pl->graph = nullptr;
        }
        if (!pl->graph) capture_levels(c, pl, S, K);
        if (pl->graph) {
            e = cudaGraphLaunch(pl->graph, c->stream);
            replayed = true;
        }
    }
    for (size_t l = 0; !replayed && e == cudaSuccess && l + 1 < pl->level_off.size(); ++l) {
        const uint32_t off = pl->level_off[l], cnt = pl->level_off[l + 1] - off;
        e = timed(c, MK_KERNEL_BOOTSTRAP, [&] {
            return launch_bootstrap_ntt(S, K, pl->d_desc + off, pl->d_pool, pl->d_pool, pl->d_ext, cnt, c->stream);
        });
        if (e == cudaSuccess)
            e = timed(c, MK_KERNEL_KEYSWITCH,
                      [&] { return launch_keyswitch(S, K, pl->d_desc + off, pl->d_ext, pl->d_pool, cnt, c->stream); });
    }
    const uint32_t nout = (uint32_t)pl->net.outputs.size();
    if (e == cudaSuccess && !d_out2) e = launch_circuit_outputs(d_out, pl->d_pool, pl->d_outs, nout, P, W, c->stream);
    if (e == cudaSuccess && d_out2) {
        e = launch_circuit_outputs(d_out, pl->d_pool, pl->d_outs, nout / 2, P, W, c->stream);
        if (e == cudaSuccess)
            e = launch_circuit_outputs(d_out2, pl->d_pool, pl->d_outs + nout / 2, nout - nout / 2, P, W, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "circuit");
    return MK_OK;
}

// Random ciphertexts (every CMux step active, as for real multi-party
// inputs): two operand blocks of cnt rows each, for the tuners.
int sample_inputs(mk_ctx *c, uint32_t cnt, uint32_t **d_in) {
    const size_t W = c->W();
    std::vector<uint32_t> h((size_t)2 * cnt * W);
    const Philox r(0xA5A5A5A5ull, 0x7F);
    for (size_t q = 0; q < h.size(); ++q) h[q] = r.word(q);
    MK_CUDA(c, cudaMalloc(d_in, h.size() * 4));
    const cudaError_t e = cudaMemcpy(*d_in, h.data(), h.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(*d_in);
        *d_in = nullptr;
        return cuda_fail(c, e, "tuner inputs");
    }
    return MK_OK;
}

// One untimed and one timed bootstrap launch of cnt NAND gates on the
// context's current form and variant (needs device_ready(c, cnt)).
cudaError_t time_sample(mk_ctx *c, uint32_t cnt, const uint32_t *d_in, float *ms) {
    const size_t W = c->W();
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaError_t err = launch_desc_uniform(MK_NAND, c->d_desc, 0, cnt, c->stream);
    if (err == cudaSuccess)
        err = launch_bootstrap_ntt(c->shape(), c->dkeys(), c->d_desc, d_in, d_in + (size_t)cnt * W, c->d_ext, cnt,
                                   c->stream);
    cudaEventRecord(a, c->stream);
    if (err == cudaSuccess)
        err = launch_bootstrap_ntt(c->shape(), c->dkeys(), c->d_desc, d_in, d_in + (size_t)cnt * W, c->d_ext, cnt,
                                   c->stream);
    cudaEventRecord(b, c->stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(b);
    *ms = 0;
    if (err == cudaSuccess) cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return err;
}

}  // namespace

// =================================================================== C ABI
extern "C" {

int mk_params_preset(int preset, uint32_t k, mk_params *out) {
    if (!out || k == 0) return MK_EINVAL;
    mk_params p{};
    p.k = k;
    p.bg_bit = 8;
    p.d = 3;
    p.ks_bit = 2;
    p.t = 8;
    if (preset == MK_PRESET_TOY) {
        p.n = 64;
        p.N = 256;
        p.sigma_lwe = std::ldexp(1.0, -25);
        p.sigma_rlwe = std::ldexp(1.0, -25);
    } else if (preset == MK_PRESET_FULL) {
        p.n = 560;
        p.N = 1024;
        p.sigma_lwe = std::ldexp(1.0, -15);
        p.sigma_rlwe = std::ldexp(1.0, k == 1 ? -28 : (k <= 3 ? -30 : -32));
    } else if (preset == MK_PRESET_PAPER) {
        p.n = 560;
        p.N = 1024;
        p.bg_bit = 9;
        p.sigma_lwe = 3.05e-5;
        p.sigma_rlwe = 3.72e-9;
    } else {
        return MK_EINVAL;
    }
    *out = p;
    return MK_OK;
}

int mk_ctx_create(const mk_params *params, uint64_t crs_seed, int device, void *stream, mk_ctx **out) {
    if (!params || !out) return MK_EINVAL;
    *out = nullptr;
    std::string why;
    if (!params_supported(*params, why)) return MK_EPARAMS;
    mk_ctx *c = new (std::nothrow) mk_ctx();
    if (!c) return MK_ENOMEM;
    c->P = *params;
    c->P.reserved = 0;
    while ((1u << c->logN) < c->P.N) ++c->logN;
    c->crs_seed = crs_seed;
    c->device = device;
    c->stream = (cudaStream_t)stream;
    if (!c->ntt.init(c->P.N)) {
        delete c;
        return MK_EPARAMS;
    }
    c->party.resize(c->P.k);
    // Setup: the common reference string a in T_N[X]^d.
    const uint32_t N = c->P.N, d = c->P.d;
    c->crs.resize((size_t)d * N);
    Philox crs_rng(crs_seed, kTagCrs);
    for (size_t q = 0; q < c->crs.size(); ++q) c->crs[q] = crs_rng.word(q);
    if (device >= 0) {
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || device >= ndev) {
            delete c;
            return MK_EDEVICE;
        }
        if (cudaSetDevice(device) != cudaSuccess) {
            delete c;
            return MK_EDEVICE;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && sms > 0)
            c->sm_count = (uint32_t)sms;
    }
    *out = c;
    return MK_OK;
}

int mk_ctx_destroy(mk_ctx *c) {
    if (!c) return MK_EINVAL;
    if (c->device >= 0) {
        cudaSetDevice(c->device);
        cudaStreamSynchronize(c->stream);
    }
    free_device(c);
    delete c;
    return MK_OK;
}

int mk_ctx_set_stream(mk_ctx *c, void *stream) {
    if (!c) return MK_EINVAL;
    c->stream = (cudaStream_t)stream;
    return MK_OK;
}

int mk_ctx_get_params(const mk_ctx *c, mk_params *out) {
    if (!c || !out) return MK_EINVAL;
    *out = c->P;
    return MK_OK;
}

int mk_ctx_set_form(mk_ctx *c, int form) {
    if (!c) return MK_EINVAL;
    if (form != MK_FORM_NTT && form != MK_FORM_NTT2 && form != MK_FORM_FFT && form != MK_FORM_TC)
        return fail(c, MK_EINVAL, "unknown product form");
    if (form == MK_FORM_TC) {
        LaunchShape S = c->shape();
        S.form = form;
        if (!tc_shape_supported(S))
            return fail(c, MK_EPARAMS, "the tensor form needs N in {256, 1024}, d = 3 and bg_bit <= 8");
    }
    if (form != c->form) c->dev_keys_valid = false;  // the NTT-domain keys are rebuilt on next use
    c->form = form;
    return MK_OK;
}

int mk_ctx_get_form(const mk_ctx *c, int *form) {
    if (!c || !form) return MK_EINVAL;
    *form = c->form;
    return MK_OK;
}

int mk_ctx_set_cluster(mk_ctx *c, int mode) {
    if (!c) return MK_EINVAL;
    if (mode != MK_CLUSTER_AUTO && mode != MK_CLUSTER_OFF && mode != MK_CLUSTER_ON)
        return fail(c, MK_EINVAL, "cluster mode must be MK_CLUSTER_AUTO, _OFF or _ON");
    c->cluster_mode = mode;
    return MK_OK;
}

int mk_debug_fault(mk_ctx *c, int kind, int64_t arg, uint64_t wait_ns) {
    if (!c) return MK_EINVAL;
    if (kind != MK_FAULT_NONE && kind != MK_FAULT_SKIP_KEY_STEP && kind != MK_FAULT_SKIP_DIGIT_TILE &&
        kind != MK_FAULT_SKIP_WIRE_READY)
        return fail(c, MK_EINVAL, "unknown fault kind");
    if (kind != MK_FAULT_NONE && arg < 0) return fail(c, MK_EINVAL, "fault argument must be >= 0");
    c->debug_skip_item = kind == MK_FAULT_SKIP_WIRE_READY ? arg : -1;
    if (kind == MK_FAULT_SKIP_DIGIT_TILE && c->device < 0) return fail(c, MK_EDEVICE, "host-only context");
    c->wait_ns = wait_ns ? wait_ns : 1000000000ull;
    c->debug_skip_key_step = kind == MK_FAULT_SKIP_KEY_STEP ? arg : -1;
    if (c->device >= 0) {
        MK_CUDA(c, cudaSetDevice(c->device));
        MK_CUDA(c, cudaStreamSynchronize(c->stream));
        MK_CUDA(c, tc05_arm_skip(kind == MK_FAULT_SKIP_DIGIT_TILE ? (uint32_t)arg + 1 : 0u));
    }
    // captured level loops hold the old launch parameters
    for (auto &kv : c->plans)
        if (kv.second->graph) {
            cudaGraphExecDestroy(kv.second->graph);
            kv.second->graph = nullptr;
        }
    return MK_OK;
}

int mk_ctx_set_circuit_exec(mk_ctx *c, int mode) {
    if (!c) return MK_EINVAL;
    if (mode != MK_EXEC_AUTO && mode != MK_EXEC_LEVELS && mode != MK_EXEC_PERSISTENT)
        return fail(c, MK_EINVAL, "circuit execution must be MK_EXEC_AUTO, _LEVELS or _PERSISTENT");
    c->circuit_exec = mode;
    return MK_OK;
}

int mk_ctx_set_graphs(mk_ctx *c, int on) {
    if (!c) return MK_EINVAL;
    c->use_graphs = on != 0;
    return MK_OK;
}

int mk_ctx_set_circuit_style(mk_ctx *c, int style) {
    if (!c) return MK_EINVAL;
    if (style != MK_CIRCUIT_ARRAY && style != MK_CIRCUIT_SHALLOW && style != MK_CIRCUIT_PAPER &&
        style != MK_CIRCUIT_NAND)
        return fail(c, MK_EINVAL, "unknown circuit style");
    c->circuit_style = style;
    return MK_OK;
}

int mk_ctx_get_circuit_style(const mk_ctx *c, int *style) {
    if (!c || !style) return MK_EINVAL;
    *style = c->circuit_style;
    return MK_OK;
}

int mk_ctx_set_batch(mk_ctx *c, uint32_t max_gates) {
    if (!c || max_gates == 0 || max_gates > (1u << 20)) return c ? fail(c, MK_EINVAL, "batch must be in [1, 2^20]") : MK_EINVAL;
    c->max_batch = max_gates;
    return MK_OK;
}

int mk_ctx_set_variant(mk_ctx *c, int v) {
    if (!c) return MK_EINVAL;
    if (v < 0 || v >= kNumVariants) return fail(c, MK_EINVAL, "variant out of range");
    c->variant = v;
    return MK_OK;
}

int mk_ctx_get_variant(const mk_ctx *c, int *v) {
    if (!c || !v) return MK_EINVAL;
    *v = c->variant;
    return MK_OK;
}

int mk_autotune(mk_ctx *c, uint32_t sample_gates, int *best, float *ms_out) {
    if (!c || sample_gates == 0) return MK_EINVAL;
    int rc = device_ready(c, sample_gates);
    if (rc) return rc;
    if (c->form == MK_FORM_FFT) {  // one kernel serves every variant number
        if (ms_out)
            for (int v = 0; v < kNumVariants; ++v) ms_out[v] = 0.f;
        if (best) *best = c->variant;
        return MK_OK;
    }
    // the tensor form has two engines: variant 0 (mma.sync) and 1 (tcgen05)
    const int nvar = c->form == MK_FORM_TC ? 2 : kNumVariants;
    if (ms_out)
        for (int v = nvar; v < kNumVariants; ++v) ms_out[v] = 0.f;
    const uint32_t cnt = std::min<uint32_t>(sample_gates, c->max_batch);
    uint32_t *d_in = nullptr;
    rc = sample_inputs(c, cnt, &d_in);
    if (rc) return rc;
    int bestv = c->variant;
    float bestms = 1e30f;
    cudaError_t err = cudaSuccess;
    const int saved = c->variant;
    for (int v = 0; v < nvar && err == cudaSuccess; ++v) {
        c->variant = v;
        float ms = 0;
        err = time_sample(c, cnt, d_in, &ms);
        if (ms_out) ms_out[v] = ms;
        if (err == cudaSuccess && ms < bestms) {
            bestms = ms;
            bestv = v;
        }
    }
    c->variant = (err == cudaSuccess) ? bestv : saved;
    cudaFree(d_in);
    if (err != cudaSuccess) return cuda_fail(c, err, "autotune");
    if (best) *best = c->variant;
    return MK_OK;
}

int mk_autotune_form(mk_ctx *c, uint32_t sample_gates, uint32_t forms, int *best_form, float *ms_out) {
    if (!c) return MK_EINVAL;
    if (sample_gates == 0 || forms == 0 || (forms >> MK_NUM_FORMS))
        return fail(c, MK_EINVAL, "sample_gates must be positive and forms a non-empty set of MK_FORM_* bits");
    if (ms_out)
        for (int f = 0; f < MK_NUM_FORMS; ++f) ms_out[f] = 0.f;
    const int saved_form = c->form, saved_variant = c->variant;
    int bestf = -1, bestv = saved_variant;
    float bestms = 1e30f;
    for (int f = 0; f < MK_NUM_FORMS; ++f) {
        if (!((forms >> f) & 1u)) continue;
        if (mk_ctx_set_form(c, f) != MK_OK) continue;  // not supported by these parameters
        int v = c->variant;
        int rc = mk_autotune(c, sample_gates, &v, nullptr);
        uint32_t *d_in = nullptr;
        const uint32_t cnt = std::min<uint32_t>(sample_gates, c->max_batch);
        if (rc == MK_OK) rc = sample_inputs(c, cnt, &d_in);
        float ms = 0;
        if (rc == MK_OK) {
            const cudaError_t err = time_sample(c, cnt, d_in, &ms);
            cudaFree(d_in);
            if (err != cudaSuccess) rc = cuda_fail(c, err, "form autotune");
        }
        if (rc != MK_OK) {
            mk_ctx_set_form(c, saved_form);
            c->variant = saved_variant;
            return rc;
        }
        if (ms_out) ms_out[f] = ms;
        if (ms < bestms) {
            bestms = ms;
            bestf = f;
            bestv = v;
        }
    }
    if (bestf < 0) {
        mk_ctx_set_form(c, saved_form);
        c->variant = saved_variant;
        return fail(c, MK_EPARAMS, "none of the requested product forms supports these parameters");
    }
    mk_ctx_set_form(c, bestf);
    c->variant = bestv;
    if (best_form) *best_form = bestf;
    return MK_OK;
}

const char *mk_last_error(const mk_ctx *c) {
    if (!c) return "null context";
    return c->err.c_str();
}

int mk_sync(mk_ctx *c) {
    if (!c) return MK_EINVAL;
    if (c->device < 0) return MK_OK;
    MK_CUDA(c, cudaSetDevice(c->device));
    MK_CUDA(c, cudaStreamSynchronize(c->stream));
    MK_CUDA(c, cudaGetLastError());
    if (c->form == MK_FORM_TC && c->dev_keys_valid) {  // the tcgen05 engine's bounded waits
        unsigned int timeout = 0;
        MK_CUDA(c, tc05_error(&timeout, true));
        if (timeout) return fail(c, MK_ETIMEOUT, "a bounded wait of the tensor-core product kernel gave up");
    }
    if (c->d_status) {  // bounded waits of the staged and cluster blind rotations and the persistent operator launch
        uint32_t st = 0;
        MK_CUDA(c, cudaMemcpy(&st, c->d_status, sizeof(st), cudaMemcpyDeviceToHost));
        if (st) {
            MK_CUDA(c, cudaMemset(c->d_status, 0, sizeof(st)));
            if (st & kStatusStaged)
                return fail(c, MK_ETIMEOUT, "a bounded wait of the staged blind rotation for a key copy gave up");
            if (st & kStatusCluster)
                return fail(c, MK_ETIMEOUT, "a bounded wait of the cluster blind rotation for a key copy gave up");
            return fail(c, MK_ETIMEOUT, "the persistent operator launch made no progress within its bound");
        }
    }
    return MK_OK;
}

// ------------------------------------------------------------------- keys
int mk_keygen(mk_ctx *c, uint32_t party, uint64_t seed) {
    if (!c) return MK_EINVAL;
    if (party >= c->P.k) return fail(c, MK_EINVAL, "party index out of range");
    const uint32_t n = c->P.n, N = c->P.N, d = c->P.d, t = c->P.t;
    const uint32_t nb = (1u << c->P.ks_bit) - 1;
    PartyKeys K;
    K.s.resize(n);
    K.z.resize(N);
    K.pk.resize((size_t)d * N);
    K.bk.resize(c->bk_words());
    K.ks.resize(c->ks_words());
    const Philox rs(seed, kTagS), rz(seed, kTagZ), rpe(seed, kTagPkE);
    for (uint32_t j = 0; j < n; ++j) K.s[j] = rs.word(j) & 1u;
    for (uint32_t m = 0; m < N; ++m) K.z[m] = rz.word(m) & 1u;
    const HostNtt &T = c->ntt;
    std::vector<uint64_t> z_hat(N);
    for (uint32_t m = 0; m < N; ++m) z_hat[m] = K.z[m];
    T.forward(z_hat.data());
    {
        std::vector<uint64_t> tmp;
        std::vector<uint32_t> prod(N);
        for (uint32_t l = 0; l < d; ++l) {
            T.mul_binary(z_hat.data(), c->crs.data() + (size_t)l * N, prod.data(), tmp);
            for (uint32_t m = 0; m < N; ++m)
                K.pk[(size_t)l * N + m] = (0u - prod[m]) + rpe.gauss32((uint64_t)l * N + m, c->P.sigma_rlwe);
        }
    }
    // BK_j = UniEnc(s_j; z): r binary, d_l = r*a_l + s_j*g_l + e1, f1_l uniform, f0_l = -z*f1_l + r*g_l + e2.
    const Philox rr(seed, kTagBkR), rf1(seed, kTagBkF1), re1(seed, kTagBkE1), re2(seed, kTagBkE2);
    parallel_for(n, [&](size_t jj) {
        const uint32_t j = (uint32_t)jj;
        std::vector<uint64_t> r_hat(N), tmp;
        std::vector<uint32_t> r(N), prod(N);
        for (uint32_t m = 0; m < N; ++m) {
            r[m] = rr.word((uint64_t)j * N + m) & 1u;
            r_hat[m] = r[m];
        }
        T.forward(r_hat.data());
        uint32_t *ent = K.bk.data() + (size_t)j * 3 * d * N;
        for (uint32_t l = 0; l < d; ++l) {
            const uint64_t qb = ((uint64_t)j * d + l) * N;
            const uint32_t g = 1u << (32 - c->P.bg_bit * (l + 1));
            uint32_t *dv = ent + (size_t)l * N, *f0 = ent + (size_t)(d + l) * N, *f1 = ent + (size_t)(2 * d + l) * N;
            T.mul_binary(r_hat.data(), c->crs.data() + (size_t)l * N, prod.data(), tmp);
            for (uint32_t m = 0; m < N; ++m) dv[m] = prod[m] + re1.gauss32(qb + m, c->P.sigma_rlwe);
            dv[0] += K.s[j] * g;
            for (uint32_t m = 0; m < N; ++m) f1[m] = rf1.word(qb + m);
            T.mul_binary(z_hat.data(), f1, prod.data(), tmp);
            for (uint32_t m = 0; m < N; ++m) f0[m] = (0u - prod[m]) + r[m] * g + re2.gauss32(qb + m, c->P.sigma_rlwe);
        }
    });
    // KS[j][l][delta-1] = LWE_s(delta * z_j * 2^(32 - ks_bit*(l+1))).
    const Philox rka(seed, kTagKsA), rke(seed, kTagKsE);
    const size_t rows = (size_t)N * t * nb;
    parallel_for((rows + 255) / 256, [&](size_t blk) {
        for (size_t row = blk * 256; row < std::min(rows, (blk + 1) * 256); ++row) {
            const uint32_t delta = (uint32_t)(row % nb) + 1;
            const uint32_t l = (uint32_t)((row / nb) % t);
            const uint32_t j = (uint32_t)(row / ((size_t)nb * t));
            uint32_t *dst = K.ks.data() + row * (n + 1);
            uint32_t dot = 0;
            for (uint32_t x = 0; x < n; ++x) {
                dst[x] = rka.word((uint64_t)row * n + x);
                dot += dst[x] * K.s[x];
            }
            dst[n] = (0u - dot) + delta * K.z[j] * (1u << (32 - c->P.ks_bit * (l + 1))) + rke.gauss32(row, c->P.sigma_lwe);
        }
    });
    K.has_public = K.has_secret = true;
    c->party[party] = std::move(K);
    c->dev_keys_valid = false;
    return MK_OK;
}

int mk_import_crs(mk_ctx *c, const uint32_t *h_crs) {
    if (!c || !h_crs) return MK_EINVAL;
    std::memcpy(c->crs.data(), h_crs, c->crs.size() * 4);
    c->dev_keys_valid = false;
    return MK_OK;
}

int mk_import_party(mk_ctx *c, uint32_t party, const uint32_t *s, const uint32_t *z, const uint32_t *pk,
                    const uint32_t *bk, const uint32_t *ks) {
    if (!c) return MK_EINVAL;
    if (party >= c->P.k) return fail(c, MK_EINVAL, "party index out of range");
    if (!pk || !bk || !ks) return fail(c, MK_EINVAL, "public key pointers must not be null");
    if ((s == nullptr) != (z == nullptr)) return fail(c, MK_EINVAL, "give both secrets or neither");
    PartyKeys K;
    K.pk.assign(pk, pk + c->pk_words());
    K.bk.assign(bk, bk + c->bk_words());
    K.ks.assign(ks, ks + c->ks_words());
    K.has_public = true;
    if (s) {
        K.s.assign(s, s + c->P.n);
        K.z.assign(z, z + c->P.N);
        K.has_secret = true;
    }
    c->party[party] = std::move(K);
    c->dev_keys_valid = false;
    return MK_OK;
}

int mk_export_crs(const mk_ctx *c, uint32_t *h_crs) {
    if (!c || !h_crs) return MK_EINVAL;
    std::memcpy(h_crs, c->crs.data(), c->crs.size() * 4);
    return MK_OK;
}

int mk_export_party(const mk_ctx *cc, uint32_t party, uint32_t *s, uint32_t *z, uint32_t *pk, uint32_t *bk,
                    uint32_t *ks) {
    mk_ctx *c = const_cast<mk_ctx *>(cc);
    if (!c) return MK_EINVAL;
    if (party >= c->P.k) return fail(c, MK_EINVAL, "party index out of range");
    const PartyKeys &K = c->party[party];
    if ((pk || bk || ks) && !K.has_public) return fail(c, MK_ESTATE, "no public keys for this party");
    if ((s || z) && !K.has_secret) return fail(c, MK_ESTATE, "no secret keys for this party");
    if (s) std::memcpy(s, K.s.data(), K.s.size() * 4);
    if (z) std::memcpy(z, K.z.data(), K.z.size() * 4);
    if (pk) std::memcpy(pk, K.pk.data(), K.pk.size() * 4);
    if (bk) std::memcpy(bk, K.bk.data(), K.bk.size() * 4);
    if (ks) std::memcpy(ks, K.ks.data(), K.ks.size() * 4);
    return MK_OK;
}

namespace {
struct BlobHeader {
    char magic[8];
    uint32_t version, header_bytes;
    mk_params params;
    uint64_t crs_seed;
    uint32_t party_mask, secret_mask;
    uint64_t payload_words;
};
const char kMagic[8] = {'M', 'K', 'T', 'F', 'H', 'E', 'K', '1'};
}  // namespace

int mk_save_keys(const mk_ctx *cc, int include_secrets, void *h_blob, size_t cap, size_t *len) {
    mk_ctx *c = const_cast<mk_ctx *>(cc);
    if (!c || !len) return MK_EINVAL;
    BlobHeader H{};
    std::memcpy(H.magic, kMagic, 8);
    H.version = 1;
    H.header_bytes = sizeof(BlobHeader);
    H.params = c->P;
    H.crs_seed = c->crs_seed;
    size_t words = c->crs.size();
    for (uint32_t i = 0; i < c->P.k; ++i) {
        const PartyKeys &K = c->party[i];
        if (!K.has_public) continue;
        H.party_mask |= 1u << i;
        words += c->pk_words() + c->bk_words() + c->ks_words();
        if (include_secrets && K.has_secret) {
            H.secret_mask |= 1u << i;
            words += c->P.n + c->P.N;
        }
    }
    H.payload_words = words;
    const size_t total = sizeof(BlobHeader) + words * 4 + 8;
    *len = total;
    if (!h_blob) return MK_OK;
    if (cap < total) return fail(c, MK_EINVAL, "blob buffer too small");
    unsigned char *p = (unsigned char *)h_blob;
    std::memcpy(p, &H, sizeof(H));
    size_t off = sizeof(H);
    auto put = [&](const std::vector<uint32_t> &v) {
        std::memcpy(p + off, v.data(), v.size() * 4);
        off += v.size() * 4;
    };
    put(c->crs);
    for (uint32_t i = 0; i < c->P.k; ++i) {
        const PartyKeys &K = c->party[i];
        if (!(H.party_mask >> i & 1)) continue;
        if (H.secret_mask >> i & 1) {
            put(K.s);
            put(K.z);
        }
        put(K.pk);
        put(K.bk);
        put(K.ks);
    }
    const uint64_t h = fnv1a64(p, off);
    std::memcpy(p + off, &h, 8);
    return MK_OK;
}

int mk_load_keys(mk_ctx *c, const void *h_blob, size_t len) {
    if (!c || !h_blob) return MK_EINVAL;
    if (len < sizeof(BlobHeader) + 8) return fail(c, MK_EFORMAT, "blob too short");
    BlobHeader H;
    std::memcpy(&H, h_blob, sizeof(H));
    if (std::memcmp(H.magic, kMagic, 8) != 0 || H.version != 1 || H.header_bytes != sizeof(BlobHeader))
        return fail(c, MK_EFORMAT, "bad blob header");
    mk_params a = H.params, b = c->P;
    a.reserved = b.reserved = 0;
    if (std::memcmp(&a, &b, sizeof(mk_params)) != 0) return fail(c, MK_EFORMAT, "blob parameters differ from the context's");
    if (sizeof(BlobHeader) + H.payload_words * 4 + 8 != len) return fail(c, MK_EFORMAT, "blob size mismatch");
    const unsigned char *p = (const unsigned char *)h_blob;
    uint64_t stored;
    std::memcpy(&stored, p + len - 8, 8);
    if (fnv1a64(p, len - 8) != stored) return fail(c, MK_EFORMAT, "blob checksum mismatch");
    size_t expect = c->crs.size();
    for (uint32_t i = 0; i < c->P.k; ++i) {
        if (H.party_mask >> i & 1) expect += c->pk_words() + c->bk_words() + c->ks_words();
        if (H.secret_mask >> i & 1) {
            if (!(H.party_mask >> i & 1)) return fail(c, MK_EFORMAT, "secret without public keys");
            expect += c->P.n + c->P.N;
        }
    }
    if (expect != H.payload_words || (H.party_mask >> c->P.k) != 0) return fail(c, MK_EFORMAT, "blob party layout mismatch");
    size_t off = sizeof(H);
    auto get = [&](std::vector<uint32_t> &v, size_t words) {
        v.resize(words);
        std::memcpy(v.data(), p + off, words * 4);
        off += words * 4;
    };
    std::vector<uint32_t> crs;
    get(crs, c->crs.size());
    std::vector<PartyKeys> parties(c->P.k);
    for (uint32_t i = 0; i < c->P.k; ++i) {
        PartyKeys &K = parties[i];
        if (!(H.party_mask >> i & 1)) continue;
        if (H.secret_mask >> i & 1) {
            get(K.s, c->P.n);
            get(K.z, c->P.N);
            K.has_secret = true;
        }
        get(K.pk, c->pk_words());
        get(K.bk, c->bk_words());
        get(K.ks, c->ks_words());
        K.has_public = true;
    }
    c->crs = std::move(crs);
    for (uint32_t i = 0; i < c->P.k; ++i)
        if (parties[i].has_public) c->party[i] = std::move(parties[i]);
    c->crs_seed = H.crs_seed;
    c->dev_keys_valid = false;
    return MK_OK;
}

// ------------------------------------------------------------------- enc / dec
int mk_encrypt(mk_ctx *c, uint32_t party, const uint8_t *bits, size_t count, uint64_t seed, uint32_t *ct) {
    if (!c) return MK_EINVAL;
    if (party >= c->P.k) return fail(c, MK_EINVAL, "party index out of range");
    if (count && (!bits || !ct)) return fail(c, MK_EINVAL, "null pointer");
    if (!c->party[party].has_secret) return fail(c, MK_ESTATE, "secret key of this party missing");
    const uint32_t n = c->P.n, k = c->P.k;
    const size_t W = c->W();
    const std::vector<uint32_t> &s = c->party[party].s;
    const Philox ra(seed, kTagEncA), re(seed, kTagEncE);
    parallel_for((count + 63) / 64, [&](size_t blk) {
        for (size_t g = blk * 64; g < std::min(count, (blk + 1) * 64); ++g) {
            uint32_t *row = ct + g * W;
            std::memset(row, 0, W * 4);
            uint32_t dot = 0;
            for (uint32_t x = 0; x < n; ++x) {
                const uint32_t a = ra.word((uint64_t)g * n + x);
                row[(size_t)party * n + x] = a;
                dot += a * s[x];
            }
            row[(size_t)k * n] = (0u - dot) + ((bits[g] & 1u) ? (1u << 30) : 0u) + re.gauss32(g, c->P.sigma_lwe);
        }
    });
    return MK_OK;
}

int mk_encrypt_joint(mk_ctx *c, const uint8_t *bits, size_t count, uint64_t seed, uint32_t *ct) {
    if (!c) return MK_EINVAL;
    if (count && (!bits || !ct)) return fail(c, MK_EINVAL, "null pointer");
    int rc = check_all_secret(c);
    if (rc) return rc;
    const uint32_t n = c->P.n, k = c->P.k;
    const size_t W = c->W();
    const Philox ra(seed, kTagEncA), re(seed, kTagEncE);
    parallel_for((count + 63) / 64, [&](size_t blk) {
        for (size_t g = blk * 64; g < std::min(count, (blk + 1) * 64); ++g) {
            uint32_t *row = ct + g * W;
            uint32_t dot = 0;
            for (size_t x = 0; x < (size_t)k * n; ++x) {
                const uint32_t a = ra.word((uint64_t)g * k * n + x);
                row[x] = a;
                dot += a * c->party[x / n].s[x % n];
            }
            row[(size_t)k * n] = (0u - dot) + ((bits[g] & 1u) ? (1u << 30) : 0u) + re.gauss32(g, c->P.sigma_lwe);
        }
    });
    return MK_OK;
}

int mk_trivial(mk_ctx *c, const uint8_t *bits, size_t count, uint32_t *ct) {
    if (!c) return MK_EINVAL;
    if (count && (!bits || !ct)) return fail(c, MK_EINVAL, "null pointer");
    const size_t W = c->W();
    for (size_t g = 0; g < count; ++g) {
        uint32_t *row = ct + g * W;
        std::memset(row, 0, W * 4);
        row[W - 1] = (bits[g] & 1u) ? (1u << 30) : 0u;
    }
    return MK_OK;
}

static int get_host_rows(mk_ctx *c, const uint32_t *ct, size_t count, int on_device, std::vector<uint32_t> &buf,
                         const uint32_t **rows) {
    if (!on_device) {
        *rows = ct;
        return MK_OK;
    }
    if (c->device < 0) return fail(c, MK_EDEVICE, "host-only context");
    buf.resize(count * c->W());
    MK_CUDA(c, cudaSetDevice(c->device));
    MK_CUDA(c, cudaMemcpyAsync(buf.data(), ct, buf.size() * 4, cudaMemcpyDeviceToHost, c->stream));
    MK_CUDA(c, cudaStreamSynchronize(c->stream));
    *rows = buf.data();
    return MK_OK;
}

int mk_phase(mk_ctx *c, const uint32_t *ct, size_t count, int on_device, uint32_t *phase) {
    if (!c) return MK_EINVAL;
    if (count && (!ct || !phase)) return fail(c, MK_EINVAL, "null pointer");
    int rc = check_all_secret(c);
    if (rc) return rc;
    std::vector<uint32_t> buf;
    const uint32_t *rows = nullptr;
    rc = get_host_rows(c, ct, count, on_device, buf, &rows);
    if (rc) return rc;
    const uint32_t n = c->P.n, k = c->P.k;
    const size_t W = c->W();
    for (size_t g = 0; g < count; ++g) {
        const uint32_t *row = rows + g * W;
        uint32_t ph = row[(size_t)k * n];
        for (uint32_t i = 0; i < k; ++i) {
            const uint32_t *s = c->party[i].s.data();
            for (uint32_t x = 0; x < n; ++x) ph += row[(size_t)i * n + x] * s[x];
        }
        phase[g] = ph;
    }
    return MK_OK;
}

int mk_decrypt(mk_ctx *c, const uint32_t *ct, size_t count, int on_device, uint8_t *bits) {
    if (!c) return MK_EINVAL;
    if (count && !bits) return fail(c, MK_EINVAL, "null pointer");
    std::vector<uint32_t> ph(count);
    int rc = mk_phase(c, ct, count, on_device, ph.data());
    if (rc) return rc;
    // m = 1 iff the phase lies in [1/8, 5/8): the nearer of 0 and 1/4.
    for (size_t g = 0; g < count; ++g) bits[g] = (uint8_t)((uint32_t)(ph[g] - (1u << 29)) < (1u << 31));
    return MK_OK;
}

// ------------------------------------------------------------------- gates
int mk_gate(mk_ctx *c, int type, const uint32_t *d_a, const uint32_t *d_b, uint32_t *d_out, size_t count) {
    if (!c) return MK_EINVAL;
    if (type < MK_AND || type > MK_XNOR) return fail(c, MK_EINVAL, "unknown gate type");
    return run_gates(c, kDescUniform, nullptr, type, d_a, d_b, d_out, count);
}

int mk_gates(mk_ctx *c, const uint8_t *d_types, const uint32_t *d_a, const uint32_t *d_b, uint32_t *d_out,
             size_t count) {
    if (!c) return MK_EINVAL;
    if (count && !d_types) return fail(c, MK_EINVAL, "null type pointer");
    return run_gates(c, kDescTypes, d_types, 0, d_a, d_b, d_out, count);
}

int mk_gates_lin(mk_ctx *c, const mk_lin *d_lin, const uint32_t *d_a, const uint32_t *d_b, uint32_t *d_out,
                 size_t count) {
    if (!c) return MK_EINVAL;
    if (count && !d_lin) return fail(c, MK_EINVAL, "null mk_lin pointer");
    return run_gates(c, kDescLin, d_lin, 0, d_a, d_b, d_out, count);
}

int mk_not(mk_ctx *c, const uint32_t *d_a, uint32_t *d_out, size_t count) {
    if (!c) return MK_EINVAL;
    if (count == 0) return MK_OK;
    if (!d_a || !d_out) return fail(c, MK_EINVAL, "null pointer");
    if (c->device < 0) return fail(c, MK_EDEVICE, "host-only context");
    MK_CUDA(c, cudaSetDevice(c->device));
    cudaError_t e = launch_not(c->shape(), d_a, d_out, count, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "not kernel");
    return MK_OK;
}

// ------------------------------------------------------------------- operators
int mk_add_kbit(mk_ctx *c, uint32_t kbits, const uint32_t *d_a, const uint32_t *d_b, uint32_t *d_out, size_t pairs) {
    if (!c) return MK_EINVAL;
    return run_circuit(c, MK_OP_ADD, kbits, d_a, d_b, d_out, pairs);
}

int mk_sub_kbit(mk_ctx *c, uint32_t kbits, const uint32_t *d_a, const uint32_t *d_b, uint32_t *d_out, size_t pairs) {
    if (!c) return MK_EINVAL;
    return run_circuit(c, MK_OP_SUB, kbits, d_a, d_b, d_out, pairs);
}

int mk_mul_kbit(mk_ctx *c, uint32_t kbits, const uint32_t *d_a, const uint32_t *d_b, uint32_t *d_out, size_t pairs) {
    if (!c) return MK_EINVAL;
    return run_circuit(c, MK_OP_MUL, kbits, d_a, d_b, d_out, pairs);
}

int mk_div_kbit(mk_ctx *c, uint32_t kbits, const uint32_t *d_a, const uint32_t *d_b, uint32_t *d_q, uint32_t *d_r,
                size_t pairs) {
    if (!c) return MK_EINVAL;
    if (pairs && !d_r) return fail(c, MK_EINVAL, "null pointer");
    return run_circuit(c, MK_OP_DIV, kbits, d_a, d_b, d_q, pairs, d_r);
}

int mk_circuit_netlist(int op, uint32_t kbits, int style, mk_gate_rec *gates, uint32_t gate_cap,
                       uint32_t *n_gates, int32_t *outputs, uint32_t out_cap, uint32_t *n_outputs,
                       uint32_t *n_levels) {
    Netlist net;
    if (!build_netlist(op, kbits, style, net)) return MK_EINVAL;
    if (n_gates) *n_gates = (uint32_t)net.gates.size();
    if (n_outputs) *n_outputs = (uint32_t)net.outputs.size();
    if (n_levels) {
        const std::vector<uint32_t> lev = netlist_levels(net);
        *n_levels = lev.empty() ? 0 : *std::max_element(lev.begin(), lev.end());
    }
    if (gates)
        for (uint32_t g = 0; g < net.gates.size() && g < gate_cap; ++g) gates[g] = net.gates[g];
    if (outputs)
        for (uint32_t i = 0; i < net.outputs.size() && i < out_cap; ++i)
            outputs[i] = net.outputs[i].w * 2 + net.outputs[i].neg;
    return MK_OK;
}

// ------------------------------------------------------------------- no allocation
int mk_gates_noalloc(mk_ctx *c, const uint8_t *d_types, const uint32_t *d_a, const uint32_t *d_b, uint32_t *d_out,
                     size_t count) {
    if (!c) return MK_EINVAL;
    if (count == 0) return MK_OK;
    if (!d_types || !d_a || !d_b || !d_out) return fail(c, MK_EINVAL, "null pointer");
    if (c->device < 0) return fail(c, MK_EDEVICE, "host-only context (device = -1)");

    const size_t per_gate = 4 * c->E() + sizeof(GateDesc);
    const size_t cap = (kNoAllocScratchBytes - 256) / per_gate;
    if (count > cap)
        return fail(c, MK_EINVAL, "count " + std::to_string(count) + " exceeds the fixed scratch capacity of " +
                                      std::to_string(cap) + " gates for these parameters");
    if (!c->dev_keys_valid)
        return fail(c, MK_ESTATE, "keys are not on the device yet: make one ordinary gate call on this context first");
    MK_CUDA(c, cudaSetDevice(c->device));
    void *base = nullptr;
    MK_CUDA(c, noalloc_scratch(c->device, &base));
    GateDesc *desc = reinterpret_cast<GateDesc *>(base);
    const size_t desc_bytes = ((count * sizeof(GateDesc)) + 255) & ~size_t(255);
    uint32_t *ext = reinterpret_cast<uint32_t *>(static_cast<unsigned char *>(base) + desc_bytes);
    const uint32_t cnt = (uint32_t)count;
    cudaError_t e = launch_desc_from_types(d_types, desc, 0, cnt, c->stream);
    if (e == cudaSuccess) e = launch_bootstrap_ntt(c->shape(), c->dkeys(), desc, d_a, d_b, ext, cnt, c->stream);
    if (e == cudaSuccess) e = launch_keyswitch(c->shape(), c->dkeys(), desc, ext, d_out, cnt, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "mk_gates_noalloc");
    return MK_OK;
}

// ------------------------------------------------------------------- stages
int mk_stage_modswitch(mk_ctx *c, const mk_lin *d_lin, const uint32_t *d_a, const uint32_t *d_b, uint32_t *d_abar,
                       size_t count) {
    if (!c) return MK_EINVAL;
    if (count == 0) return MK_OK;
    if (!d_lin || !d_a || !d_b || !d_abar) return fail(c, MK_EINVAL, "null pointer");
    int rc = device_ready(c, count);
    if (rc) return rc;
    for (size_t start = 0; start < count; start += c->max_batch) {
        const uint32_t cnt = (uint32_t)std::min<size_t>(c->max_batch, count - start);
        cudaError_t e = launch_desc_from_lin(d_lin, c->d_desc, (uint32_t)start, cnt, c->stream);
        if (e == cudaSuccess)
            e = launch_modswitch(c->shape(), c->d_desc, d_a, d_b, d_abar + start * c->W(), cnt, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "modswitch");
    }
    return MK_OK;
}

int mk_stage_blind_rotate(mk_ctx *c, const uint32_t *d_abar, size_t count, int64_t max_steps, uint32_t *d_acc) {
    if (!c) return MK_EINVAL;
    if (count == 0) return MK_OK;
    if (!d_abar || !d_acc) return fail(c, MK_EINVAL, "null pointer");
    if (count > 0xFFFFFFFFull) return fail(c, MK_EINVAL, "count too large");
    int rc = device_ready(c, 1);
    if (rc) return rc;
    cudaError_t e = launch_blind_rotate_ntt(c->shape(), c->dkeys(), d_abar, (uint32_t)count, max_steps, d_acc, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "blind rotation");
    return MK_OK;
}

int mk_stage_bootstrap(mk_ctx *c, const mk_lin *d_lin, const uint32_t *d_a, const uint32_t *d_b, uint32_t *d_ext,
                       size_t count) {
    if (!c) return MK_EINVAL;
    if (count == 0) return MK_OK;
    if (!d_lin || !d_a || !d_b || !d_ext) return fail(c, MK_EINVAL, "null pointer");
    int rc = device_ready(c, count);
    if (rc) return rc;
    for (size_t start = 0; start < count; start += c->max_batch) {
        const uint32_t cnt = (uint32_t)std::min<size_t>(c->max_batch, count - start);
        cudaError_t e = launch_desc_from_lin(d_lin, c->d_desc, (uint32_t)start, cnt, c->stream);
        if (e == cudaSuccess)
            e = launch_bootstrap_ntt(c->shape(), c->dkeys(), c->d_desc, d_a, d_b, d_ext + start * c->E(), cnt,
                                     c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "bootstrap");
    }
    return MK_OK;
}

int mk_stage_keyswitch(mk_ctx *c, const uint32_t *d_ext, uint32_t *d_out, size_t count) {
    if (!c) return MK_EINVAL;
    if (count == 0) return MK_OK;
    if (!d_ext || !d_out) return fail(c, MK_EINVAL, "null pointer");
    if (count > 0xFFFFFFFFull) return fail(c, MK_EINVAL, "count too large");
    int rc = device_ready(c, 1);
    if (rc) return rc;
    cudaError_t e = launch_keyswitch(c->shape(), c->dkeys(), nullptr, d_ext, d_out, (uint32_t)count, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "keyswitch");
    return MK_OK;
}

// ------------------------------------------------------------------- measurement
int mk_timing_enable(mk_ctx *c, int on) {
    if (!c) return MK_EINVAL;
    if (c->device < 0) return fail(c, MK_EDEVICE, "host-only context");
    c->timing = on != 0;
    return MK_OK;
}

int mk_timing_reset(mk_ctx *c) {
    if (!c) return MK_EINVAL;
    if (c->device < 0) return MK_OK;
    MK_CUDA(c, cudaSetDevice(c->device));
    MK_CUDA(c, cudaStreamSynchronize(c->stream));
    release_timing(c);
    return MK_OK;
}

int mk_timing_read(mk_ctx *c, int kernel, double *ms_total, uint64_t *launches) {
    if (!c || !ms_total || !launches || kernel < 0 || kernel > 1) return MK_EINVAL;
    *ms_total = 0;
    *launches = c->ev[kernel].size();
    if (c->device < 0) return MK_OK;
    MK_CUDA(c, cudaSetDevice(c->device));
    MK_CUDA(c, cudaStreamSynchronize(c->stream));
    for (auto &pr : c->ev[kernel]) {
        float ms = 0;
        MK_CUDA(c, cudaEventElapsedTime(&ms, pr.first, pr.second));
        *ms_total += ms;
    }
    return MK_OK;
}

int mk_measure_butterfly_rate(int device, void *stream, int form, uint32_t iters, double *per_s) {
    if (!per_s || iters == 0 ||
        (form != MK_FORM_NTT && form != MK_FORM_NTT2 && form != MK_FORM_FFT && form != MK_FORM_TC))
        return MK_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return MK_EDEVICE;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return MK_EDEVICE;
    const uint32_t threads = 256, blocks = (uint32_t)prop.multiProcessorCount * 8;
    cudaStream_t st = (cudaStream_t)stream;
    uint64_t *sink = nullptr;
    if (cudaMalloc(&sink, blocks * sizeof(uint64_t)) != cudaSuccess) return MK_ENOMEM;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    int rc = MK_OK;
    auto launch = [&](uint32_t it) {
        if (form == MK_FORM_NTT) return launch_butterfly_peak(blocks, threads, it, sink, st);
        if (form == MK_FORM_FFT) return launch_butterfly_peak_fft(blocks, threads, it, reinterpret_cast<double *>(sink), st);
        if (form == MK_FORM_TC) return launch_mma_peak(blocks, threads, it, reinterpret_cast<float *>(sink), st);
        return launch_butterfly_peak2(blocks, threads, it, reinterpret_cast<uint32_t *>(sink), st);
    };
    if (launch(iters / 8 + 1) != cudaSuccess) rc = MK_EDEVICE;  // warm-up
    cudaEventRecord(a, st);
    if (launch(iters) != cudaSuccess) rc = MK_EDEVICE;
    cudaEventRecord(b, st);
    if (cudaEventSynchronize(b) != cudaSuccess) rc = MK_EDEVICE;
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    // MK_FORM_TC: 8 MMAs of 16 x 8 x 16 multiply-accumulates per warp and iteration
    const double per_thread_iter = form == MK_FORM_TC ? 8.0 * 16 * 8 * 16 / 32 : 8.0;
    *per_s = (double)blocks * threads * iters * per_thread_iter / (ms * 1e-3);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    return rc;
}

int mk_tc_negacyclic(int device, void *stream, uint32_t N, uint32_t G, uint32_t nchunks, const uint32_t *keys,
                     const int8_t *digits, int32_t *out, int engine) {
    if (!keys || !digits || !out || (N != 256 && N != 1024) || G == 0 || G % (engine == 1 ? 128u : 64u) ||
        nchunks == 0 || nchunks > 3 || engine < 0 || engine > 1)
        return MK_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return MK_EDEVICE;
    cudaStream_t st = (cudaStream_t)stream;
    void *work = nullptr;
    if (cudaMalloc(&work, (size_t)nchunks * G * N * 2) != cudaSuccess) return MK_ENOMEM;
    int rc = MK_OK;
    unsigned int timeout = 0;
    if (engine == 1 && tc05_error(&timeout, true) != cudaSuccess) rc = MK_EDEVICE;
    if (rc == MK_OK && launch_negacyclic_tc(N, G, nchunks, keys, digits, out, work, engine, st) != cudaSuccess)
        rc = MK_EDEVICE;
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = MK_EDEVICE;
    if (rc == MK_OK && engine == 1 && (tc05_error(&timeout, true) != cudaSuccess || timeout != 0)) rc = MK_ETIMEOUT;
    cudaFree(work);
    return rc;
}

}  // extern "C"
