// mk_kernels.cu -- sm_103a kernels of multi-key TFHE gates other than the
// blind rotation (which lives in mk_bootstrap.cuh): modulus switch stage,
// MKKeySwitch (Sec. 3.2 of arXiv 2205.05825), MKNOT (Eq. 8), gate
// descriptors, and the dispatch to the per-ring-dimension blind rotation.
#include "mk_internal.h"

namespace mk {
namespace {

__global__ void modswitch_kernel(LaunchShape S, const GateDesc *__restrict__ desc, const uint32_t *__restrict__ ct_a,
                                 const uint32_t *__restrict__ ct_b, uint32_t *__restrict__ abar_out) {
    const uint32_t W = S.k * S.n + 1;
    const uint32_t sh = 32 - (S.logN + 1);
    const GateDesc g = desc[blockIdx.x];
    const uint32_t *ca = ct_a + (size_t)g.ia * W;
    const uint32_t *cb = ct_b + (size_t)g.ib * W;
    for (uint32_t x = threadIdx.x; x < W; x += blockDim.x) {
        uint32_t v = (uint32_t)g.s1 * ca[x] + (uint32_t)g.s2 * cb[x];
        if (x == W - 1) v += g.cst - (1u << 30);
        abar_out[(size_t)blockIdx.x * W + x] = (v + (1u << (sh - 1))) >> sh;
    }
}

// ------------------------------------------------------------ key switch
// One CTA per gate, one thread per output column x in [0, n]: for every party
// i and coefficient j, round a_{i,j} to ks_bit*t bits, take t base-2^ks_bit
// digits delta_l and add column x of KS_i[j][l][delta_l - 1] for delta_l != 0.
__global__ void keyswitch_kernel(LaunchShape S, const uint32_t *__restrict__ ks, const GateDesc *__restrict__ desc,
                                 const uint32_t *__restrict__ ext, uint32_t *__restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *ein = reinterpret_cast<uint32_t *>(smem);
    const uint32_t n = S.n, N = S.N, k = S.k, t = S.t;
    const uint32_t nb = (1u << S.ks_bit) - 1;
    const uint32_t E = k * N + 1, W = k * n + 1;
    const uint32_t round_off = 1u << (32 - S.ks_bit * t - 1);
    const uint32_t *src = ext + (size_t)blockIdx.x * E;
    for (uint32_t x = threadIdx.x; x < E; x += blockDim.x) ein[x] = src[x];
    __syncthreads();
    const uint32_t orow = desc ? desc[blockIdx.x].out : blockIdx.x;
    uint32_t *dst = out + (size_t)orow * W;
    const size_t rowlen = n + 1;
    const size_t party_stride = (size_t)N * t * nb * rowlen;
    for (uint32_t x = threadIdx.x; x <= n; x += blockDim.x) {
        uint32_t bsum = 0;
        for (uint32_t i = 0; i < k; ++i) {
            const uint32_t *ksi = ks + i * party_stride + x;
            uint32_t accv = 0;
            for (uint32_t j = 0; j < N; ++j) {
                const uint32_t abar = ein[i * N + j] + round_off;
                const uint32_t *rowj = ksi + (size_t)j * t * nb * rowlen;
                for (uint32_t l = 0; l < t; ++l) {
                    const uint32_t delta = (abar >> (32 - S.ks_bit * (l + 1))) & nb;
                    if (delta) accv += __ldg(rowj + ((size_t)l * nb + (delta - 1)) * rowlen);
                }
            }
            if (x < n) dst[i * n + x] = accv;
            else bsum += accv;
        }
        if (x == n) dst[k * n] = ein[k * N] + bsum;
    }
}

// Batched key switch for 2-bit digits (three rows per digit level): a CTA
// owns KS_GB gates and KS_CX output columns, so every key-switch row it reads
// from L2 serves all its gates.  Per party i and block of KS_JB coefficients
// the gates' digit words (a_{i,j} rounded to ks_bit*t bits) are staged in
// shared memory; per (j, l) each thread puts its column of the rows
// KS_i[j][l][0..2] into private shared-memory slots 1..3 (slot 0 holds zero)
// and every gate adds the slot its digit delta_l selects.  The row loads of
// the next (j, l) are issued before the adds of the current one.
constexpr int KS_GB = 32, KS_CX = 128, KS_JB = 64;

__global__ void __launch_bounds__(KS_CX) keyswitch_batched_kernel(LaunchShape S, const uint32_t *__restrict__ ks,
                                                                  const GateDesc *__restrict__ desc,
                                                                  const uint32_t *__restrict__ ext,
                                                                  uint32_t *__restrict__ out, uint32_t count) {
    __shared__ __align__(16) uint32_t s_dw[KS_JB * KS_GB];
    __shared__ uint32_t s_rows[4 * KS_CX];
    const uint32_t n = S.n, N = S.N, k = S.k, t = S.t;
    const uint32_t E = k * N + 1, W = k * n + 1;
    const uint32_t dbits = 2 * t;
    const uint32_t round_off = 1u << (32 - dbits - 1);
    const uint32_t g0 = blockIdx.x * KS_GB;
    const uint32_t ng = min((uint32_t)KS_GB, count - g0);
    const uint32_t tx = threadIdx.x;
    const uint32_t x = blockIdx.y * KS_CX + tx;  // output column
    const uint32_t xc = x <= n ? x : n;          // columns past n read column n and write nothing
    const size_t rowlen = n + 1;
    const size_t jstride = (size_t)t * 3 * rowlen;  // rows of one coefficient
    s_rows[tx] = 0;  // slot 0: digit 0 adds nothing
    uint32_t acc[KS_GB];
#pragma unroll
    for (int g = 0; g < KS_GB; ++g) acc[g] = 0;
    for (uint32_t i = 0; i < k; ++i) {
        const uint32_t *ksi = ks + (size_t)i * N * jstride + xc;
        for (uint32_t j0 = 0; j0 < N; j0 += KS_JB) {
            __syncthreads();  // the previous block's digit words are consumed
            for (uint32_t q = tx; q < KS_JB * KS_GB; q += KS_CX) {
                const uint32_t g = q / KS_JB, jj = q % KS_JB;
                uint32_t w = 0;
                if (g < ng) w = (ext[(size_t)(g0 + g) * E + i * N + j0 + jj] + round_off) >> (32 - dbits);
                s_dw[jj * KS_GB + g] = w;
            }
            __syncthreads();
            const uint32_t *rows = ksi + (size_t)j0 * jstride;  // (j0, l = 0), advancing by rowlen * 3 per l
            uint32_t r0 = __ldg(rows), r1 = __ldg(rows + rowlen), r2 = __ldg(rows + 2 * rowlen);
            for (uint32_t jj = 0; jj < KS_JB; ++jj) {
                uint32_t dw[KS_GB];
                const uint4 *pw = reinterpret_cast<const uint4 *>(s_dw + jj * KS_GB);
#pragma unroll
                for (int q = 0; q < KS_GB / 4; ++q) {
                    const uint4 v = pw[q];
                    dw[4 * q] = v.x, dw[4 * q + 1] = v.y, dw[4 * q + 2] = v.z, dw[4 * q + 3] = v.w;
                }
                for (uint32_t l = 0; l < t; ++l) {
                    s_rows[KS_CX + tx] = r0;
                    s_rows[2 * KS_CX + tx] = r1;
                    s_rows[3 * KS_CX + tx] = r2;
                    rows += 3 * rowlen;  // next (j, l); one row past the block's end is never read
                    if (jj + 1 < KS_JB || l + 1 < t) {
                        r0 = __ldg(rows), r1 = __ldg(rows + rowlen), r2 = __ldg(rows + 2 * rowlen);
                    }
                    const uint32_t sh = dbits - 2 * (l + 1);
#pragma unroll
                    for (int g = 0; g < KS_GB; ++g) acc[g] += s_rows[((dw[g] >> sh) & 3u) * KS_CX + tx];
                }
            }
        }
        if (x < n) {
#pragma unroll
            for (int g = 0; g < KS_GB; ++g) {
                if ((uint32_t)g < ng) {
                    const uint32_t orow = desc ? desc[g0 + g].out : g0 + g;
                    out[(size_t)orow * W + i * n + x] = acc[g];
                }
                acc[g] = 0;
            }
        }
    }
    if (x == n) {  // the b column sums over every party
#pragma unroll
        for (int g = 0; g < KS_GB; ++g) {
            if ((uint32_t)g < ng) {
                const uint32_t orow = desc ? desc[g0 + g].out : g0 + g;
                out[(size_t)orow * W + k * n] = ext[(size_t)(g0 + g) * E + k * N] + acc[g];
            }
        }
    }
}

// ------------------------------------------------------------ NOT and descriptors
__global__ void not_kernel(uint32_t W, const uint32_t *__restrict__ in, uint32_t *__restrict__ out, size_t total) {
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total; x += (size_t)gridDim.x * blockDim.x) {
        const uint32_t v = in[x];
        out[x] = ((x % W) == W - 1) ? (1u << 30) - v : 0u - v;  // (0, 1/4) - c
    }
}

// (cst, s1, s2) of each gate type: AND Eq. 6, OR Eq. 7, NAND Sec. 3.2,
// NOR Eq. 9 (constant 3/8), XOR Eq. 10, XNOR Eq. 11 (1/2 + 2(c1 - c2)).
__constant__ uint32_t c_gate_cst[6] = {0xE0000000u, 0x20000000u, 0xA0000000u, 0x60000000u, 0x0u, 0x80000000u};
__constant__ int32_t c_gate_s1[6] = {1, 1, -1, -1, 2, 2};
__constant__ int32_t c_gate_s2[6] = {1, 1, -1, -1, -2, -2};

__global__ void desc_types_kernel(const uint8_t *__restrict__ types, GateDesc *__restrict__ desc, uint32_t base,
                                  uint32_t count) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= count) return;
    uint32_t ty = types[base + g];
    if (ty > 5) ty = 0;  // validated on the host for mk_gate; defensive here
    desc[g] = GateDesc{base + g, base + g, c_gate_cst[ty], c_gate_s1[ty], c_gate_s2[ty], base + g};
}

__global__ void desc_lin_kernel(const mk_lin *__restrict__ lin, GateDesc *__restrict__ desc, uint32_t base,
                                uint32_t count) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= count) return;
    const mk_lin L = lin[base + g];
    desc[g] = GateDesc{base + g, base + g, L.cst, L.s1, L.s2, base + g};
}

__global__ void desc_uniform_kernel(int ty, GateDesc *__restrict__ desc, uint32_t base, uint32_t count) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= count) return;
    desc[g] = GateDesc{base + g, base + g, c_gate_cst[ty], c_gate_s1[ty], c_gate_s2[ty], base + g};
}

// Independent Goldilocks butterflies in registers: 8 chains per thread so the
// multiply latency is covered by ILP; the twiddle changes every iteration so
// nothing is loop-invariant.
__global__ void butterfly_peak_kernel(uint32_t iters, uint64_t *sink) {
    constexpr uint64_t P = kGoldilocks, EPS = 0xFFFFFFFFull;
    uint64_t x[8], y[8];
    uint64_t w = 0x123456789ull + threadIdx.x;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        x[c] = (uint64_t)(blockIdx.x * 977 + threadIdx.x * 131 + c) * 0x9E3779B97F4A7C15ull % P;
        y[c] = x[c] ^ 0x5555;
    }
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const uint64_t lo = y[c] * w, hi = __umul64hi(y[c], w);
            const uint64_t hh = hi >> 32, hl = hi & EPS;
            uint64_t t0 = lo - hh;
            t0 = (lo < hh) ? t0 - EPS : t0;
            const uint64_t t1 = hl * EPS;
            uint64_t V = t0 + t1;
            V = (V < t1) ? V + EPS : V;
            V = (V >= P) ? V - P : V;
            const uint64_t U = x[c];
            uint64_t s = U + V;
            s = (s < U) ? s + EPS : s;
            s = (s >= P) ? s - P : s;
            uint64_t d = U - V;
            d = (U < V) ? d - EPS : d;
            x[c] = s;
            y[c] = d;
        }
        w += 0x10001;
    }
    uint64_t r = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) r ^= x[c] ^ y[c];
    if (r == 0x1234567ull) sink[blockIdx.x] = r;  // keeps the loop live; practically never stores
}

// Wire buffer of a circuit: rows 0..P-1 = trivial 0, rows P..2P-1 = trivial 1.
__global__ void circuit_consts_kernel(uint32_t *pool, uint32_t P, uint32_t W) {
    const uint32_t r = blockIdx.x;  // 0 .. 2P-1
    uint32_t *row = pool + (size_t)r * W;
    for (uint32_t x = threadIdx.x; x < W; x += blockDim.x) row[x] = (x == W - 1 && r >= P) ? (1u << 30) : 0u;
}

// Operand bits into the wire buffer: row (wire0 + i) * P + p <- src[p][i].
__global__ void circuit_inputs_kernel(uint32_t *pool, const uint32_t *src, uint32_t kbits, uint32_t P,
                                      uint32_t wire0, uint32_t W) {
    const uint32_t r = blockIdx.x;  // i * P + p
    const uint32_t i = r / P, p = r % P;
    const uint32_t *s = src + ((size_t)p * kbits + i) * W;
    uint32_t *d = pool + ((size_t)(wire0 + i) * P + p) * W;
    for (uint32_t x = threadIdx.x; x < W; x += blockDim.x) d[x] = s[x];
}

// Outputs out of the wire buffer: dst[p][i] <- wire outs[i] >> 1, negated
// (MKNOT, Eq. 8: (0, 1/4) - c) when outs[i] & 1.
__global__ void circuit_outputs_kernel(uint32_t *dst, const uint32_t *pool, const int32_t *outs, uint32_t nout,
                                       uint32_t P, uint32_t W) {
    const uint32_t r = blockIdx.x;  // p * nout + i
    const uint32_t p = r / nout, i = r % nout;
    const int32_t o = outs[i];
    const uint32_t *s = pool + ((size_t)(o >> 1) * P + p) * W;
    uint32_t *d = dst + (size_t)r * W;
    const bool ng = o & 1;
    for (uint32_t x = threadIdx.x; x < W; x += blockDim.x) {
        const uint32_t v = s[x];
        d[x] = ng ? ((x == W - 1) ? (1u << 30) - v : 0u - v) : v;
    }
}

// Independent Harvey butterflies mod a 30-bit prime with Shoup twiddles (the
// inner operation of MK_FORM_NTT2), 8 chains per thread, both primes.
__global__ void butterfly_peak2_kernel(uint32_t iters, uint32_t *sink) {
    constexpr uint32_t p1 = kP1, p2 = kP2;
    uint32_t x[8], y[8];
    uint32_t w = 12345u + threadIdx.x, wp = (uint32_t)(((uint64_t)w << 32) / p1);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        x[c] = (blockIdx.x * 977u + threadIdx.x * 131u + c) % p1;
        y[c] = x[c] ^ 0x5555u;
    }
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const uint32_t p = (c & 1) ? p2 : p1;
            const uint32_t X = min(x[c], x[c] - 2 * p);
            const uint32_t T = y[c] * w - __umulhi(y[c], wp) * p;
            x[c] = X + T;
            y[c] = X - T + 2 * p;
        }
        w += 3;
        wp += 11;
    }
    uint32_t r = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) r ^= x[c] ^ y[c];
    if (r == 0x1234567u) sink[blockIdx.x] = r;  // keeps the loop live; practically never stores
}

// Independent complex FP64 butterflies (one complex multiply, two complex
// additions): the inner operation of MK_FORM_FFT.
__global__ void butterfly_peak_fft_kernel(uint32_t iters, double *sink) {
    double xr[8], xi[8], yr[8], yi[8];
    double wr = 0.7071067811865476 + 1e-9 * threadIdx.x, wi = 0.7071067811865475;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        xr[c] = 1.0 + c + blockIdx.x;
        xi[c] = 0.5 * c;
        yr[c] = 2.0 - c;
        yi[c] = 0.25 + threadIdx.x;
    }
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const double vr = fma(yr[c], wr, -yi[c] * wi), vi = fma(yr[c], wi, yi[c] * wr);
            const double ur = xr[c], ui = xi[c];
            xr[c] = ur + vr;
            xi[c] = ui + vi;
            yr[c] = ur - vr;
            yi[c] = ui - vi;
        }
        wr = fma(wr, 0.9999999, 1e-12);
    }
    double r = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) r += xr[c] + xi[c] + yr[c] + yi[c];
    if (r == 1.2345) sink[blockIdx.x] = r;  // keeps the loop live; practically never stores
}

}  // namespace

cudaError_t launch_butterfly_peak_fft(uint32_t blocks, uint32_t threads, uint32_t iters, double *sink,
                                      cudaStream_t st) {
    butterfly_peak_fft_kernel<<<blocks, threads, 0, st>>>(iters, sink);
    return cudaGetLastError();
}

cudaError_t launch_butterfly_peak2(uint32_t blocks, uint32_t threads, uint32_t iters, uint32_t *sink,
                                   cudaStream_t st) {
    butterfly_peak2_kernel<<<blocks, threads, 0, st>>>(iters, sink);
    return cudaGetLastError();
}

cudaError_t launch_circuit_consts(uint32_t *pool, uint32_t P, uint32_t W, cudaStream_t st) {
    circuit_consts_kernel<<<2 * P, 256, 0, st>>>(pool, P, W);
    return cudaGetLastError();
}

cudaError_t launch_circuit_inputs(uint32_t *pool, const uint32_t *src, uint32_t kbits, uint32_t P, uint32_t wire0,
                                  uint32_t W, cudaStream_t st) {
    circuit_inputs_kernel<<<kbits * P, 256, 0, st>>>(pool, src, kbits, P, wire0, W);
    return cudaGetLastError();
}

cudaError_t launch_circuit_outputs(uint32_t *dst, const uint32_t *pool, const int32_t *outs, uint32_t nout,
                                   uint32_t P, uint32_t W, cudaStream_t st) {
    circuit_outputs_kernel<<<nout * P, 256, 0, st>>>(dst, pool, outs, nout, P, W);
    return cudaGetLastError();
}

cudaError_t launch_butterfly_peak(uint32_t blocks, uint32_t threads, uint32_t iters, uint64_t *sink,
                                  cudaStream_t st) {
    butterfly_peak_kernel<<<blocks, threads, 0, st>>>(iters, sink);
    return cudaGetLastError();
}

namespace {
using BootstrapFn = cudaError_t (*)(const LaunchShape &, const DeviceKeys &, const GateDesc *, const uint32_t *,
                                    const uint32_t *, const uint32_t *, int64_t, uint32_t *, uint32_t *, uint32_t,
                                    cudaStream_t);
BootstrapFn pick(const LaunchShape &S) {
#define MK_ROW(LOGN, F)                                                                                   \
    {launch_bootstrap_logn##LOGN##_f##F##_v0, launch_bootstrap_logn##LOGN##_f##F##_v1,                   \
     launch_bootstrap_logn##LOGN##_f##F##_v2, launch_bootstrap_logn##LOGN##_f##F##_v3,                   \
     launch_bootstrap_logn##LOGN##_f##F##_v4, launch_bootstrap_logn##LOGN##_f##F##_v5,                   \
     launch_bootstrap_logn##LOGN##_f##F##_v6, launch_bootstrap_logn##LOGN##_f##F##_v7,                   \
     launch_bootstrap_logn##LOGN##_f##F##_v8}
    static const BootstrapFn t8[2][kNumVariants] = {MK_ROW(8, 0), MK_ROW(8, 1)};
    static const BootstrapFn t10[2][kNumVariants] = {MK_ROW(10, 0), MK_ROW(10, 1)};
#undef MK_ROW
    if (S.form == MK_FORM_FFT) {  // one kernel for every variant number
        if (S.logN == 8) return launch_bootstrap_logn8_f2_v0;
        if (S.logN == 10) return launch_bootstrap_logn10_f2_v0;
        return nullptr;
    }
    if (S.variant < 0 || S.variant >= kNumVariants || S.form < 0 || S.form > 1) return nullptr;
    if (S.logN == 8) return t8[S.form][S.variant];
    if (S.logN == 10) return t10[S.form][S.variant];
    return nullptr;
}

// The cluster (latency) launcher for this shape and batch, or nullptr.
BootstrapFn pick_cluster(const LaunchShape &S, uint32_t count) {
    if (count > S.cluster_max || S.k + 1 > 8 || (S.form != MK_FORM_NTT && S.form != MK_FORM_NTT2)) return nullptr;
    if (S.logN == 8) return S.form == MK_FORM_NTT ? launch_cluster_logn8_f0 : launch_cluster_logn8_f1;
    if (S.logN == 10) return S.form == MK_FORM_NTT ? launch_cluster_logn10_f0 : launch_cluster_logn10_f1;
    return nullptr;
}
}  // namespace

int cluster_capacity(const LaunchShape &S) {
    if (S.k + 1 > 8 || (S.form != MK_FORM_NTT && S.form != MK_FORM_NTT2)) return 0;
    if (S.logN == 8) return S.form == MK_FORM_NTT ? cluster_capacity_logn8_f0(S.k, S.n) : cluster_capacity_logn8_f1(S.k, S.n);
    if (S.logN == 10)
        return S.form == MK_FORM_NTT ? cluster_capacity_logn10_f0(S.k, S.n) : cluster_capacity_logn10_f1(S.k, S.n);
    return 0;
}

cudaError_t launch_bootstrap_ntt(const LaunchShape &S, const DeviceKeys &K, const GateDesc *desc,
                                 const uint32_t *ct_a, const uint32_t *ct_b, uint32_t *ext, uint32_t count,
                                 cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    if (S.form == MK_FORM_TC) return launch_bootstrap_tc(S, K, desc, ct_a, ct_b, nullptr, -1, ext, nullptr, count, st);
    if (BootstrapFn fc = pick_cluster(S, count)) return fc(S, K, desc, ct_a, ct_b, nullptr, -1, ext, nullptr, count, st);
    BootstrapFn f = pick(S);
    if (!f) return cudaErrorInvalidValue;
    return f(S, K, desc, ct_a, ct_b, nullptr, -1, ext, nullptr, count, st);
}

cudaError_t launch_blind_rotate_ntt(const LaunchShape &S, const DeviceKeys &K, const uint32_t *abar,
                                    uint32_t count, int64_t max_steps, uint32_t *acc, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    if (S.form == MK_FORM_TC) return launch_bootstrap_tc(S, K, nullptr, nullptr, nullptr, abar, max_steps, nullptr, acc, count, st);
    if (BootstrapFn fc = pick_cluster(S, count))
        return fc(S, K, nullptr, nullptr, nullptr, abar, max_steps, nullptr, acc, count, st);
    BootstrapFn f = pick(S);
    if (!f) return cudaErrorInvalidValue;
    return f(S, K, nullptr, nullptr, nullptr, abar, max_steps, nullptr, acc, count, st);
}

cudaError_t launch_netlist(const LaunchShape &S, const DeviceKeys &K, const NetlistArgs &A, uint32_t sm_count,
                           cudaStream_t st) {
    if (S.form == MK_FORM_NTT && S.logN == 8) return launch_netlist_logn8_f0(S, K, A, sm_count, st);
    if (S.form == MK_FORM_NTT && S.logN == 10) return launch_netlist_logn10_f0(S, K, A, sm_count, st);
    if (S.form == MK_FORM_NTT2 && S.logN == 8) return launch_netlist_logn8_f1(S, K, A, sm_count, st);
    if (S.form == MK_FORM_NTT2 && S.logN == 10) return launch_netlist_logn10_f1(S, K, A, sm_count, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_modswitch(const LaunchShape &S, const GateDesc *desc, const uint32_t *ct_a,
                             const uint32_t *ct_b, uint32_t *abar, uint32_t count, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    modswitch_kernel<<<count, 256, 0, st>>>(S, desc, ct_a, ct_b, abar);
    return cudaGetLastError();
}

cudaError_t launch_keyswitch(const LaunchShape &S, const DeviceKeys &K, const GateDesc *desc,
                             const uint32_t *ext, uint32_t *out, uint32_t count, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    if (S.ks_bit == 2 && count >= kKeyswitchBatchMin) {
        const dim3 grid((count + KS_GB - 1) / KS_GB, (S.n + 1 + KS_CX - 1) / KS_CX);
        keyswitch_batched_kernel<<<grid, KS_CX, 0, st>>>(S, K.ks, desc, ext, out, count);
        return cudaGetLastError();
    }
    const uint32_t threads = ((S.n + 1 + 31) / 32) * 32 > 1024 ? 1024 : ((S.n + 1 + 31) / 32) * 32;
    const size_t sm = sizeof(uint32_t) * (S.k * S.N + 1);
    cudaError_t e = cudaFuncSetAttribute(keyswitch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    keyswitch_kernel<<<count, threads, sm, st>>>(S, K.ks, desc, ext, out);
    return cudaGetLastError();
}

cudaError_t launch_not(const LaunchShape &S, const uint32_t *in, uint32_t *out, size_t count, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    const uint32_t W = S.k * S.n + 1;
    const size_t total = count * W;
    size_t blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    not_kernel<<<(unsigned)blocks, 256, 0, st>>>(W, in, out, total);
    return cudaGetLastError();
}

cudaError_t launch_desc_from_types(const uint8_t *types, GateDesc *desc, uint32_t base, uint32_t count,
                                   cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    desc_types_kernel<<<(count + 255) / 256, 256, 0, st>>>(types, desc, base, count);
    return cudaGetLastError();
}

cudaError_t launch_desc_from_lin(const mk_lin *lin, GateDesc *desc, uint32_t base, uint32_t count,
                                 cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    desc_lin_kernel<<<(count + 255) / 256, 256, 0, st>>>(lin, desc, base, count);
    return cudaGetLastError();
}

cudaError_t launch_desc_uniform(int type, GateDesc *desc, uint32_t base, uint32_t count, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    if (type < 0 || type > 5) return cudaErrorInvalidValue;
    desc_uniform_kernel<<<(count + 255) / 256, 256, 0, st>>>(type, desc, base, count);
    return cudaGetLastError();
}

}  // namespace mk
