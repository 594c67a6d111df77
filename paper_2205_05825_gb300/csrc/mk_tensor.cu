// mk_tensor.cu -- the exact tensor-core product form (MK_FORM_TC).
//
// A negacyclic product key * u in T_N[X] is the matrix-vector product T u with
// the negacyclic Toeplitz matrix T[m][t] = ext[m - t], where ext[x] = key[x]
// for 0 <= x < N and ext[x] = -key[x + N] for -N < x < 0.  For a wave of G
// gates in lockstep at one CMux step, the digit polynomials of all gates are
// the columns of one matrix, so each key polynomial meets the whole wave in
// one GEMM (rows: output coefficients; columns: gates; depth: N):
//   - the key's torus32 words are split into four signed byte planes,
//     key = sum_b 2^(8b) key_b (mod 2^32), key_b in [-128, 128);
//   - the gadget digits of base 2^8 are in [-128, 128) as well, so every
//     product is at most 2^14 in magnitude and a sum over one polynomial
//     (N <= 1024 terms) at most 2^24: bf16 operands with fp32 accumulation
//     hold every partial sum exactly;
//   - after each (key polynomial, plane) the fp32 sums are converted to
//     integers, weighted by 2^(8b) and added mod 2^32.
// The result is the schoolbook product, bit for bit.
//
// Per CMux step (i, j) of the blind rotation, for the hybrid product of
// Algorithm 1 (u_jj = g^-1((X^-e - 1) ACC_jj); v = <u_0, -a> + sum <u_jj, pk_jj>;
// w = g^-1(v); ACC_jj += <u_jj, d>; ACC_0 += <w, f0>; ACC_i += <w, f1>):
//   tc_rotate_digits: ACC += C (previous step), then the digits u_jj,l of
//                     (X^-e - 1) ACC_jj for every gate
//   tc_products (A):  C_jj = sum_l T(d_l) u_jj,l and the partial sums
//                     V_jj = sum_l T(A_jj,l) u_jj,l (A_0,l = -a_l, A_jj,l = pk_jj,l)
//   tc_vdigits:       w = g^-1(sum_jj V_jj)
//   tc_products (B):  C_0 += sum_l T(f0_l) w_l ; C_i += sum_l T(f1_l) w_l
// The tensor instruction is the warp-level mma.sync m16n8k16 (bf16 inputs,
// fp32 accumulation): the integer kind of tcgen05 is not available on
// sm_103a.  The Toeplitz structure makes one A fragment serve a whole
// diagonal of 16x16 tiles, so a warp loads one new A fragment per k-step.
#include <cuda_bf16.h>

#include "mk_internal.h"

namespace mk {
namespace {

constexpr int TC_GT = 64;         // gates per CTA tile
constexpr int TC_PAD = 128;       // waves are padded to this many gates (either engine)
constexpr int TC_MS = 256;        // output coefficients per CTA tile
constexpr int TC_THREADS = 256;   // 8 warps: 4 row groups of 64 x 2 gate groups of 32

template <int LOGN>
struct TcSmem {
    static constexpr int N = 1 << LOGN;
    static constexpr int US = N + 8;       // digit tile row stride (elements): rows 16 bytes apart mod 128
    static constexpr int CS = 2 * N + 32;  // Toeplitz source copy stride (elements): copies 16 banks apart
    static constexpr size_t bytes = sizeof(__nv_bfloat16) * ((size_t)TC_GT * US + 8 * (size_t)CS);
};

__device__ __forceinline__ uint32_t gadget_offset(uint32_t bg_bit) {
    uint32_t off = 0;
    for (uint32_t l = 1; l <= 3; ++l) off += (1u << (bg_bit - 1)) << (32 - bg_bit * l);
    if (3 * bg_bit < 32) off += 1u << (32 - 3 * bg_bit - 1);
    return off;
}

// Digit l (0 = most significant) of the signed base-2^bg_bit decomposition.
__device__ __forceinline__ int32_t gadget_digit(uint32_t x, int l, uint32_t bg_bit, uint32_t offset) {
    const uint32_t xp = x + offset;
    return (int32_t)((xp >> (32 - bg_bit * (l + 1))) & ((1u << bg_bit) - 1)) - (int32_t)(1u << (bg_bit - 1));
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[3], uint32_t b0, uint32_t b1) {
    // A registers {a0, a1, a2, a3}; Toeplitz tiles have a3 == a0
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%4}, {%7,%8}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(s));
}

// Grid (N / TC_MS, G / TC_GT, outputs), TC_THREADS threads.
// Shared memory: the CTA's digit tile [64 gates][N] and, per byte plane b,
// two copies of the reversed extended plane R_b[y] = ext_b[-y] (the second
// shifted by one element), so that the two bf16 elements of every A register
// are one aligned 32-bit load: element (row m, column t) of T is R[t - m].
template <int LOGN>
__global__ void __launch_bounds__(TC_THREADS, 1) tc_products_kernel(TcArgs A, uint32_t G) {
    using L = TcSmem<LOGN>;
    constexpr int N = L::N, US = L::US, CS = L::CS;
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16 *Us = reinterpret_cast<__nv_bfloat16 *>(smem);
    __nv_bfloat16 *R = Us + TC_GT * US;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int grp = lane >> 2, tig = lane & 3;
    const int type = blockIdx.z & 1, zi = blockIdx.z >> 1;
    const int g0 = blockIdx.y * TC_GT;
    const int mw = blockIdx.x * TC_MS + (warp & 3) * 64;  // this warp's 64 output rows
    const int gw = (warp >> 2) * 32;                        // and 32 gates of the tile
    const uint32_t *keyz = type ? A.key[1] + zi * A.key_zstride[1] : A.key[0] + zi * A.key_zstride[0];
    const __nv_bfloat16 *digz = reinterpret_cast<const __nv_bfloat16 *>(A.dig) + zi * A.dig_zstride + (size_t)g0 * N;

    uint32_t iacc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) iacc[i][nt][r] = 0;

    // ldmatrix row of this lane: matrix q = lane / 8 covers n-tile (q / 2) of a
    // pair and k half (q % 2)
    const int lrow = gw + ((lane >> 4) * 8) + (lane & 7), lcol = ((lane >> 3) & 1) * 8;

#pragma unroll 1
    for (int c = 0; c < A.nchunks; ++c) {
        const uint32_t *key = keyz + (size_t)c * N;
        const __nv_bfloat16 *dig = digz + (size_t)c * G * N;
        __syncthreads();  // the previous chunk's tiles are no longer read
        for (int x = tid; x < TC_GT * (N / 8); x += TC_THREADS) {
            const int g = x / (N / 8), q = x % (N / 8);
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(dig + (size_t)g * N) + q);
            *reinterpret_cast<uint4 *>(Us + g * US + q * 8) = v;
        }
        for (int y = tid - (N - 1); y <= N - 1; y += TC_THREADS) {
            const int x = -y;  // R[y] = ext[-y]
            uint32_t v = key[x >= 0 ? x : x + N];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int by = (int)(int8_t)(uint8_t)(v & 0xFFu);
                v = (v - (uint32_t)by) >> 8;
                const __nv_bfloat16 h = __int2bfloat16_rn(x >= 0 ? by : -by);
                R[(2 * b) * CS + N + y] = h;          // copy 0: index N + y in [1, 2N - 1]
                R[(2 * b + 1) * CS + N + y - 1] = h;  // copy 1 holds R[z + 1] at z: index in [0, 2N - 2]
            }
        }
        __syncthreads();
#pragma unroll 1
        for (int b = 0; b < 4; ++b) {
            // Fragment of the tile with t0 - m0 = delta: register a0 holds
            // R[delta + 2 tig - grp] and the next element, a1 the same at -8,
            // a2 at +8, a3 = a0.  The parity of the index is that of grp.
            const __nv_bfloat16 *P =
                ((grp & 1) ? R + (2 * b + 1) * CS + N - 1 : R + (2 * b) * CS + N) + 2 * tig - grp;
            auto frag = [&](uint32_t (&a)[3], int delta) {
                a[0] = *reinterpret_cast<const uint32_t *>(P + delta);
                a[1] = *reinterpret_cast<const uint32_t *>(P + delta - 8);
                a[2] = *reinterpret_cast<const uint32_t *>(P + delta + 8);
            };
            float f[4][4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                    for (int r = 0; r < 4; ++r) f[i][nt][r] = 0.f;
            // m-tile i at k-step s has delta = 16 (s - i) - mw: fr[j & 3] holds j = s - i
            uint32_t fr[4][3];
            frag(fr[3], -16 - mw);
            frag(fr[2], -32 - mw);
            frag(fr[1], -48 - mw);
#pragma unroll 1
            for (int s4 = 0; s4 < N / 16; s4 += 4) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int s = s4 + u;
                    frag(fr[u], 16 * s - mw);
                    uint32_t bq[4][2];
                    ldmatrix_x4(bq[0][0], bq[0][1], bq[1][0], bq[1][1], Us + lrow * US + 16 * s + lcol);
                    ldmatrix_x4(bq[2][0], bq[2][1], bq[3][0], bq[3][1], Us + (lrow + 16) * US + 16 * s + lcol);
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int nt = 0; nt < 4; ++nt) mma_bf16_16816(f[i][nt], fr[(u - i) & 3], bq[nt][0], bq[nt][1]);
                }
            }
            // |f| <= 2^24: exact integers
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                    for (int r = 0; r < 4; ++r) iacc[i][nt][r] += (uint32_t)__float2int_rn(f[i][nt][r]) << (8 * b);
        }
    }
    int32_t *dst = (type ? A.dst[1] : A.dst[0]) + zi * A.dst_zstride;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = mw + 16 * i + grp + ((r & 2) ? 8 : 0);
                const int g = g0 + gw + nt * 8 + 2 * tig + (r & 1);
                int32_t *d = dst + (size_t)g * A.dst_stride + row;
                *d = A.accumulate ? (int32_t)((uint32_t)*d + iacc[i][nt][r]) : (int32_t)iacc[i][nt][r];
            }
}

// ACC_jj (+= C_jj, or the initial (X^-bbar testv, 0, ..., 0) when init), then,
// for step >= 0, the digits of (X^-e - 1) ACC_jj with e = abar[step] into
// U[jj][l][g][.].  Grid (G, k + 1).
template <int LOGN>
__global__ void tc_rotate_digits_kernel(uint32_t k, uint32_t W, uint32_t G, int step, int init, uint32_t bg_bit,
                                        const uint32_t *__restrict__ abar, uint32_t *__restrict__ acc,
                                        const int32_t *__restrict__ C, __nv_bfloat16 *__restrict__ U) {
    constexpr int N = 1 << LOGN;
    __shared__ uint32_t a[N];
    const uint32_t g = blockIdx.x, jj = blockIdx.y;
    uint32_t *ap = acc + ((size_t)g * (k + 1) + jj) * N;
    const int32_t *cp = C ? C + ((size_t)g * (k + 1) + jj) * N : nullptr;
    const uint32_t bbar = abar[(size_t)g * W + W - 1];
    for (int m = threadIdx.x; m < N; m += blockDim.x) {
        uint32_t v;
        if (init) {
            uint32_t r = m + bbar;  // X^-bbar * (1/8) sum X^m
            if (r >= 2 * N) r -= 2 * N;
            v = jj ? 0u : ((r >= (uint32_t)N) ? (0u - (1u << 29)) : (1u << 29));
        } else {
            v = ap[m] + (cp ? (uint32_t)cp[m] : 0u);
        }
        a[m] = v;
        if (init || cp) ap[m] = v;
    }
    if (step < 0) return;
    __syncthreads();
    const uint32_t e = abar[(size_t)g * W + step];
    const uint32_t off = gadget_offset(bg_bit);
    for (int m = threadIdx.x; m < N; m += blockDim.x) {
        uint32_t r = m + e;
        if (r >= 2 * N) r -= 2 * N;
        uint32_t x = a[r & (N - 1)];
        if (r >= (uint32_t)N) x = 0u - x;
        const uint32_t D = x - a[m];
#pragma unroll
        for (int l = 0; l < 3; ++l)
            U[(((size_t)jj * 3 + l) * G + g) * N + m] = __int2bfloat16_rn(gadget_digit(D, l, bg_bit, off));
    }
}

// w = g^-1(sum_jj V_jj) into Wd[l][g][.].  Grid G.
template <int LOGN>
__global__ void tc_vdigits_kernel(uint32_t k, uint32_t G, uint32_t bg_bit, const int32_t *__restrict__ V,
                                  __nv_bfloat16 *__restrict__ Wd) {
    constexpr int N = 1 << LOGN;
    const uint32_t g = blockIdx.x;
    const uint32_t off = gadget_offset(bg_bit);
    for (int m = threadIdx.x; m < N; m += blockDim.x) {
        uint32_t v = 0;
        for (uint32_t jj = 0; jj <= k; ++jj) v += (uint32_t)V[((size_t)g * (k + 1) + jj) * N + m];
#pragma unroll
        for (int l = 0; l < 3; ++l) Wd[((size_t)l * G + g) * N + m] = __int2bfloat16_rn(gadget_digit(v, l, bg_bit, off));
    }
}

// SampleExtract of ACC and +1/8 into ext [count][k N + 1].  Grid count.
template <int LOGN>
__global__ void tc_extract_kernel(uint32_t k, const uint32_t *__restrict__ acc, uint32_t *__restrict__ ext) {
    constexpr int N = 1 << LOGN;
    const uint32_t g = blockIdx.x;
    const uint32_t *a = acc + (size_t)g * (k + 1) * N;
    uint32_t *d = ext + (size_t)g * (k * N + 1);
    for (uint32_t i = 1; i <= k; ++i)
        for (int m = threadIdx.x; m < N; m += blockDim.x) d[(i - 1) * N + m] = (m == 0) ? a[i * N] : 0u - a[i * N + N - m];
    if (threadIdx.x == 0) d[k * N] = a[0] + (1u << 29);
}

__global__ void tc_int8_to_bf16_kernel(const int8_t *__restrict__ src, __nv_bfloat16 *__restrict__ dst, size_t count) {
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < count; x += (size_t)gridDim.x * blockDim.x)
        dst[x] = __int2bfloat16_rn((int)src[x]);
}

// Independent bf16 m16n8k16 MMAs from registers (tensor ceiling of this form).
__global__ void mma_peak_kernel(uint32_t iters, float *sink) {
    uint32_t a[3] = {0x3F803F80u ^ threadIdx.x, 0x40003F80u, 0x3F804000u};
    const uint32_t b0 = 0x3F803F80u, b1 = 0x40004000u;
    float d[8][4];
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) d[q][r] = 0.f;
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < 8; ++q) mma_bf16_16816(d[q], a, b0, b1);
        a[0] += 1u;
    }
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += d[q][0] + d[q][1] + d[q][2] + d[q][3];
    if (s == 1234.5f) sink[blockIdx.x] = s;  // keeps the loop live; practically never stores
}

template <int LOGN>
cudaError_t set_products_smem() {
    return cudaFuncSetAttribute(tc_products_kernel<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)TcSmem<LOGN>::bytes);
}

template <int LOGN>
void launch_products(const TcArgs &A, uint32_t G, int outputs, cudaStream_t st) {
    constexpr int N = 1 << LOGN;
    tc_products_kernel<LOGN><<<dim3(N / TC_MS, G / TC_GT, outputs), TC_THREADS, TcSmem<LOGN>::bytes, st>>>(A, G);
}

// Engine 1: tcgen05 (G a multiple of 128); otherwise warp-level mma.sync.
template <int LOGN>
cudaError_t products(int engine, const TcArgs &A, uint32_t G, int outputs, cudaStream_t st) {
    if (engine == 1) return launch_products_tc05(A, 1u << LOGN, G, outputs, st);
    launch_products<LOGN>(A, G, outputs, st);
    return cudaSuccess;
}

// Workspace carve-up for a wave of Gp gates (multiple of TC_GT).
struct TcWave {
    uint32_t *abar;       // [Gp][W]
    uint32_t *acc;        // [Gp][k+1][N]
    int32_t *C;           // [Gp][k+1][N]
    int32_t *V;           // [Gp][k+1][N]
    __nv_bfloat16 *U;     // [k+1][3][Gp][N]
    __nv_bfloat16 *Wd;    // [3][Gp][N]
};

TcWave carve(void *ws, uint32_t Gp, const LaunchShape &S) {
    const size_t W = (size_t)S.k * S.n + 1, poly = (size_t)Gp * (S.k + 1) * S.N;
    TcWave w;
    w.abar = static_cast<uint32_t *>(ws);
    w.acc = w.abar + ((Gp * W + 63) & ~size_t(63));
    w.C = reinterpret_cast<int32_t *>(w.acc + poly);
    w.V = w.C + poly;
    w.U = reinterpret_cast<__nv_bfloat16 *>(w.V + poly);
    w.Wd = w.U + 3 * poly;
    return w;
}

// The rotation of one wave (Gp gates) from w.abar; ACC left in w.acc.
template <int LOGN>
cudaError_t blind_rotate_wave(const LaunchShape &S, const DeviceKeys &K, const TcWave &w, uint32_t Gp,
                              int64_t max_steps, cudaStream_t st) {
    constexpr int N = 1 << LOGN;
    const uint32_t k = S.k, n = S.n, W = k * n + 1;
    const uint32_t *bk_all = static_cast<const uint32_t *>(K.bk);
    const uint32_t *keyA = static_cast<const uint32_t *>(K.keyA);
    cudaError_t e = set_products_smem<LOGN>();
    if (e != cudaSuccess) return e;
    const int64_t total = (int64_t)k * n;
    const int64_t steps = (max_steps >= 0 && max_steps < total) ? max_steps : total;
    tc_rotate_digits_kernel<LOGN><<<dim3(Gp, k + 1), 256, 0, st>>>(k, W, Gp, steps > 0 ? 0 : -1, 1, S.bg_bit,
                                                                    w.abar, w.acc, nullptr, w.U);
    for (int64_t step = 0; step < steps; ++step) {
        const uint32_t i = (uint32_t)(step / n) + 1;
        const uint32_t *bk = bk_all + (size_t)step * 9 * N;  // d[3], f0[3], f1[3] of BK_{i,j}
        TcArgs a{};
        a.dst[0] = w.C;
        a.dst[1] = w.V;
        a.dst_zstride = N;
        a.dst_stride = (k + 1) * N;
        a.accumulate = 0;
        a.key[0] = bk;
        a.key_zstride[0] = 0;
        a.key[1] = keyA;
        a.key_zstride[1] = 3 * (size_t)N;
        a.dig = reinterpret_cast<const uint16_t *>(w.U);
        a.dig_zstride = 3 * (size_t)Gp * N;
        a.nchunks = 3;
        a.dig_chunks = 3 * (int)(k + 1);
        a.wait_ns = S.wait_ns;
        e = products<LOGN>(S.variant, a, Gp, 2 * (int)(k + 1), st);
        if (e != cudaSuccess) return e;
        tc_vdigits_kernel<LOGN><<<Gp, 256, 0, st>>>(k, Gp, S.bg_bit, w.V, w.Wd);
        TcArgs b{};
        b.dst[0] = w.C;
        b.dst[1] = w.C + (size_t)i * N;
        b.dst_zstride = 0;
        b.dst_stride = (k + 1) * N;
        b.accumulate = 1;
        b.key[0] = bk + 3 * (size_t)N;
        b.key[1] = bk + 6 * (size_t)N;
        b.key_zstride[0] = b.key_zstride[1] = 0;
        b.dig = reinterpret_cast<const uint16_t *>(w.Wd);
        b.dig_zstride = 0;
        b.nchunks = 3;
        b.dig_chunks = 3;
        b.wait_ns = S.wait_ns;
        e = products<LOGN>(S.variant, b, Gp, 2, st);
        if (e != cudaSuccess) return e;
        const int next = (step + 1 < steps) ? (int)(step + 1) : -1;
        tc_rotate_digits_kernel<LOGN><<<dim3(Gp, k + 1), 256, 0, st>>>(k, W, Gp, next, 0, S.bg_bit, w.abar, w.acc,
                                                                        w.C, w.U);
    }
    return cudaGetLastError();
}

template <int LOGN>
cudaError_t bootstrap_tc(const LaunchShape &S, const DeviceKeys &K, const GateDesc *desc, const uint32_t *ct_a,
                         const uint32_t *ct_b, const uint32_t *abar_in, int64_t max_steps, uint32_t *ext,
                         uint32_t *acc_out, uint32_t count, cudaStream_t st) {
    constexpr int N = 1 << LOGN;
    const uint32_t k = S.k, W = k * S.n + 1, cap = K.tc_ws_gates;
    for (uint32_t start = 0; start < count; start += cap) {
        const uint32_t cnt = count - start < cap ? count - start : cap;
        const uint32_t Gp = (cnt + TC_PAD - 1) / TC_PAD * TC_PAD;
        const TcWave w = carve(K.tc_ws, Gp, S);
        cudaError_t e;
        if (abar_in)
            e = cudaMemcpyAsync(w.abar, abar_in + (size_t)start * W, (size_t)cnt * W * 4, cudaMemcpyDeviceToDevice, st);
        else
            e = launch_modswitch(S, desc + start, ct_a, ct_b, w.abar, cnt, st);
        if (e == cudaSuccess && Gp > cnt)  // padding gates: rotation by 0, results unused
            e = cudaMemsetAsync(w.abar + (size_t)cnt * W, 0, (size_t)(Gp - cnt) * W * 4, st);
        if (e == cudaSuccess) e = blind_rotate_wave<LOGN>(S, K, w, Gp, max_steps, st);
        if (e != cudaSuccess) return e;
        if (acc_out) {
            e = cudaMemcpyAsync(acc_out + (size_t)start * (k + 1) * N, w.acc, (size_t)cnt * (k + 1) * N * 4,
                                cudaMemcpyDeviceToDevice, st);
        } else {
            tc_extract_kernel<LOGN><<<cnt, 256, 0, st>>>(k, w.acc, ext + (size_t)start * (k * N + 1));
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

size_t tc_workspace_bytes(const LaunchShape &S, uint32_t gates) {
    const uint32_t Gp = (gates + TC_PAD - 1) / TC_PAD * TC_PAD;
    const size_t W = (size_t)S.k * S.n + 1, poly = (size_t)Gp * (S.k + 1) * S.N;
    return 4 * (((Gp * W + 63) & ~size_t(63)) + 3 * poly) + 2 * (3 * poly + 3 * (size_t)Gp * S.N);
}

uint32_t tc_wave_granularity() { return TC_PAD; }

bool tc_shape_supported(const LaunchShape &S) {
    // exactness needs |digit| * |key byte| * N <= 2^24: digits of at most 8 bits, N <= 1024
    return (S.N == 256 || S.N == 1024) && S.d == 3 && S.bg_bit >= 2 && S.bg_bit <= 8 && S.k >= 1 && S.k <= 8;
}

cudaError_t launch_bootstrap_tc(const LaunchShape &S, const DeviceKeys &K, const GateDesc *desc, const uint32_t *ct_a,
                                const uint32_t *ct_b, const uint32_t *abar_in, int64_t max_steps, uint32_t *ext,
                                uint32_t *acc_out, uint32_t count, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    if (!tc_shape_supported(S) || !K.tc_ws || K.tc_ws_gates == 0 || K.tc_ws_gates % TC_PAD) return cudaErrorInvalidValue;
    if (S.N == 256) return bootstrap_tc<8>(S, K, desc, ct_a, ct_b, abar_in, max_steps, ext, acc_out, count, st);
    return bootstrap_tc<10>(S, K, desc, ct_a, ct_b, abar_in, max_steps, ext, acc_out, count, st);
}

cudaError_t launch_negacyclic_tc(uint32_t N, uint32_t G, uint32_t nchunks, const uint32_t *keys, const int8_t *digits,
                                 int32_t *out, void *work, int engine, cudaStream_t st) {
    if ((N != 256 && N != 1024) || G == 0 || G % (engine == 1 ? 128 : TC_GT) || nchunks == 0 || nchunks > 3)
        return cudaErrorInvalidValue;
    __nv_bfloat16 *d = static_cast<__nv_bfloat16 *>(work);
    const size_t total = (size_t)nchunks * G * N;
    tc_int8_to_bf16_kernel<<<1024, 256, 0, st>>>(digits, d, total);
    TcArgs a{};
    a.dst[0] = a.dst[1] = out;
    a.dst_stride = N;
    a.key[0] = a.key[1] = keys;
    a.dig = reinterpret_cast<const uint16_t *>(d);
    a.nchunks = (int)nchunks;
    a.dig_chunks = (int)nchunks;
    a.wait_ns = 1000000000ull;  // 1 s
    if (engine == 1) return launch_products_tc05(a, N, G, 1, st);
    cudaError_t e = N == 256 ? set_products_smem<8>() : set_products_smem<10>();
    if (e != cudaSuccess) return e;
    if (N == 256) launch_products<8>(a, G, 1, st);
    else launch_products<10>(a, G, 1, st);
    return cudaGetLastError();
}

cudaError_t launch_mma_peak(uint32_t blocks, uint32_t threads, uint32_t iters, float *sink, cudaStream_t st) {
    mma_peak_kernel<<<blocks, threads, 0, st>>>(iters, sink);
    return cudaGetLastError();
}

}  // namespace mk
