// mk_bootstrap_split.cuh -- the two-prime blind rotation with the primes
// split across warps.
//
// Same arithmetic and results as bootstrap_ntt_kernel over FieldDual (gate
// linear part and modulus switch, Sec. 4.1, Eq. 6-11; the CMux steps
// ACC += HP((X^-e - 1) ACC, BK_{i,j}) of GB, Sec. 3.2, with the MKTFHE hybrid
// product; SampleExtract and +1/8).  There one thread carries both residues
// of its eight elements through every transform, which takes about 168
// registers and leaves room for 12 warps per SM; the kernel waits mostly on
// fixed-latency dependencies that more warps would hide.  Here a gate has
// 2 N/8 threads: the first N/8 run every transform mod p1, the second N/8
// mod p2, each with one 32-bit residue per element, so a thread needs about
// half the registers.  Both halves read the accumulator and derive the same
// digits (that work is done twice); each reads its own plane of the keys and
// its own twiddles.  After each inverse transform the halves swap residues
// through shared memory and each recombines (CRT) half of the elements.
#pragma once
#include "mk_bootstrap.cuh"

namespace mk {
namespace br {

// One prime of the two-prime form, as warp-uniform values.
struct PrimeOne {
    uint32_t p, twop, pinv;
};

// Negacyclic transforms over one prime: EPT = 8 elements per thread, T = N/8
// threads, the pass structure and index conventions of Ntt<F, LOGN, true, 8>.
template <int LOGN>
struct NttOne {
    static constexpr int N = 1 << LOGN, EPT = 8, SB = 3, T = N / EPT;
    static constexpr int PN = padded_len(N);  // padded polynomial stride in the exchange buffer

    // Harvey/Shoup butterflies: forward inputs and outputs in [0, 4p); inverse in [0, 2p).
    __device__ static __forceinline__ void fwd(uint32_t &X, uint32_t &Y, const uint2 &W, const PrimeOne &P) {
        const uint32_t x = red2p(X, P.twop);
        const uint32_t t = shoup(Y, W.x, W.y, P.p);
        X = x + t;
        Y = x - t + P.twop;
    }
    __device__ static __forceinline__ void inv(uint32_t &X, uint32_t &Y, const uint2 &W, const PrimeOne &P) {
        const uint32_t u = X, v = Y;
        X = red2p(u + v, P.twop);
        Y = shoup(u - v + P.twop, W.x, W.y, P.p);
    }

    template <int NP, int D, bool FWD>
    __device__ static __forceinline__ void stage(uint32_t (&x)[NP][EPT], int jb, int b, const uint2 *tw,
                                                 const PrimeOne &P) {
        constexpr int NT = EPT / (2 * D), SH = (D == 4 ? 3 : (D == 2 ? 2 : 1));
        const int base = (1 << (LOGN - 1 - b)) + (jb >> (b + 1));
        uint2 S[NT];
#pragma unroll
        for (int q = 0; q < NT; ++q) S[q] = __ldg(tw + base + q);
#pragma unroll
        for (int c = 0; c < EPT; ++c) {
            if (c & D) continue;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                if constexpr (FWD) fwd(x[p][c], x[p][c + D], S[c >> SH], P);
                else inv(x[p][c], x[p][c + D], S[c >> SH], P);
            }
        }
    }

    template <int NP>
    __device__ static __forceinline__ void exchange(uint32_t (&x)[NP][EPT], int tid, uint32_t *buf, int LOf, int LOt,
                                                    int bar_id) {
        const int bf = jbase<SB>(tid, LOf);
#pragma unroll
        for (int p = 0; p < NP; ++p)
#pragma unroll
            for (int c = 0; c < EPT; ++c) buf[p * PN + pidx(bf | (c << LOf))] = x[p][c];
        group_sync(bar_id, T);
        const int bt = jbase<SB>(tid, LOt);
#pragma unroll
        for (int p = 0; p < NP; ++p)
#pragma unroll
            for (int c = 0; c < EPT; ++c) x[p][c] = buf[p * PN + pidx(bt | (c << LOt))];
        group_sync(bar_id, T);
    }

    // natural (layout logN-3) -> bit-reversed (layout 0)
    template <int NP>
    __device__ static __forceinline__ void forward(uint32_t (&x)[NP][EPT], int tid, const uint2 *tw, uint32_t *buf,
                                                   int bar_id, const PrimeOne &P) {
        int prev = LOGN - SB;
#pragma unroll 1
        for (int hi = LOGN - 1; hi >= 0; hi -= SB) {
            const int LO = hi >= SB - 1 ? hi - (SB - 1) : 0;
            if (LO != prev) exchange<NP>(x, tid, buf, prev, LO, bar_id);
            const int jb = jbase<SB>(tid, LO);
            if (hi - LO == 2) stage<NP, 4, true>(x, jb, LO + 2, tw, P);
            if (hi - LO >= 1) stage<NP, 2, true>(x, jb, LO + 1, tw, P);
            stage<NP, 1, true>(x, jb, LO, tw, P);
            prev = LO;
        }
    }

    // bit-reversed (layout 0) -> natural (layout logN-3), without 1/N
    template <int NP>
    __device__ static __forceinline__ void inverse(uint32_t (&x)[NP][EPT], int tid, const uint2 *tw, uint32_t *buf,
                                                   int bar_id, const PrimeOne &P) {
        int prev = 0;
#pragma unroll 1
        for (int lo = 0; lo < LOGN; lo += SB) {
            const int hi = (lo + SB - 1 < LOGN - 1) ? lo + SB - 1 : LOGN - 1;
            const int LO = (lo < LOGN - SB) ? lo : LOGN - SB;
            if (LO != prev) exchange<NP>(x, tid, buf, prev, LO, bar_id);
            const int jb = jbase<SB>(tid, LO);
            if (lo == LO) stage<NP, 1, false>(x, jb, LO, tw, P);
            if (lo <= LO + 1 && hi >= LO + 1) stage<NP, 2, false>(x, jb, LO + 1, tw, P);
            if (hi == LO + 2) stage<NP, 4, false>(x, jb, LO + 2, tw, P);
            prev = LO;
        }
    }
};

// A += x * key over thread tid's eight elements of one key plane (Montgomery
// form; plane_unit_pos layout).
template <int LOGN>
__device__ __forceinline__ void mac_plane(uint32_t (&A)[8], const uint32_t (&x)[8], const uint32_t *__restrict__ plane,
                                          int tid, const PrimeOne &P) {
    constexpr int N = 1 << LOGN;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(plane);
    const uint4 a = __ldg(s4 + tid), b = __ldg(s4 + N / 8 + tid);
    const uint32_t kv[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
    for (int c = 0; c < 8; ++c) A[c] = red2p(A[c] + montmul(x[c], kv[c], P.p, P.pinv), P.twop);
}

// Garner CRT of residues r1 mod p1, r2 mod p2 (each in [0, 2p)) to the exact
// integer in (-p1 p2 / 2, p1 p2 / 2), reduced mod 2^32.
__device__ __forceinline__ uint32_t crt_u32(uint32_t r1, uint32_t r2) {
    return FieldDual::to_u32(make_uint2(r1, r2));
}

struct SplitLayout {
    size_t xbuf, xwords, acc, vbuf, abar, total;
};

template <int LOGN, int NPF>
__host__ __device__ inline SplitLayout split_layout(uint32_t k, uint32_t n) {
    constexpr size_t N = (size_t)1 << LOGN;
    SplitLayout L;
    L.xwords = (NPF > 2 ? NPF : 2) * padded_len(N);  // one prime's exchange buffer, in words
    L.xbuf = 0;
    L.acc = L.xbuf + 2 * sizeof(uint32_t) * L.xwords;
    L.vbuf = L.acc + sizeof(uint32_t) * (k + 1) * N;
    L.abar = L.vbuf + sizeof(uint32_t) * N;
    L.total = L.abar + ((sizeof(uint16_t) * (k * n + 1) + 15) & ~size_t(15));
    return L;
}

// After an inverse transform of NO outputs (y), the two halves swap residues
// and each recombines elements c in [4 pi, 4 pi + 4) of its eight: output o
// goes to dst[o][m] (added when add[o], stored otherwise).  Both CTA barriers
// are part of the protocol: the first makes the other half's residues visible
// (and ends both halves' use of their exchange buffers), the second ends the
// reads of this buffer before the next transform overwrites it and makes the
// results visible to both halves.
template <int LOGN, int NO, int KEEP>
__device__ __forceinline__ void crt_swap_half(uint32_t (&y)[NO][8], int tid, uint32_t *mine, const uint32_t *other,
                                              uint32_t *dst0, bool add0, uint32_t *dst1, bool add1) {
    constexpr int N = 1 << LOGN, T = N / 8, GIVE = 4 - KEEP;
#pragma unroll
    for (int o = 0; o < NO; ++o)
#pragma unroll
        for (int c = 0; c < 4; ++c) mine[o * N + tid + T * (GIVE + c)] = y[o][GIVE + c];
    __syncthreads();
#pragma unroll
    for (int o = 0; o < NO; ++o) {
        uint32_t *dst = o == 0 ? dst0 : dst1;
        const bool add = o == 0 ? add0 : add1;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int m = tid + T * (KEEP + c);
            const uint32_t r_own = y[o][KEEP + c], r_other = other[o * N + m];
            const uint32_t v = KEEP ? crt_u32(r_other, r_own) : crt_u32(r_own, r_other);
            dst[m] = add ? dst[m] + v : v;
        }
    }
    __syncthreads();
}

// The p1 half keeps elements 0-3 of its eight, the p2 half 4-7 (compile-time
// indices, so y stays in registers).
template <int LOGN, int NO>
__device__ __forceinline__ void crt_swap(uint32_t (&y)[NO][8], int pi, int tid, uint32_t *mine, const uint32_t *other,
                                         uint32_t *dst0, bool add0, uint32_t *dst1, bool add1) {
    if (pi == 0) crt_swap_half<LOGN, NO, 0>(y, tid, mine, other, dst0, add0, dst1, add1);
    else crt_swap_half<LOGN, NO, 4>(y, tid, mine, other, dst0, add0, dst1, add1);
}

// One CMux step (party i, rotation e != 0) of this half's prime; slot order
// and transform pairing as cmux_step.
template <int LOGN, int NPF>
__device__ __forceinline__ void split_step(const LaunchShape &S, const uint32_t *bk, const uint32_t *keyA,
                                           const Gadget &Gd, int i, uint32_t e, uint32_t *acc, uint32_t *vbuf,
                                           uint32_t *mine, const uint32_t *other, const uint2 *twf, const uint2 *twi,
                                           int pi, int tid, const PrimeOne &P) {
    using NT = NttOne<LOGN>;
    constexpr int N = NT::N, T = NT::T, EPT = 8;
    const int k = (int)S.k, bar_id = 1 + pi;
    const size_t poly = 2 * (size_t)N;  // words per key polynomial (two planes)
    uint32_t C0[EPT], CI[EPT], CJ[EPT], V[EPT];
#pragma unroll
    for (int c = 0; c < EPT; ++c) C0[c] = CI[c] = CJ[c] = V[c] = 0;
#pragma unroll 1
    for (int q = 0; q <= k + 1; ++q) {
        const int jj = (q == 0) ? 0 : (q == 1 ? i : (q - 1 < i ? q - 1 : q));  // q <= k only
        if (q >= 2 && q <= k) {
#pragma unroll
            for (int c = 0; c < EPT; ++c) CJ[c] = 0;
        }
#pragma unroll 1
        for (int l0 = 0; l0 < 3; l0 += NPF) {
            uint32_t x[NPF][EPT];
#pragma unroll
            for (int c = 0; c < EPT; ++c) {
                const uint32_t m = tid + T * c;
                uint32_t D;
                if (q <= k) {
                    const uint32_t *ap = acc + jj * N;
                    uint32_t r = m + e;
                    if (r >= 2 * N) r -= 2 * N;
                    uint32_t a = ap[r & (N - 1)];
                    if (r >= N) a = 0u - a;
                    D = a - ap[m];
                } else {
                    D = vbuf[m];
                }
#pragma unroll
                for (int p = 0; p < NPF; ++p) x[p][c] = P.p + (uint32_t)Gd.digit(D, l0 + p);
            }
            NT::template forward<NPF>(x, tid, twf, mine, bar_id, P);
#pragma unroll
            for (int p = 0; p < NPF; ++p) {
                const int l = l0 + p;
                if (q <= k) {
                    const uint32_t *kd = bk + l * poly + pi * N;                          // d_l
                    const uint32_t *ka = keyA + ((size_t)jj * 3 + l) * poly + pi * N;     // -a_l or pk_jj[l]
                    if (q == 0) mac_plane<LOGN>(C0, x[p], kd, tid, P);
                    else if (q == 1) mac_plane<LOGN>(CI, x[p], kd, tid, P);
                    else mac_plane<LOGN>(CJ, x[p], kd, tid, P);
                    mac_plane<LOGN>(V, x[p], ka, tid, P);
                } else {
                    mac_plane<LOGN>(C0, x[p], bk + (3 + l) * poly + pi * N, tid, P);  // f0_l
                    mac_plane<LOGN>(CI, x[p], bk + (6 + l) * poly + pi * N, tid, P);  // f1_l
                }
            }
        }
        const bool pair = (q == k && k >= 2) || q == k + 1;
        const bool single = (q >= 2 && q < k) || (q == k && k == 1);
        if (pair) {
            const bool last = (q == k + 1);
            uint32_t y[2][EPT];
#pragma unroll
            for (int c = 0; c < EPT; ++c) {
                y[0][c] = last ? C0[c] : CJ[c];
                y[1][c] = last ? CI[c] : V[c];
            }
            NT::template inverse<2>(y, tid, twi, mine, bar_id, P);
            crt_swap<LOGN, 2>(y, pi, tid, mine, other, acc + (last ? 0 : jj) * N, true, last ? acc + i * N : vbuf,
                              last);
        } else if (single) {
            const bool is_v = (q == k);
            uint32_t y[1][EPT];
#pragma unroll
            for (int c = 0; c < EPT; ++c) y[0][c] = is_v ? V[c] : CJ[c];
            NT::template inverse<1>(y, tid, twi, mine, bar_id, P);
            crt_swap<LOGN, 1>(y, pi, tid, mine, other, is_v ? vbuf : acc + jj * N, !is_v, nullptr, false);
        }
    }
}

// One CTA of 2 N/8 threads per gate; inputs and outputs as bootstrap_ntt_kernel.
template <int LOGN, int NPF, int MINB>
__global__ void __launch_bounds__(2 * ((1 << LOGN) / 8), MINB)
bootstrap_split_kernel(LaunchShape S, DeviceKeys K, const GateDesc *__restrict__ desc,
                       const uint32_t *__restrict__ ct_a, const uint32_t *__restrict__ ct_b,
                       const uint32_t *__restrict__ abar_in, int64_t max_steps, uint32_t *__restrict__ ext,
                       uint32_t *__restrict__ acc_out) {
    constexpr int N = 1 << LOGN, T = N / 8, EPT = 8;
    extern __shared__ __align__(16) unsigned char smem[];
    const int pi = threadIdx.x / T, tid = threadIdx.x % T;
    const SplitLayout L = split_layout<LOGN, NPF>(S.k, S.n);
    uint32_t *xall = reinterpret_cast<uint32_t *>(smem + L.xbuf);
    uint32_t *mine = xall + pi * L.xwords;
    const uint32_t *other = xall + (1 - pi) * L.xwords;
    uint32_t *acc = reinterpret_cast<uint32_t *>(smem + L.acc);
    uint32_t *vbuf = reinterpret_cast<uint32_t *>(smem + L.vbuf);
    uint16_t *abar = reinterpret_cast<uint16_t *>(smem + L.abar);
    const PrimeOne P = pi ? PrimeOne{P2, TWO_P2, PINV2} : PrimeOne{P1, TWO_P1, PINV1};
    const uint2 *tws = static_cast<const uint2 *>(K.tw_split);
    const uint2 *twf = tws + (size_t)pi * N, *twi = tws + (size_t)(2 + pi) * N;
    const uint32_t *bk_all = static_cast<const uint32_t *>(K.bk);
    const uint32_t *keyA = static_cast<const uint32_t *>(K.keyA);

    if (abar_in) {
        const uint32_t W = S.k * S.n + 1;
        for (uint32_t x = threadIdx.x; x < W; x += 2 * T) abar[x] = (uint16_t)abar_in[(size_t)blockIdx.x * W + x];
    } else {
        lin_modswitch(S, desc[blockIdx.x], ct_a, ct_b, abar, threadIdx.x, 2 * T);
    }
    __syncthreads();
    if (pi == 0) init_acc<LOGN, EPT>(acc, S.k, abar[S.k * S.n], tid);
    __syncthreads();

    const Gadget Gd = make_gadget(S.bg_bit);
    const int n = (int)S.n, k = (int)S.k;
    int64_t steps = 0;
#pragma unroll 1
    for (int i = 1; i <= k; ++i) {
#pragma unroll 1
        for (int j = 0; j < n; ++j) {
            if (max_steps >= 0 && steps >= max_steps) goto done;
            ++steps;
            const uint32_t e = abar[(i - 1) * n + j];
            if (e == 0) continue;  // X^0 - 1 = 0: every digit is 0, HP adds nothing
            const uint32_t *bk = bk_all + (size_t)((i - 1) * n + j) * 9 * 2 * N;
            split_step<LOGN, NPF>(S, bk, keyA, Gd, i, e, acc, vbuf, mine, other, twf, twi, pi, tid, P);
            __syncthreads();
        }
    }
done:
    __syncthreads();
    if (acc_out) {
        uint32_t *dst = acc_out + (size_t)blockIdx.x * (S.k + 1) * N;
        for (uint32_t x = threadIdx.x; x < (S.k + 1) * N; x += 2 * T) dst[x] = acc[x];
    } else {
        sample_extract<LOGN, 2 * T>(S, acc, ext + (size_t)blockIdx.x * (S.k * N + 1), threadIdx.x);
    }
}

template <int LOGN, int NPF, int MINB>
cudaError_t launch_split(const LaunchShape &S, const DeviceKeys &K, const GateDesc *desc, const uint32_t *ct_a,
                         const uint32_t *ct_b, const uint32_t *abar_in, int64_t max_steps, uint32_t *ext,
                         uint32_t *acc_out, uint32_t count, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    if (K.tw_split == nullptr) return cudaErrorInvalidValue;
    const SplitLayout L = split_layout<LOGN, NPF>(S.k, S.n);
    auto kern = bootstrap_split_kernel<LOGN, NPF, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return e;
    kern<<<count, 2 * ((1 << LOGN) / 8), L.total, st>>>(S, K, desc, ct_a, ct_b, abar_in, max_steps, ext, acc_out);
    return cudaGetLastError();
}

}  // namespace br
}  // namespace mk
