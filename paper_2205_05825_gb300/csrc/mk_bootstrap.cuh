// mk_bootstrap.cuh -- device building blocks of the blind rotation (NTT form).
// Included by one translation unit per ring dimension (mk_br_<N>.cu) so that
// the template instantiations compile in parallel.
//
// One CTA owns one gate for the whole blind rotation ("CTA-owns-gate"): the
// accumulator ACC (k+1 polynomials of N torus32 words) lives in shared memory
// for all k*n CMux steps, so the only L2/HBM traffic per step is the
// bootstrapping-key entry BK_{i,j} (3*d polynomials in the NTT domain) and the
// public keys.  Negacyclic products are exact: a negacyclic NTT over the
// Goldilocks prime p = 2^64 - 2^32 + 1, whose half exceeds every product sum
// (|sum| < (k+1) * d * N * 2^7 * 2^32 < 2^55), so the integer result is
// recovered exactly and reduced mod 2^32 -- bit-identical to schoolbook
// wrapping uint32 arithmetic.
//
// Code size is a first-order cost here: the step body runs k*n times per gate
// and an unrolled 1024-point NTT per call site does not fit the instruction
// caches.  So each transform direction has exactly one call site inside the
// CMux loop, and its passes run in a rolled loop (three radix-2 stages per
// pass in registers, compile-time butterfly patterns D = 4, 2, 1).
//
// Two exact fields implement the transform (template parameter F):
//   FieldGold: the prime p = 2^64 - 2^32 + 1, one 64-bit residue per element;
//   FieldDual: two 28-bit primes p1, p2 (p1 p2 > 2^55.9 > 2 |sum|, keys as
//     signed 32-bit values), a pair of 32-bit residues per element,
//     recombined by CRT after the inverse transform.  Harvey's lazy
//     butterflies (values kept in [0, 4p)) with Shoup's precomputed quotients
//     for the twiddles (two dependent multiplies); keys in Montgomery form
//     (times 2^32 mod p), so a pointwise product is three multiply-adds
//     without a second table.  (Letting forward values grow for six stages
//     before one reduction -- fewer instructions on paper -- measured slower
//     and with more executed instructions on GB300.)
// Both give the exact integer product sums, hence identical ciphertexts.
//
// Paper steps (arXiv 2205.05825): gate linear part (Sec. 4.1, Eq. 6-11,
// Algorithms 1-2), gate bootstrapping GB (Sec. 3.2).  The hybrid product
// follows the MKTFHE construction the paper builds on (named in Sec. 3.2):
// u_j = g^-1(c_j); v = -<u_0, a> + sum_{j>=1} <u_j, pk_j>; w = g^-1(v);
// c'_j = <u_j, d>; c'_0 += <w, f0>; c'_i += <w, f1>.
#pragma once
#include <type_traits>

#include "mk_internal.h"

namespace mk {
namespace br {

constexpr uint64_t P = kGoldilocks;
constexpr uint64_t EPS = 0xFFFFFFFFull;  // 2^64 mod p
constexpr uint64_t HALF_P = P >> 1;

// ------------------------------------------------------------ Goldilocks field
// Values are kept in [0, 2^64), congruent mod p but not always below p; the
// multiply reduces any 128-bit product and returns a canonical value (< p).
// add1/sub1 need their second operand canonical; add2/sub2 take any operands.
__device__ __forceinline__ uint64_t gmul(uint64_t a, uint64_t b) {
    const uint64_t lo = a * b;
    const uint64_t hi = __umul64hi(a, b);
    const uint64_t hh = hi >> 32, hl = hi & EPS;
    // x = lo + hl * 2^64 + hh * 2^96 = lo + hl * (2^32 - 1) - hh  (mod p)
    uint64_t t0 = lo - hh;
    t0 = (lo < hh) ? t0 - EPS : t0;
    const uint64_t t1 = hl * EPS;
    uint64_t r = t0 + t1;
    r = (r < t1) ? r + EPS : r;
    return (r >= P) ? r - P : r;
}

// a + b with b < p: one wrap (2^64 = EPS mod p) cannot overflow again.
__device__ __forceinline__ uint64_t add1(uint64_t a, uint64_t b) {
    const uint64_t s = a + b;
    return (s < b) ? s + EPS : s;
}

// a - b with b < p: the borrow correction (add p = subtract EPS) cannot underflow.
__device__ __forceinline__ uint64_t sub1(uint64_t a, uint64_t b) {
    const uint64_t d = a - b;
    return (a < b) ? d - EPS : d;
}

__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t s = a + b;
    if (s < a) {
        s += EPS;
        if (s < EPS) s += EPS;
    }
    return s;
}

__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
    uint64_t d = a - b;
    if (a < b) {
        const uint64_t e = d - EPS;
        d = (d < EPS) ? e - EPS : e;
    }
    return d;
}

struct FieldGold {
    using E = uint64_t;   // element
    using Tw = uint64_t;  // twiddle
    static constexpr int kForm = 0;
    __device__ static __forceinline__ E zero() { return 0; }
    __device__ static __forceinline__ E from_digit(int32_t u) {
        return u >= 0 ? (uint64_t)u : P - (uint64_t)(-(int64_t)u);
    }
    // Cooley-Tukey: (X, Y) <- (X + S Y, X - S Y)
    __device__ static __forceinline__ void fwd(E &X, E &Y, const Tw &S) {
        const uint64_t U = X, V = gmul(Y, S);
        X = add1(U, V);
        Y = sub1(U, V);
    }
    // Gentleman-Sande: (X, Y) <- (X + Y, S (X - Y))
    __device__ static __forceinline__ void inv(E &X, E &Y, const Tw &S) {
        const uint64_t U = X, V = Y;
        X = add2(U, V);
        Y = gmul(sub2(U, V), S);
    }
    // acc += x * k (k a key word)
    __device__ static __forceinline__ void mac(E &acc, const E &x, const E &k) { acc = add1(acc, gmul(x, k)); }
    // Field element of an exact integer in (-p/2, p/2) -> that integer mod 2^32 (p = 1 mod 2^32).
    __device__ static __forceinline__ uint32_t to_u32(E y) {
        if (y >= P) y -= P;
        return (uint32_t)y - (y > HALF_P ? 1u : 0u);
    }
};

// ------------------------------------------------------------ two 30-bit primes
constexpr uint32_t P1 = kP1, P2 = kP2;
constexpr uint32_t TWO_P1 = 2 * kP1, TWO_P2 = 2 * kP2;
// -p^-1 mod 2^32 (Montgomery), by Newton iteration at compile time.
constexpr uint32_t neg_inv32(uint32_t p) {
    uint32_t x = p;  // p * p = 1 mod 8
    for (int i = 0; i < 5; ++i) x *= 2u - p * x;
    return 0u - x;
}
constexpr uint32_t PINV1 = neg_inv32(kP1), PINV2 = neg_inv32(kP2);
constexpr uint64_t P12 = (uint64_t)kP1 * kP2;
constexpr uint64_t HALF_P12 = P12 >> 1;
constexpr uint32_t modpow32(uint64_t b, uint64_t e, uint32_t m) {
    uint64_t r = 1;
    b %= m;
    while (e) {
        if (e & 1) r = r * b % m;
        b = b * b % m;
        e >>= 1;
    }
    return (uint32_t)r;
}
constexpr uint32_t CRT_C = modpow32(kP1, kP2 - 2, kP2);                         // p1^-1 mod p2
constexpr uint32_t CRT_CP = (uint32_t)(((uint64_t)CRT_C << 32) / kP2);           // Shoup companion

// Shoup: x * w mod p in [0, 2p) for any x < 2^32, w < p, wp = floor(w 2^32 / p).
__device__ __forceinline__ uint32_t shoup(uint32_t x, uint32_t w, uint32_t wp, uint32_t p) {
    const uint32_t q = __umulhi(x, wp);
    return x * w - q * p;
}

__device__ __forceinline__ uint32_t red2p(uint32_t x, uint32_t twop) { return min(x, x - twop); }

// Montgomery: x * k * 2^-32 mod p in [0, 2p) for any x < 2^32 and k < p
// ((x k + m p) / 2^32 < k + p).
__device__ __forceinline__ uint32_t montmul(uint32_t x, uint32_t k, uint32_t p, uint32_t pinv) {
    const uint64_t t = (uint64_t)x * k;
    const uint32_t m = (uint32_t)t * pinv;
    return (uint32_t)((t + (uint64_t)m * p) >> 32);
}

struct FieldDual {
    using E = uint2;   // (residue mod p1, residue mod p2)
    using Tw = uint4;  // (w1, w2, w1', w2'): twiddles with Shoup companions
    static constexpr int kForm = 1;
    __device__ static __forceinline__ E zero() { return make_uint2(0, 0); }
    // u + p in [p - 2^9, p + 2^9) within [0, 2p): no branch on the sign.
    __device__ static __forceinline__ E from_digit(int32_t u) {
        return make_uint2(P1 + (uint32_t)u, P2 + (uint32_t)u);
    }
    // Harvey: inputs in [0, 4p), outputs in [0, 4p).
    __device__ static __forceinline__ void fwd(E &X, E &Y, const Tw &S) {
        const uint32_t x1 = red2p(X.x, TWO_P1), x2 = red2p(X.y, TWO_P2);
        const uint32_t t1 = shoup(Y.x, S.x, S.z, P1), t2 = shoup(Y.y, S.y, S.w, P2);
        X = make_uint2(x1 + t1, x2 + t2);
        Y = make_uint2(x1 - t1 + TWO_P1, x2 - t2 + TWO_P2);
    }
    // Inputs and outputs in [0, 2p).
    __device__ static __forceinline__ void inv(E &X, E &Y, const Tw &S) {
        const uint32_t u1 = X.x, u2 = X.y, v1 = Y.x, v2 = Y.y;
        X = make_uint2(red2p(u1 + v1, TWO_P1), red2p(u2 + v2, TWO_P2));
        Y = make_uint2(shoup(u1 - v1 + TWO_P1, S.x, S.z, P1), shoup(u2 - v2 + TWO_P2, S.y, S.w, P2));
    }
    // acc in [0, 2p), any x, k in Montgomery form.
    __device__ static __forceinline__ void mac(E &acc, const E &x, const E &k) {
        acc.x = red2p(acc.x + montmul(x.x, k.x, P1, PINV1), TWO_P1);
        acc.y = red2p(acc.y + montmul(x.y, k.y, P2, PINV2), TWO_P2);
    }
    // CRT (Garner) of residues in [0, 2p) to the exact integer in (-p1p2/2, p1p2/2), mod 2^32.
    __device__ static __forceinline__ uint32_t to_u32(E y) {
        const uint32_t x1 = min(y.x, y.x - P1), x2 = min(y.y, y.y - P2);
        uint32_t t = shoup(x2 + TWO_P2 - x1, CRT_C, CRT_CP, P2);
        t = min(t, t - P2);
        const uint64_t X = (uint64_t)t * P1 + x1;
        return (uint32_t)X - (X > HALF_P12 ? (uint32_t)P12 : 0u);
    }
};

// Layouts of an NTT-domain key polynomial (transform order), chosen so that
// a thread holding EPT = 8 consecutive elements reads them with 16-byte loads
// that are contiguous across the warp: coalesced in global memory and free of
// bank conflicts in shared memory.
//  * 8-byte elements (MK_FORM_NTT): the 16-byte unit u (elements 2u, 2u + 1)
//    is stored at unit position (u % 4) * (N / 8) + u / 4, so unit q of
//    thread t's four is at q * (N / 8) + t.
//  * two residues (MK_FORM_NTT2): two planes of N words (residues mod p1,
//    then mod p2); in each plane the 16-byte unit u (elements 4u .. 4u + 3)
//    is stored at (u % 2) * (N / 8) + u / 2, so unit r of thread t's two is
//    at r * (N / 8) + t.  A kernel that works on one prime reads one plane.
template <int LOGN>
__host__ __device__ __forceinline__ int key_unit_pos(int u) {
    return (u & 3) * ((1 << LOGN) / 8) + (u >> 2);
}
template <int LOGN>
__host__ __device__ __forceinline__ int plane_unit_pos(int u) {
    return (u & 1) * ((1 << LOGN) / 8) + (u >> 1);
}

template <bool SMEM>
__device__ __forceinline__ uint4 load16(const uint4 *p) {
    if constexpr (SMEM) return *p;
    else return __ldg(p);
}

// The EPT elements of thread tid (transform positions EPT*tid ..) of one key
// polynomial; global memory through the read-only cache, or shared memory.
template <int LOGN, int EPT, bool SMEM = false, class E>
__device__ __forceinline__ void load_ept(const E *__restrict__ poly, int tid, E (&v)[EPT]) {
    static_assert(sizeof(E) == 8 && EPT % 4 == 0, "8-byte elements, a multiple of four");
    const uint4 *s4 = reinterpret_cast<const uint4 *>(poly);
    if constexpr (std::is_same<E, uint2>::value) {
        constexpr int PU = (1 << LOGN) / 4;  // 16-byte units per plane
#pragma unroll
        for (int r = 0; r < EPT / 4; ++r) {
            const int pos = plane_unit_pos<LOGN>(tid * (EPT / 4) + r);
            const uint4 a = load16<SMEM>(s4 + pos), b = load16<SMEM>(s4 + PU + pos);
            v[4 * r] = make_uint2(a.x, b.x);
            v[4 * r + 1] = make_uint2(a.y, b.y);
            v[4 * r + 2] = make_uint2(a.z, b.z);
            v[4 * r + 3] = make_uint2(a.w, b.w);
        }
    } else {
#pragma unroll
        for (int q = 0; q < EPT / 2; ++q) {
            const uint4 t = load16<SMEM>(s4 + key_unit_pos<LOGN>(tid * (EPT / 2) + q));
            reinterpret_cast<uint4 *>(v)[q] = t;
        }
    }
}

// Named barrier of the bar_id-th thread group of nthreads (bar_id 0: the CTA).
__device__ __forceinline__ void group_sync(int bar_id, int nthreads) {
    if (bar_id == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;\n" ::"r"(bar_id), "r"(nthreads) : "memory");
}

// ------------------------------------------------------------ negacyclic NTT
// Thread `tid` (of T = N/EPT) holds EPT = 2^SB elements per polynomial (8 or
// 4).  A pass processes up to SB consecutive butterfly stages in registers;
// its EPT elements are the indices whose bits [LO, LO+SB) vary:
// j = base(tid, LO) | c << LO with base = tid[0,LO) | tid[LO,..) << (LO+SB).
// Forward (Cooley-Tukey, twist folded into psi^bitrev): input natural order in
// layout LO = logN-SB (coefficient tid + T*c), output bit-reversed order in
// layout LO = 0 (index EPT*tid + c).  Inverse (Gentleman-Sande) goes back, and
// omits the 1/N factor (the keys carry it).  Between passes the elements move
// through padded shared memory, two pad elements after every 16: measured
// on GB300 (ncu, a 608-gate launch of the two-prime form), the exchanges'
// bank conflicts fell from 1.40 G wavefronts with one pad element per 16 to
// 0.01 G, and the launch from 64.5 to 61.4 ms.  The padding adds a fixed
// offset per index bit, which the compile-time exchange relies on.
__host__ __device__ constexpr int pidx(int j) { return j + 2 * (j >> 4); }
// Length of one padded polynomial of n elements in an exchange buffer.
__host__ __device__ constexpr int padded_len(int n) { return n + n / 8; }

// Twiddle tables are stored with one pad entry every 4, so the stride-2 and
// stride-4 twiddle reads of the late stages hit distinct banks.
__device__ __forceinline__ int twp(int t) { return t + (t >> 2); }

template <int SB = 3>
__device__ __forceinline__ int jbase(int tid, int LO) {
    return (tid & ((1 << LO) - 1)) | ((tid >> LO) << (LO + SB));
}

constexpr int log2_ept(int ept) { return ept == 8 ? 3 : (ept == 4 ? 2 : 1); }

// TWG: twiddles read from global memory through the read-only cache
// (unpadded table) instead of a per-CTA shared-memory copy.
template <class F, int LOGN, bool TWG, int EPT = 8>
struct Ntt {
    using E = typename F::E;
    using Tw = typename F::Tw;
    __device__ static __forceinline__ Tw twiddle(const Tw *tw, int t) {
        if constexpr (TWG) return __ldg(tw + t);
        else return tw[twp(t)];
    }
    static constexpr int N = 1 << LOGN;
    static constexpr int SB = log2_ept(EPT);
    static_assert(EPT == 8 || EPT == 4, "8 or 4 elements per thread");
    static constexpr int T = N / EPT;
    static constexpr int PN = padded_len(N);  // padded polynomial stride in xbuf

    // Forward stage at bit b (distance 2^b) inside a pass with element bits
    // [LO, LO+SB): element pairs (c, c + D), D = 2^(b - LO).  The pair's
    // twiddle index m + ((jb | c << LO) >> (b + 1)) splits into a per-stage
    // base m + (jb >> (b + 1)) plus c / (2 D) (jb has no bits in [LO, LO+SB)),
    // so a stage needs only EPT / (2 D) distinct twiddles.
    template <int NP, int D>
    __device__ static __forceinline__ void fwd_stage(E (&x)[NP][EPT], int jb, int LO, int b, const Tw *tw) {
        constexpr int NT = EPT / (2 * D), SH = (D == 4 ? 3 : (D == 2 ? 2 : 1));  // 2 D = 2^SH
        const int base = (1 << (LOGN - 1 - b)) + (jb >> (b + 1));
        Tw S[NT];
#pragma unroll
        for (int q = 0; q < NT; ++q) S[q] = twiddle(tw, base + q);
#pragma unroll
        for (int c = 0; c < EPT; ++c) {
            if (c & D) continue;
#pragma unroll
            for (int p = 0; p < NP; ++p) F::fwd(x[p][c], x[p][c + D], S[c >> SH]);
        }
    }

    template <int NP, int D>
    __device__ static __forceinline__ void inv_stage(E (&x)[NP][EPT], int jb, int LO, int b, const Tw *tw) {
        constexpr int NT = EPT / (2 * D), SH = (D == 4 ? 3 : (D == 2 ? 2 : 1));  // 2 D = 2^SH
        const int base = (1 << (LOGN - 1 - b)) + (jb >> (b + 1));
        Tw S[NT];
#pragma unroll
        for (int q = 0; q < NT; ++q) S[q] = twiddle(tw, base + q);
#pragma unroll
        for (int c = 0; c < EPT; ++c) {
            if (c & D) continue;
#pragma unroll
            for (int p = 0; p < NP; ++p) F::inv(x[p][c], x[p][c + D], S[c >> SH]);
        }
    }

    // bar_id: the named barrier of the T threads that own the polynomials
    // (0: the whole CTA is those threads).
    template <int NP>
    __device__ static __forceinline__ void exchange(E (&x)[NP][EPT], int tid, E *buf, int LOf, int LOt, int bar_id) {
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

    // The same exchange with both layouts known at compile time.  jbase's
    // bits and c << LO are disjoint, so their sum carries nothing and
    // pidx(jbase | c << LO) = pidx(jbase) + pidx(c << LO): one address per
    // thread and layout, every element at an immediate offset from it.
    template <int NP, int LOF, int LOT>
    __device__ static __forceinline__ void exchange_ct(E (&x)[NP][EPT], int tid, E *buf, int bar_id) {
        const int bf = jbase<SB>(tid, LOF);
        E *wb = buf + pidx(bf);
#pragma unroll
        for (int p = 0; p < NP; ++p)
#pragma unroll
            for (int c = 0; c < EPT; ++c) wb[p * PN + pidx(c << LOF)] = x[p][c];
        group_sync(bar_id, T);
        const int bt = jbase<SB>(tid, LOT);
        const E *rb = buf + pidx(bt);
#pragma unroll
        for (int p = 0; p < NP; ++p)
#pragma unroll
            for (int c = 0; c < EPT; ++c) x[p][c] = rb[p * PN + pidx(c << LOT)];
        group_sync(bar_id, T);
    }

    // Layout (LO) of pass q of the forward / inverse transform, as the pass
    // loops below compute it.
    __host__ __device__ static constexpr int pass_lo(bool fwd, int q) {
        return fwd ? ((LOGN - 1 - SB * q) >= SB - 1 ? (LOGN - 1 - SB * q) - (SB - 1) : 0)
                   : ((SB * q < LOGN - SB) ? SB * q : LOGN - SB);
    }
    static constexpr int NPASS = (LOGN + SB - 1) / SB;

    // Exchange before pass q (1 <= q < NPASS) with compile-time layouts for
    // the passes of a transform of up to five passes; runtime layouts beyond.
    template <int NP, bool FWD>
    __device__ static __forceinline__ void exchange_pass(E (&x)[NP][EPT], int tid, E *buf, int q, int LOf, int LOt,
                                                         int bar_id) {
        constexpr int L0 = pass_lo(FWD, 0), L1 = pass_lo(FWD, 1), L2 = pass_lo(FWD, 2), L3 = pass_lo(FWD, 3),
                      L4 = pass_lo(FWD, 4);
        if constexpr (L0 != L1) {
            if (q == 1) {
                exchange_ct<NP, L0, L1>(x, tid, buf, bar_id);
                return;
            }
        }
        if constexpr (NPASS > 2 && L1 != L2) {
            if (q == 2) {
                exchange_ct<NP, L1, L2>(x, tid, buf, bar_id);
                return;
            }
        }
        if constexpr (NPASS > 3 && L2 != L3) {
            if (q == 3) {
                exchange_ct<NP, L2, L3>(x, tid, buf, bar_id);
                return;
            }
        }
        if constexpr (NPASS > 4 && L3 != L4) {
            if (q == 4) {
                exchange_ct<NP, L3, L4>(x, tid, buf, bar_id);
                return;
            }
        }
        exchange<NP>(x, tid, buf, LOf, LOt, bar_id);
    }

    // natural (layout logN-SB) -> bit-reversed (layout 0)
    template <int NP>
    __device__ static __forceinline__ void forward(E (&x)[NP][EPT], int tid, const Tw *tw, E *buf, int bar_id = 0) {
        int prev = LOGN - SB;
        int q = 0;
#pragma unroll 1
        for (int hi = LOGN - 1; hi >= 0; hi -= SB, ++q) {
            const int LO = hi >= SB - 1 ? hi - (SB - 1) : 0;
            if (LO != prev) exchange_pass<NP, true>(x, tid, buf, q, prev, LO, bar_id);
            const int jb = jbase<SB>(tid, LO);
            if constexpr (SB == 3) {
                if (hi - LO == 2) fwd_stage<NP, 4>(x, jb, LO, LO + 2, tw);
            }
            if (hi - LO >= 1) fwd_stage<NP, 2>(x, jb, LO, LO + 1, tw);
            fwd_stage<NP, 1>(x, jb, LO, LO, tw);
            prev = LO;
        }
    }

    // bit-reversed (layout 0) -> natural (layout logN-SB), without 1/N
    template <int NP>
    __device__ static __forceinline__ void inverse(E (&x)[NP][EPT], int tid, const Tw *tw, E *buf, int bar_id = 0) {
        int prev = 0;
        int q = 0;
#pragma unroll 1
        for (int lo = 0; lo < LOGN; lo += SB, ++q) {
            const int hi = (lo + SB - 1 < LOGN - 1) ? lo + SB - 1 : LOGN - 1;
            const int LO = (lo < LOGN - SB) ? lo : LOGN - SB;
            if (LO != prev) exchange_pass<NP, false>(x, tid, buf, q, prev, LO, bar_id);
            const int jb = jbase<SB>(tid, LO);
            if (lo == LO) inv_stage<NP, 1>(x, jb, LO, LO, tw);
            if (lo <= LO + 1 && hi >= LO + 1) inv_stage<NP, 2>(x, jb, LO, LO + 1, tw);
            if constexpr (SB == 3) {
                if (hi == LO + 2) inv_stage<NP, 4>(x, jb, LO, LO + 2, tw);
            }
            prev = LO;
        }
    }
};

// ------------------------------------------------------------ gadget g^-1
// Signed base-2^bg digits with round-to-nearest at the last digit (d = 3).
struct Gadget {
    uint32_t offset;
    uint32_t bg_bit;
    uint32_t mask, half;
    __device__ __forceinline__ int32_t digit(uint32_t x, int l) const {
        const uint32_t xp = x + offset;
        return (int32_t)((xp >> (32 - bg_bit * (l + 1))) & mask) - (int32_t)half;
    }
};

__device__ __forceinline__ Gadget make_gadget(uint32_t bg_bit) {
    Gadget g;
    g.bg_bit = bg_bit;
    g.mask = (1u << bg_bit) - 1;
    g.half = 1u << (bg_bit - 1);
    uint32_t off = 0;
    for (uint32_t l = 1; l <= 3; ++l) off += g.half << (32 - bg_bit * l);
    if (3 * bg_bit < 32) off += 1u << (32 - 3 * bg_bit - 1);
    g.offset = off;
    return g;
}

// ------------------------------------------------------------ blind rotation
struct SmemLayout {
    size_t twf, twi, xbuf, acc, abar, total;
};

template <class F, int LOGN, int NPF, bool TWG>
__host__ __device__ inline SmemLayout smem_layout(uint32_t k, uint32_t n) {
    constexpr int N = 1 << LOGN;
    using E = typename F::E;
    using Tw = typename F::Tw;
    constexpr size_t tw_bytes = TWG ? 0 : sizeof(Tw) * (N + N / 4);
    SmemLayout L;
    L.twf = 0;
    L.twi = L.twf + tw_bytes;
    L.xbuf = L.twi + tw_bytes;
    // exchange buffer for NPF forward or 2 inverse transforms at once
    L.acc = L.xbuf + sizeof(E) * (NPF > 2 ? NPF : 2) * padded_len(N);
    L.abar = L.acc + sizeof(uint32_t) * (k + 1) * N;
    L.total = L.abar + ((sizeof(uint16_t) * (k * n + 1) + 15) & ~size_t(15));
    return L;
}

// A += x * key over the EPT elements of thread tid (transform layout 0) of
// the key polynomial `key` (unit-interleaved, in global or shared memory).
template <class F, int LOGN, int EPT, bool SMEM = false>
__device__ __forceinline__ void mac_ept(typename F::E (&A)[EPT], const typename F::E (&x)[EPT],
                                        const typename F::E *__restrict__ key, int tid) {
    typename F::E kv[EPT];
    load_ept<LOGN, EPT, SMEM>(key, tid, kv);
#pragma unroll
    for (int c = 0; c < EPT; ++c) F::mac(A[c], x[c], kv[c]);
}

template <class F, int LOGN>
__device__ __forceinline__ void mac8(typename F::E (&A)[8], const typename F::E (&x)[8],
                                     const typename F::E *__restrict__ key, int tid) {
    mac_ept<F, LOGN, 8>(A, x, key, tid);
}

// Montgomery reduction of t < 2^32 p: t * 2^-32 mod p in [0, 2p).
__device__ __forceinline__ uint32_t redc(uint64_t t, uint32_t p, uint32_t pinv) {
    const uint32_t m = (uint32_t)t * pinv;
    return (uint32_t)((t + (uint64_t)m * p) >> 32);
}

// Two-prime form, three digit polynomials at once (EPT = 8):
//   A += x[0] * key[0] + x[1] * key[1] + x[2] * key[2]
// with key[l] = key + l N.  The three products of an element are summed in
// 64 bits and reduced once: each is below 4p * p (x from the forward
// transform, below 4p; key words below p), so the sum is below 12 p^2 <
// 2^32 p for p < 2^28 and redc returns it in [0, 2p).  One multiply-add per
// product instead of a Montgomery reduction per product.
template <int LOGN, bool SMEM = false>
__device__ __forceinline__ void mac3_dual(uint2 (&A)[8], const uint2 (&x)[3][8], const uint2 *__restrict__ key,
                                          int tid) {
    constexpr int N = 1 << LOGN, PU = N / 4;  // 16-byte units per plane
    const uint4 *k4 = reinterpret_cast<const uint4 *>(key);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int pos = plane_unit_pos<LOGN>(2 * tid + r);
#pragma unroll
        for (int pl = 0; pl < 2; ++pl) {
            const uint32_t p = pl ? P2 : P1, pinv = pl ? PINV2 : PINV1, twop = pl ? TWO_P2 : TWO_P1;
            uint4 kw[3];
#pragma unroll
            for (int l = 0; l < 3; ++l) kw[l] = load16<SMEM>(k4 + (size_t)l * 2 * PU + pl * PU + pos);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = 4 * r + e;
                uint64_t t = 0;
#pragma unroll
                for (int l = 0; l < 3; ++l) {
                    const uint32_t kv = e == 0 ? kw[l].x : (e == 1 ? kw[l].y : (e == 2 ? kw[l].z : kw[l].w));
                    const uint32_t xv = pl ? x[l][c].y : x[l][c].x;
                    t += (uint64_t)xv * kv;
                }
                uint32_t &a = pl ? A[c].y : A[c].x;
                a = red2p(a + redc(t, p, pinv), twop);
            }
        }
    }
}

// A += sum_l x[l] * key[l] over the NPF digit polynomials of a forward pass.
template <class F, int LOGN, int EPT, int NPF, bool SMEM = false>
__device__ __forceinline__ void mac_npf(typename F::E (&A)[EPT], const typename F::E (&x)[NPF][EPT],
                                        const typename F::E *__restrict__ key, int tid) {
    if constexpr (NPF == 3 && EPT == 8 && std::is_same<typename F::E, uint2>::value) {
        mac3_dual<LOGN, SMEM>(A, x, key, tid);
    } else {
#pragma unroll
        for (int p = 0; p < NPF; ++p) mac_ept<F, LOGN, EPT, SMEM>(A, x[p], key + (size_t)p * (1 << LOGN), tid);
    }
}

// One CMux step for party i (1..k) at rotation e:
//   ACC += HP((X^{-e} - 1) ACC, BK_{i,j}).
// Slots q = 0..k take the accumulator polynomials in the order: the k - 1
// others (ascending, i left out), then 0, then i (phase A); slot k + 1 is
// phase B (w = g^-1(v) against f0, f1).  NPF digit polynomials go through
// one forward transform together.  The order lets every inverse transform
// run in a pair (two polynomials per pass, twice the independent work of a
// single): the others' c'_jj two by two, an odd last one with v, and c'_0
// with c'_i.  Four accumulator sets: C0 and CI hold the first and second of
// an others' pair, then c'_0 and c'_i; CJ the odd last other; V.
template <class F, int LOGN, int NPF, bool TWG, int EPT>
__device__ __forceinline__ void cmux_step(const LaunchShape &S, const DeviceKeys &K, const Gadget &G,
                                          const typename F::E *bk, int i, uint32_t e, uint32_t *acc,
                                          typename F::E *xbuf, const typename F::Tw *twf,
                                          const typename F::Tw *twi, int tid) {
    using NT = Ntt<F, LOGN, TWG, EPT>;
    using E = typename F::E;
    constexpr int N = NT::N, T = NT::T;
    const int k = (int)S.k;
    const int nothers = k - 1;
    const int npaired = nothers & ~1;  // others that go through paired inverses
    const E *keyA = static_cast<const E *>(K.keyA);
    E C0[EPT], CI[EPT], CJ[EPT], V[EPT];
    uint32_t vv[EPT];
#pragma unroll
    for (int c = 0; c < EPT; ++c) C0[c] = CI[c] = CJ[c] = V[c] = F::zero();
#pragma unroll 1
    for (int q = 0; q <= k + 1; ++q) {
        // polynomial of slot q (q <= k): the q-th other (i skipped), 0, then i
        const int jj = q < nothers ? (q + 1 < i ? q + 1 : q + 2) : (q == nothers ? 0 : i);
        // accumulator of slot q: 0 = C0, 1 = CI, 2 = CJ
        const int slot = q < npaired ? (q & 1) : (q < nothers ? 2 : (q == nothers ? 0 : 1));
        if (q <= k && slot < 2 && (q == nothers || (q < npaired && (q & 1) == 0))) {
#pragma unroll
            for (int c = 0; c < EPT; ++c) C0[c] = CI[c] = F::zero();  // a fresh pair (or c'_0, c'_i)
        }
#pragma unroll 1
        for (int l0 = 0; l0 < 3; l0 += NPF) {
            E x[NPF][EPT];
            if (q <= k) {
                const uint32_t *ap = acc + jj * N;
#pragma unroll
                for (int c = 0; c < EPT; ++c) {
                    const uint32_t m = tid + T * c;
                    uint32_t r = m + e;
                    if (r >= 2 * N) r -= 2 * N;
                    uint32_t a = ap[r & (N - 1)];
                    if (r >= N) a = 0u - a;
                    const uint32_t D = a - ap[m];
#pragma unroll
                    for (int p = 0; p < NPF; ++p) x[p][c] = F::from_digit(G.digit(D, l0 + p));
                }
            } else {
#pragma unroll
                for (int c = 0; c < EPT; ++c)
#pragma unroll
                    for (int p = 0; p < NPF; ++p) x[p][c] = F::from_digit(G.digit(vv[c], l0 + p));
            }
            NT::template forward<NPF>(x, tid, twf, xbuf);
            if (q <= k) {
                const E *kd = bk + l0 * N;                              // d_l0.. of BK_{i,j}
                const E *ka = keyA + ((size_t)jj * 3 + l0) * N;         // -a_l0.. or pk_jj[l0..]
                if (slot == 0) mac_npf<F, LOGN, EPT, NPF>(C0, x, kd, tid);
                else if (slot == 1) mac_npf<F, LOGN, EPT, NPF>(CI, x, kd, tid);
                else mac_npf<F, LOGN, EPT, NPF>(CJ, x, kd, tid);
                mac_npf<F, LOGN, EPT, NPF>(V, x, ka, tid);
            } else {
                mac_npf<F, LOGN, EPT, NPF>(C0, x, bk + (3 + l0) * N, tid);  // f0_l0..
                mac_npf<F, LOGN, EPT, NPF>(CI, x, bk + (6 + l0) * N, tid);  // f1_l0..
            }
        }
        // Inverse transforms due after this slot (two call sites):
        //   q < npaired, q odd:  the others' pair in C0, CI   -> ACC of both
        //   q == k, odd others:  c'_last (CJ) and v together  -> ACC_last, v in registers
        //   q == k, even others: v alone                      -> v in registers
        //   q == k + 1:          c'_0 and c'_i together       -> ACC_0, ACC_i
        const bool pair_others = q < npaired && (q & 1);
        const bool pair_v = q == k && (nothers & 1);
        const bool pair_last = q == k + 1;
        if (pair_others || pair_v || pair_last) {
            E y[2][EPT];
#pragma unroll
            for (int c = 0; c < EPT; ++c) {
                y[0][c] = pair_v ? CJ[c] : C0[c];
                y[1][c] = pair_v ? V[c] : CI[c];
            }
            NT::template inverse<2>(y, tid, twi, xbuf);
            // destinations: the pair's polynomials (the previous other, this one), (last other, v), (0, i)
            const int d0 = pair_others ? (jj - 1 == i ? jj - 2 : jj - 1) : (pair_v ? (nothers + 1 > i ? nothers + 1 : nothers) : 0);
            uint32_t *p0 = acc + d0 * N;
#pragma unroll
            for (int c = 0; c < EPT; ++c) p0[tid + T * c] += F::to_u32(y[0][c]);
            if (pair_v) {
#pragma unroll
                for (int c = 0; c < EPT; ++c) vv[c] = F::to_u32(y[1][c]);
            } else {
                uint32_t *p1 = acc + (pair_others ? jj : i) * N;
#pragma unroll
                for (int c = 0; c < EPT; ++c) p1[tid + T * c] += F::to_u32(y[1][c]);
            }
        } else if (q == k) {
            E y[1][EPT];
#pragma unroll
            for (int c = 0; c < EPT; ++c) y[0][c] = V[c];
            NT::template inverse<1>(y, tid, twi, xbuf);
#pragma unroll
            for (int c = 0; c < EPT; ++c) vv[c] = F::to_u32(y[0][c]);
        }
    }
}

// k*n CMux steps (i = 1..k, j = 0..n-1 ascending).
template <class F, int LOGN, int NPF, bool TWG, int EPT>
__device__ __forceinline__ void blind_rotate_core(const LaunchShape &S, const DeviceKeys &K, const uint16_t *abar,
                                                  uint32_t *acc, typename F::E *xbuf, const typename F::Tw *twf,
                                                  const typename F::Tw *twi, int64_t max_steps, int tid) {
    constexpr int N = 1 << LOGN;
    using E = typename F::E;
    const int n = (int)S.n, k = (int)S.k;
    const Gadget G = make_gadget(S.bg_bit);
    const E *bk_all = static_cast<const E *>(K.bk);
    int64_t steps = 0;
#pragma unroll 1
    for (int i = 1; i <= k; ++i) {
#pragma unroll 1
        for (int j = 0; j < n; ++j) {
            if (max_steps >= 0 && steps >= max_steps) return;
            ++steps;
            const uint32_t e = abar[(i - 1) * n + j];
            if (e == 0) continue;  // X^0 - 1 = 0: every digit is 0, HP adds nothing
            const E *bk = bk_all + ((size_t)((i - 1) * n + j) * 9) * N;
            cmux_step<F, LOGN, NPF, TWG, EPT>(S, K, G, bk, i, e, acc, xbuf, twf, twi, tid);
            __syncthreads();
        }
    }
}

template <class F, int LOGN, int EPT>
__device__ __forceinline__ void load_twiddles(const DeviceKeys &K, typename F::Tw *twf, typename F::Tw *twi,
                                              int tid) {
    constexpr int N = 1 << LOGN, T = N / EPT;
    const typename F::Tw *gf = static_cast<const typename F::Tw *>(K.tw_fwd);
    const typename F::Tw *gi = static_cast<const typename F::Tw *>(K.tw_inv);
    for (int x = tid; x < N; x += T) {
        twf[twp(x)] = gf[x];
        twi[twp(x)] = gi[x];
    }
}

template <int LOGN, int EPT>
__device__ __forceinline__ void init_acc(uint32_t *acc, uint32_t k, uint32_t bbar, int tid) {
    constexpr int N = 1 << LOGN, T = N / EPT;
#pragma unroll
    for (int c = 0; c < EPT; ++c) {
        const uint32_t m = tid + T * c;
        uint32_t r = m + bbar;
        if (r >= 2 * N) r -= 2 * N;
        acc[m] = (r >= (uint32_t)N) ? (0u - (1u << 29)) : (1u << 29);
    }
    for (uint32_t x = N + tid; x < (k + 1) * N; x += T) acc[x] = 0;
}

// Linear part + window shift + modulus switch of one gate into abar (shared).
__device__ __forceinline__ void lin_modswitch(const LaunchShape &S, const GateDesc &g, const uint32_t *ct_a,
                                              const uint32_t *ct_b, uint16_t *abar, int tid, int nthreads) {
    const uint32_t W = S.k * S.n + 1;
    const uint32_t sh = 32 - (S.logN + 1);
    const uint32_t *ca = ct_a + (size_t)g.ia * W;
    const uint32_t *cb = ct_b + (size_t)g.ib * W;
    for (uint32_t x = tid; x < W; x += nthreads) {
        uint32_t v = (uint32_t)g.s1 * ca[x] + (uint32_t)g.s2 * cb[x];
        if (x == W - 1) v += g.cst - (1u << 30);  // (0, cst) and the -1/4 window shift
        abar[x] = (uint16_t)((v + (1u << (sh - 1))) >> sh);
    }
}

template <int LOGN, int T>
__device__ __forceinline__ void sample_extract(const LaunchShape &S, const uint32_t *acc, uint32_t *dst, int tid) {
    constexpr int N = 1 << LOGN;
    for (uint32_t i = 1; i <= S.k; ++i) {
        const uint32_t *ci = acc + i * N;
        uint32_t *ai = dst + (i - 1) * N;
        for (int m = tid; m < N; m += T) ai[m] = (m == 0) ? ci[0] : 0u - ci[N - m];
    }
    if (tid == 0) dst[S.k * N] = acc[0] + (1u << 29);  // +1/8
}

// One kernel for the whole gate and for the stage entry points:
//   abar_in == nullptr: linear part + window shift + modulus switch from desc;
//   otherwise the mod-switched words are read from abar_in.
//   acc_out == nullptr: SampleExtract + 1/8 into ext; otherwise the raw ACC.
template <class F, int LOGN, int NPF, int MINB, bool TWG, int EPT>
__global__ void __launch_bounds__((1 << LOGN) / EPT, MINB)
bootstrap_ntt_kernel(LaunchShape S, DeviceKeys K, const GateDesc *__restrict__ desc,
                     const uint32_t *__restrict__ ct_a, const uint32_t *__restrict__ ct_b,
                     const uint32_t *__restrict__ abar_in, int64_t max_steps,
                     uint32_t *__restrict__ ext, uint32_t *__restrict__ acc_out) {
    constexpr int N = 1 << LOGN, T = N / EPT;
    using E = typename F::E;
    using Tw = typename F::Tw;
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x;
    const SmemLayout L = smem_layout<F, LOGN, NPF, TWG>(S.k, S.n);
    const Tw *twf, *twi;
    if constexpr (TWG) {
        twf = static_cast<const Tw *>(K.tw_fwd);
        twi = static_cast<const Tw *>(K.tw_inv);
    } else {
        twf = reinterpret_cast<Tw *>(smem + L.twf);
        twi = reinterpret_cast<Tw *>(smem + L.twi);
        load_twiddles<F, LOGN, EPT>(K, reinterpret_cast<Tw *>(smem + L.twf), reinterpret_cast<Tw *>(smem + L.twi), tid);
    }
    E *xbuf = reinterpret_cast<E *>(smem + L.xbuf);
    uint32_t *acc = reinterpret_cast<uint32_t *>(smem + L.acc);
    uint16_t *abar = reinterpret_cast<uint16_t *>(smem + L.abar);
    if (abar_in) {
        const uint32_t W = S.k * S.n + 1;
        for (uint32_t x = tid; x < W; x += T) abar[x] = (uint16_t)abar_in[(size_t)blockIdx.x * W + x];
    } else {
        lin_modswitch(S, desc[blockIdx.x], ct_a, ct_b, abar, tid, T);
    }
    __syncthreads();
    init_acc<LOGN, EPT>(acc, S.k, abar[S.k * S.n], tid);
    __syncthreads();
    blind_rotate_core<F, LOGN, NPF, TWG, EPT>(S, K, abar, acc, xbuf, twf, twi, max_steps, tid);
    __syncthreads();
    if (acc_out) {
        uint32_t *dst = acc_out + (size_t)blockIdx.x * (S.k + 1) * N;
        for (uint32_t x = tid; x < (S.k + 1) * N; x += T) dst[x] = acc[x];
    } else {
        sample_extract<LOGN, T>(S, acc, ext + (size_t)blockIdx.x * (S.k * N + 1), tid);
    }
}

template <class F, int LOGN, int NPF, int MINB, bool TWG, int EPT>
cudaError_t launch_bootstrap(const LaunchShape &S, const DeviceKeys &K, const GateDesc *desc,
                             const uint32_t *ct_a, const uint32_t *ct_b, const uint32_t *abar_in,
                             int64_t max_steps, uint32_t *ext, uint32_t *acc_out, uint32_t count,
                             cudaStream_t st) {
    const SmemLayout L = smem_layout<F, LOGN, NPF, TWG>(S.k, S.n);
    auto kern = bootstrap_ntt_kernel<F, LOGN, NPF, MINB, TWG, EPT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return e;
    kern<<<count, (1 << LOGN) / EPT, L.total, st>>>(S, K, desc, ct_a, ct_b, abar_in, max_steps, ext, acc_out);
    return cudaGetLastError();
}

}  // namespace br
}  // namespace mk
