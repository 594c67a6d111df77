// mk_bootstrap_fft.cuh -- blind rotation with the FP64 FFT product form
// (MK_FORM_FFT), the approximate form.
//
// A negacyclic product of two real polynomials of N coefficients is computed
// in C[X]/(X^M - i), M = N/2: the real ring R[X]/(X^N + 1) embeds there by
// folding, f_j = c_j + i c_{j+M} (X^M = i).  Substituting X = theta Y with
// theta^M = -i turns X^M - i into -i (Y^M + 1), so after the twist
// z_j = f_j theta^j the product is a negacyclic convolution of size M over C,
// computed with the same Cooley-Tukey / Gentleman-Sande passes as the NTT
// forms (FieldCplx: psi = exp(i pi / M) in bit-reversed powers).  The inverse
// transform, untwist by theta^-j and 1/M are folded into the keys and into
// the final rounding: keys are stored already transformed and multiplied by
// 1/M, and each output is rounded to the nearest integer (exact when the FP64
// error stays below 1/2; it is not guaranteed, which is why this form is
// compared against a tolerance instead of bit for bit).
//
// One CTA of M/8 = 64 threads per gate; thread t holds the complex points
// j = t + 64 c (c < 8), i.e. the coefficients j and j + M of every polynomial.
#pragma once
#include "mk_bootstrap.cuh"

namespace mk {
namespace br {

struct FieldCplx {
    using E = double2;
    using Tw = double2;
    __device__ static __forceinline__ E zero() { return make_double2(0.0, 0.0); }
    __device__ static __forceinline__ E cmul(const E &a, const E &b) {
        return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
    }
    __device__ static __forceinline__ void fwd(E &X, E &Y, const Tw &S) {
        const E V = cmul(Y, S);
        const E U = X;
        X = make_double2(U.x + V.x, U.y + V.y);
        Y = make_double2(U.x - V.x, U.y - V.y);
    }
    __device__ static __forceinline__ void inv(E &X, E &Y, const Tw &S) {
        const E U = X, V = Y;
        X = make_double2(U.x + V.x, U.y + V.y);
        Y = cmul(make_double2(U.x - V.x, U.y - V.y), S);
    }
    __device__ static __forceinline__ void mac(E &acc, const E &x, const E &k) {
        acc.x = fma(x.x, k.x, fma(-x.y, k.y, acc.x));
        acc.y = fma(x.x, k.y, fma(x.y, k.x, acc.y));
    }
    // nearest integer of a real value, mod 2^32
    __device__ static __forceinline__ uint32_t round_u32(double v) { return (uint32_t)(unsigned long long)__double2ll_rn(v); }
};

template <class T>
__device__ __forceinline__ void load8c(const T *__restrict__ src, T (&v)[8]) {
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __ldg(src + q);
}

template <int LOGM>
struct FftGate {
    using NT = Ntt<FieldCplx, LOGM, false>;
    using E = double2;
    static constexpr int M = 1 << LOGM, N = 2 * M, T = M / 8;

    // MAC of one transformed digit polynomial against one key polynomial
    // (keys laid out so that thread t reads its 8 points contiguously).
    __device__ static __forceinline__ void mac8(E (&A)[8], const E (&x)[8], const E *key, int tid) {
        E kv[8];
        load8c(key + tid * 8, kv);
#pragma unroll
        for (int c = 0; c < 8; ++c) FieldCplx::mac(A[c], x[c], kv[c]);
    }

    // Real digit pair (coefficients m, m + M) -> twisted complex point.
    __device__ static __forceinline__ E fold(int32_t lo, int32_t hi, const E &th) {
        return FieldCplx::cmul(make_double2((double)lo, (double)hi), th);
    }

    // One CMux step (same slot structure as the NTT forms' cmux_step).
    __device__ static void cmux_step(const LaunchShape &S, const DeviceKeys &K, const Gadget &G, const E *bk, int i,
                                     uint32_t e, uint32_t *acc, E *xbuf, const E *twf, const E *twi,
                                     const E *theta, int tid) {
        const int k = (int)S.k;
        const E *keyA = static_cast<const E *>(K.keyA);
        E C0[8], CI[8], CJ[8], V[8];
        uint32_t vv[16];
#pragma unroll
        for (int c = 0; c < 8; ++c) C0[c] = CI[c] = CJ[c] = V[c] = FieldCplx::zero();
        E th[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) th[c] = theta[tid + T * c];
#pragma unroll 1
        for (int q = 0; q <= k + 1; ++q) {
            const int jj = (q == 0) ? 0 : (q == 1 ? i : (q - 1 < i ? q - 1 : q));
            if (q >= 2 && q <= k) {
#pragma unroll
                for (int c = 0; c < 8; ++c) CJ[c] = FieldCplx::zero();
            }
#pragma unroll 1
            for (int l = 0; l < 3; ++l) {
                E x[1][8];
                if (q <= k) {
                    const uint32_t *ap = acc + jj * N;
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        int32_t dg[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const uint32_t m = tid + T * c + h * M;
                            uint32_t r = m + e;
                            if (r >= 2 * N) r -= 2 * N;
                            uint32_t a = ap[r & (N - 1)];
                            if (r >= (uint32_t)N) a = 0u - a;
                            dg[h] = G.digit(a - ap[m], l);
                        }
                        x[0][c] = fold(dg[0], dg[1], th[c]);
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 8; ++c) x[0][c] = fold(G.digit(vv[c], l), G.digit(vv[8 + c], l), th[c]);
                }
                NT::template forward<1>(x, tid, twf, xbuf);
                if (q <= k) {
                    const E *kd = bk + l * M;
                    const E *ka = keyA + ((size_t)jj * 3 + l) * M;
                    if (q == 0) mac8(C0, x[0], kd, tid);
                    else if (q == 1) mac8(CI, x[0], kd, tid);
                    else mac8(CJ, x[0], kd, tid);
                    mac8(V, x[0], ka, tid);
                } else {
                    mac8(C0, x[0], bk + (3 + l) * M, tid);
                    mac8(CI, x[0], bk + (6 + l) * M, tid);
                }
            }
            const int first = (q >= 2 && q <= k) ? 0 : (q == k ? 1 : (q == k + 1 ? 2 : 4));
            const int last = (q == k) ? 1 : (q == k + 1 ? 3 : (q >= 2 ? 0 : -1));
#pragma unroll 1
            for (int kind = first; kind <= last; ++kind) {
                E y[1][8];
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    y[0][c] = kind == 0 ? CJ[c] : (kind == 1 ? V[c] : (kind == 2 ? C0[c] : CI[c]));
                NT::template inverse<1>(y, tid, twi, xbuf);
                // untwist (theta^-j = conj(theta^j)); the 1/M factor is in the keys
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const E u = FieldCplx::cmul(y[0][c], make_double2(th[c].x, -th[c].y));
                    const uint32_t lo = FieldCplx::round_u32(u.x), hi = FieldCplx::round_u32(u.y);
                    if (kind == 1) {
                        vv[c] = lo;
                        vv[8 + c] = hi;
                    } else {
                        uint32_t *dst = acc + (kind == 0 ? jj : (kind == 2 ? 0 : i)) * N;
                        dst[tid + T * c] += lo;
                        dst[tid + T * c + M] += hi;
                    }
                }
            }
        }
    }
};

struct FftSmem {
    size_t twf, twi, theta, xbuf, acc, abar, total;
};

template <int LOGM>
__host__ __device__ inline FftSmem fft_smem_layout(uint32_t k, uint32_t n) {
    constexpr int M = 1 << LOGM;
    FftSmem L;
    L.twf = 0;
    L.twi = L.twf + sizeof(double2) * (M + M / 4);
    L.theta = L.twi + sizeof(double2) * (M + M / 4);
    L.xbuf = L.theta + sizeof(double2) * M;
    L.acc = L.xbuf + sizeof(double2) * padded_len(M);
    L.abar = L.acc + sizeof(uint32_t) * (k + 1) * 2 * M;
    L.total = L.abar + ((sizeof(uint16_t) * (k * n + 1) + 15) & ~size_t(15));
    return L;
}

// Same interface as bootstrap_ntt_kernel.  K.tw_fwd holds [twf M | twi M | theta M] (double2).
template <int LOGM>
__global__ void __launch_bounds__((1 << LOGM) / 8)
bootstrap_fft_kernel(LaunchShape S, DeviceKeys K, const GateDesc *__restrict__ desc, const uint32_t *__restrict__ ct_a,
                     const uint32_t *__restrict__ ct_b, const uint32_t *__restrict__ abar_in, int64_t max_steps,
                     uint32_t *__restrict__ ext, uint32_t *__restrict__ acc_out) {
    using FG = FftGate<LOGM>;
    using E = double2;
    constexpr int M = FG::M, N = FG::N, T = FG::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x;
    const FftSmem L = fft_smem_layout<LOGM>(S.k, S.n);
    E *twf = reinterpret_cast<E *>(smem + L.twf);
    E *twi = reinterpret_cast<E *>(smem + L.twi);
    E *theta = reinterpret_cast<E *>(smem + L.theta);
    E *xbuf = reinterpret_cast<E *>(smem + L.xbuf);
    uint32_t *acc = reinterpret_cast<uint32_t *>(smem + L.acc);
    uint16_t *abar = reinterpret_cast<uint16_t *>(smem + L.abar);
    const E *gt = static_cast<const E *>(K.tw_fwd);
    for (int x = tid; x < M; x += T) {
        twf[twp(x)] = gt[x];
        twi[twp(x)] = gt[M + x];
        theta[x] = gt[2 * M + x];
    }
    const uint32_t W = S.k * S.n + 1;
    if (abar_in) {
        for (uint32_t x = tid; x < W; x += T) abar[x] = (uint16_t)abar_in[(size_t)blockIdx.x * W + x];
    } else {
        lin_modswitch(S, desc[blockIdx.x], ct_a, ct_b, abar, tid, T);
    }
    __syncthreads();
    {
        const uint32_t bbar = abar[S.k * S.n];
        for (uint32_t m = tid; m < (uint32_t)N; m += T) {
            uint32_t r = m + bbar;
            if (r >= 2 * N) r -= 2 * N;
            acc[m] = (r >= (uint32_t)N) ? (0u - (1u << 29)) : (1u << 29);
        }
        for (uint32_t x = N + tid; x < (S.k + 1) * N; x += T) acc[x] = 0;
    }
    __syncthreads();
    const Gadget G = make_gadget(S.bg_bit);
    const E *bk_all = static_cast<const E *>(K.bk);
    int64_t steps = 0;
    bool stop = false;
#pragma unroll 1
    for (int i = 1; i <= (int)S.k && !stop; ++i) {
#pragma unroll 1
        for (int j = 0; j < (int)S.n; ++j) {
            if (max_steps >= 0 && steps >= max_steps) {
                stop = true;
                break;
            }
            ++steps;
            const uint32_t e = abar[(i - 1) * S.n + j];
            if (e == 0) continue;
            const E *bk = bk_all + ((size_t)((i - 1) * S.n + j) * 9) * M;
            FG::cmux_step(S, K, G, bk, i, e, acc, xbuf, twf, twi, theta, tid);
            __syncthreads();
        }
    }
    __syncthreads();
    if (acc_out) {
        uint32_t *dst = acc_out + (size_t)blockIdx.x * (S.k + 1) * N;
        for (uint32_t x = tid; x < (S.k + 1) * N; x += T) dst[x] = acc[x];
    } else {
        uint32_t *dst = ext + (size_t)blockIdx.x * (S.k * N + 1);
        for (uint32_t i = 1; i <= S.k; ++i) {
            const uint32_t *ci = acc + i * N;
            uint32_t *ai = dst + (i - 1) * N;
            for (int m = tid; m < N; m += T) ai[m] = (m == 0) ? ci[0] : 0u - ci[N - m];
        }
        if (tid == 0) dst[S.k * N] = acc[0] + (1u << 29);
    }
}

template <int LOGM>
cudaError_t launch_bootstrap_fft(const LaunchShape &S, const DeviceKeys &K, const GateDesc *desc, const uint32_t *ct_a,
                                 const uint32_t *ct_b, const uint32_t *abar_in, int64_t max_steps, uint32_t *ext,
                                 uint32_t *acc_out, uint32_t count, cudaStream_t st) {
    const FftSmem L = fft_smem_layout<LOGM>(S.k, S.n);
    auto kern = bootstrap_fft_kernel<LOGM>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return e;
    kern<<<count, (1 << LOGM) / 8, L.total, st>>>(S, K, desc, ct_a, ct_b, abar_in, max_steps, ext, acc_out);
    return cudaGetLastError();
}

}  // namespace br
}  // namespace mk
