// mk_netlist.cuh -- a whole k-bit operator (Alg. 3-6) in one persistent launch.
//
// The level-by-level evaluation launches one blind rotation and one key
// switch per netlist level, so every level waits for the slowest gate of the
// level before the next starts, and a level of a few gates times the pairs
// fills one or two waves of CTAs, the second mostly empty.  Here the gates of
// all levels and pairs are work items in the plan's order (level, then gate,
// then pair: topological), taken by CTAs from a global counter.  A CTA waits
// until its gate's two input wires are ready, then runs the gate end to end:
// linear part and modulus switch (Sec. 4.1, Eq. 6-11), the k*n CMux steps of
// GB (Sec. 3.2), SampleExtract into shared memory, and the key switch of that
// one gate (MKKeySwitch) into the output wire's row, and then marks the row
// ready.  A gate of level L + 1 starts as soon as its own inputs exist.
//
// No deadlock: an item waits only for items of lower index (its inputs come
// from lower levels), which running CTAs took earlier, and the unfinished item
// of lowest index has no unfinished input.  Readiness is one word per wire
// row holding the epoch of the call that wrote it (rows of the inputs and
// constants count as ready); the producer's row stores are ordered before its
// flag by a fence and a CTA barrier, and the consumer reads the row through L2
// after an acquire load of the flag.  An item deep in a narrow netlist may
// wait for many gate times, so a wait is bounded by progress, not by its own
// length: it gives up when no item of the launch has finished for S.wait_ns
// of global time.  Then the CTA sets the launch's abort word and the
// context's status word, every CTA stops taking items, and mk_sync reports
// MK_ETIMEOUT.
#pragma once
#include "mk_bootstrap.cuh"

namespace mk {
namespace br {

__device__ __forceinline__ uint32_t nl_load_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void nl_store_release(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint64_t nl_globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// Thread 0: wait until pool row `row` is ready; false if no item finished
// for wait_ns or the launch is aborting.
__device__ inline bool nl_wait_row(const NetlistArgs &A, uint32_t row, uint64_t wait_ns, uint32_t *status) {
    if (row < A.input_rows) return true;
    if (nl_load_acquire(A.ready + row) == A.epoch) return true;
    uint64_t t0 = nl_globaltimer();
    uint32_t seen = *(volatile uint32_t *)A.done;
    for (uint32_t it = 0; it < (1u << 30); ++it) {
        __nanosleep(256);
        if (nl_load_acquire(A.ready + row) == A.epoch) return true;
        if (*(volatile uint32_t *)A.abort) return false;
        const uint32_t d = *(volatile uint32_t *)A.done;
        const uint64_t now = nl_globaltimer();
        if (d != seen) {  // some gate finished: the launch is making progress
            seen = d;
            t0 = now;
        } else if (now - t0 > wait_ns) {
            break;
        }
    }
    atomicExch(A.abort, 1u);
    atomicOr(status, kStatusNetlist);
    return false;
}

// Linear part + window shift + modulus switch of one gate, reading its input
// rows through L2 (rows written during this launch).
__device__ __forceinline__ void nl_lin_modswitch(const LaunchShape &S, const GateDesc &g, const uint32_t *pool,
                                                 uint16_t *abar, int tid, int nthreads) {
    const uint32_t W = S.k * S.n + 1;
    const uint32_t sh = 32 - (S.logN + 1);
    const uint32_t *ca = pool + (size_t)g.ia * W;
    const uint32_t *cb = pool + (size_t)g.ib * W;
    for (uint32_t x = tid; x < W; x += nthreads) {
        uint32_t v = (uint32_t)g.s1 * __ldcg(ca + x) + (uint32_t)g.s2 * __ldcg(cb + x);
        if (x == W - 1) v += g.cst - (1u << 30);  // (0, cst) and the -1/4 window shift
        abar[x] = (uint16_t)((v + (1u << (sh - 1))) >> sh);
    }
}

// MKKeySwitch of one extracted sample (shared memory, k N + 1 words) into a
// row of k n + 1 words: per party i, coefficient j, digit l of a_{i,j}
// rounded to ks_bit t bits, add column x of KS_i[j][l][delta - 1] for
// delta != 0; b sums every party.
template <int T>
__device__ __forceinline__ void nl_keyswitch(const LaunchShape &S, const uint32_t *__restrict__ ks,
                                             const uint32_t *ein, uint32_t *dst, int tid) {
    const uint32_t n = S.n, N = S.N, k = S.k, t = S.t;
    const uint32_t nb = (1u << S.ks_bit) - 1;
    const uint32_t round_off = 1u << (32 - S.ks_bit * t - 1);
    const size_t rowlen = n + 1;
    const size_t party_stride = (size_t)N * t * nb * rowlen;
    for (uint32_t x = tid; x <= n; x += T) {
        uint32_t bsum = 0;
        for (uint32_t i = 0; i < k; ++i) {
            const uint32_t *ksi = ks + i * party_stride + x;
            uint32_t accv = 0;
            for (uint32_t j = 0; j < N; ++j) {
                const uint32_t abar = ein[i * N + j] + round_off;
                const uint32_t *rowj = ksi + (size_t)j * t * nb * rowlen;
#pragma unroll 4
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

template <class F, int LOGN, int NPF, bool TWG, int EPT>
__host__ __device__ inline size_t netlist_smem(uint32_t k, uint32_t n) {
    const SmemLayout L = smem_layout<F, LOGN, NPF, TWG>(k, n);
    return L.total + ((sizeof(uint32_t) * (k * (1u << LOGN) + 1) + 15) & ~size_t(15)) + 16;
}

template <class F, int LOGN, int NPF, int MINB, bool TWG, int EPT>
__global__ void __launch_bounds__((1 << LOGN) / EPT, MINB)
netlist_kernel(LaunchShape S, DeviceKeys K, NetlistArgs A) {
    constexpr int N = 1 << LOGN, T = N / EPT;
    using E = typename F::E;
    using Tw = typename F::Tw;
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x;
    const SmemLayout L = smem_layout<F, LOGN, NPF, TWG>(S.k, S.n);
    const Tw *twf = static_cast<const Tw *>(K.tw_fwd);
    const Tw *twi = static_cast<const Tw *>(K.tw_inv);
    E *xbuf = reinterpret_cast<E *>(smem + L.xbuf);
    uint32_t *acc = reinterpret_cast<uint32_t *>(smem + L.acc);
    uint16_t *abar = reinterpret_cast<uint16_t *>(smem + L.abar);
    uint32_t *ext = reinterpret_cast<uint32_t *>(smem + L.total);
    volatile int32_t *item_s = reinterpret_cast<volatile int32_t *>(
        smem + L.total + ((sizeof(uint32_t) * (S.k * N + 1) + 15) & ~size_t(15)));
    const uint32_t W = S.k * S.n + 1;
#pragma unroll 1
    for (;;) {
        if (tid == 0) {
            int32_t it = -1;
            if (!*(volatile uint32_t *)A.abort) {
                const uint32_t v = atomicAdd(A.next, 1u);
                if (v < A.count) it = (int32_t)v;
            }
            if (it >= 0) {
                const GateDesc g0 = A.desc[it];
                if (!nl_wait_row(A, g0.ia, S.wait_ns, K.status) || !nl_wait_row(A, g0.ib, S.wait_ns, K.status))
                    it = -1;
            }
            *item_s = it;
        }
        __syncthreads();
        const int32_t it = *item_s;
        if (it < 0) break;
        const GateDesc g = A.desc[it];
        nl_lin_modswitch(S, g, A.pool, abar, tid, T);
        __syncthreads();
        init_acc<LOGN, EPT>(acc, S.k, abar[S.k * S.n], tid);
        __syncthreads();
        blind_rotate_core<F, LOGN, NPF, TWG, EPT>(S, K, abar, acc, xbuf, twf, twi, -1, tid);
        __syncthreads();
        sample_extract<LOGN, T>(S, acc, ext, tid);
        __syncthreads();
        nl_keyswitch<T>(S, K.ks, ext, A.pool + (size_t)g.out * W, tid);
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            if ((int64_t)it != A.skip_item) nl_store_release(A.ready + g.out, A.epoch);
            atomicAdd(A.done, 1u);
        }
    }
}

template <class F, int LOGN, int NPF, int MINB, bool TWG, int EPT>
cudaError_t launch_netlist(const LaunchShape &S, const DeviceKeys &K, const NetlistArgs &A, uint32_t sm_count,
                           cudaStream_t st) {
    if (A.count == 0) return cudaSuccess;
    if (K.status == nullptr) return cudaErrorInvalidValue;
    auto kern = netlist_kernel<F, LOGN, NPF, MINB, TWG, EPT>;
    const size_t smem = netlist_smem<F, LOGN, NPF, TWG, EPT>(S.k, S.n);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (1 << LOGN) / EPT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    uint32_t grid = (uint32_t)per_sm * sm_count;
    if (grid > A.count) grid = A.count;
    kern<<<grid, (1 << LOGN) / EPT, smem, st>>>(S, K, A);
    return cudaGetLastError();
}

}  // namespace br
}  // namespace mk
