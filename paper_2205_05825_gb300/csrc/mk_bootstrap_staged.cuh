// mk_bootstrap_staged.cuh -- the blind rotation with each CMux step's
// bootstrapping-key entry staged once in shared memory and shared by the G
// gates of a CTA.
//
// Same arithmetic as the CTA-per-gate kernel (mk_bootstrap.cuh): gate linear
// part and modulus switch (Sec. 4.1, Eq. 6-11), then for i = 1..k, j = 0..n-1
// the CMux step ACC += HP((X^-e - 1) ACC, BK_{i,j}) with the hybrid product of
// the MKTFHE construction named in Sec. 3.2, then SampleExtract and +1/8.
// The difference is who reads BK_{i,j}.  There, every gate's CTA loads the
// 9 N-element entry of every step from L2 itself, at whatever step it has
// reached; resident CTAs drift apart, so entries are re-read from DRAM many
// times per launch.  Here a CTA holds G gates, one group of N/8 threads each,
// and the groups walk the k*n steps together: per step the entry is copied
// once from global into shared memory by the bulk-copy engine
// (cp.async.bulk, completion counted on an mbarrier) and every group reads it
// from there.
//
// The entry splits into D = (d_1..d_3), used by phase A of the step (the
// products of every accumulator polynomial's digits), and F = (f0_1..f0_3,
// f1_1..f1_3), used by phase B (the products of w = g^-1(v)).  Each has one
// buffer.  A group that has finished with a buffer at step s increments that
// buffer's counter (after a group barrier, so all its threads' reads are
// done); the group whose increment completes the step's G arrivals issues
// the copy of step s + 1 into the buffer.  The copy of D for s + 1 thus runs
// during phase B of s and the copy of F during phase A of s + 1; no group
// waits for another except through a copy it needs.  A group whose gate
// skips step s (e = 0, where HP adds nothing) still waits for and releases
// both buffers of s, so the arrivals of consecutive steps never mix.
//
// Waits on the copies are bounded in global time (S.wait_ns): a wait that
// runs out sets the CTA's abort flag and the context's status word; every
// group then leaves the step loop at its next wait, thread 0 waits (again
// bounded) for the copies still in flight, and the CTA returns without
// writing outputs.  The host reports the status as MK_ETIMEOUT.
#pragma once
#include "mk_bootstrap.cuh"
#include "mk_bulk.cuh"

namespace mk {
namespace br {

// ------------------------------------------------------------ shared-memory layout
// [D buffer: 3 N][F buffer: 6 N] elements, the control block, then per group
// [exchange buffer][ACC (k+1) N words][abar (k n + 1) half-words].
struct StagedCtl {
    unsigned long long full[2];  // mbarriers: D, F
    uint32_t count[2];           // releases of D, F (monotonic: G per step)
    uint32_t issued[2];          // copies issued into D, F
    uint32_t abort;              // some wait of this CTA ran out
    uint32_t ok[15];             // per group: the result of its leader's last wait
};

struct StagedLayout {
    size_t keyD, keyF, ctl, group0, xbuf, acc, abar, group_bytes, total;
};

template <class F, int LOGN, int NPF>
__host__ __device__ inline StagedLayout staged_layout(uint32_t k, uint32_t n, int G) {
    constexpr size_t N = (size_t)1 << LOGN;
    using E = typename F::E;
    StagedLayout L;
    L.keyD = 0;
    L.keyF = L.keyD + sizeof(E) * 3 * N;
    L.ctl = L.keyF + sizeof(E) * 6 * N;
    L.group0 = (L.ctl + sizeof(StagedCtl) + 127) & ~size_t(127);
    L.xbuf = 0;  // offsets within a group
    L.acc = L.xbuf + sizeof(E) * (NPF > 2 ? NPF : 2) * padded_len(N);
    L.abar = L.acc + sizeof(uint32_t) * (k + 1) * N;
    L.group_bytes = (L.abar + sizeof(uint16_t) * (k * n + 1) + 127) & ~size_t(127);
    L.total = L.group0 + (size_t)G * L.group_bytes;
    return L;
}

// ------------------------------------------------------------ key ring
// The two staged buffers of a CTA and its step sequence.
template <class E>
struct KeyRing {
    StagedCtl *ctl;
    uint32_t dst[2];       // shared addresses of the D and F buffers
    uint32_t bytes[2];     // their sizes
    const E *bk_all;       // BK, [k][n][3][d][N] NTT domain
    uint32_t N;
    int G;
    int64_t total;         // steps this launch runs
    int64_t skip_step;     // test hook: the copies of this step are never issued (-1: none)
    uint64_t wait_ns;
    uint32_t *status;      // the context's status word (bit 0: a wait ran out)

    // Issue the copy of buffer b (0 = D, 1 = F) for step s (s < total).
    __device__ __forceinline__ void issue(int b, int64_t s) {
        if (s == skip_step) return;
        const E *src = bk_all + (size_t)s * 9 * N + (b ? 3 * (size_t)N : 0);
        st_fence_proxy_async();
        st_bulk_load(dst[b], src, bytes[b], st_smem_addr(&ctl->full[b]));
        ctl->issued[b] += 1;  // issuers of one buffer are ordered by its counter
    }

    // Leader thread of a group: wait until buffer b holds step s; false if the
    // wait ran out or the CTA is aborting.
    __device__ bool wait_leader(int b, int64_t s) {
        const uint32_t bar = st_smem_addr(&ctl->full[b]);
        const uint32_t parity = (uint32_t)(s & 1);
        if (st_mbar_try(bar, parity)) return true;
        const uint64_t t0 = st_globaltimer();
        for (uint32_t it = 0; it < (1u << 30); ++it) {
            if (st_mbar_try(bar, parity)) return true;
            if (*(volatile uint32_t *)&ctl->abort) return false;
            if (st_globaltimer() - t0 > wait_ns) break;
        }
        *(volatile uint32_t *)&ctl->abort = 1;
        atomicOr(status, kStatusStaged);
        return false;
    }

    // All threads of group g (tid its index in the group, bar_id its barrier):
    // wait for buffer b at step s; the leader waits and the group learns the
    // outcome through shared memory, so every thread of the group takes the
    // same branch.
    __device__ __forceinline__ bool wait(int b, int64_t s, int g, int tid, int bar_id, int T) {
        if (tid == 0) ctl->ok[g] = wait_leader(b, s) ? 1u : 0u;
        group_sync(bar_id, T);
        return *(volatile uint32_t *)&ctl->ok[g] != 0;
    }

    // All threads of a group, after their last read of buffer b at step s:
    // the leader counts the release; the G-th release of the step issues the
    // copy of step s + 1.
    __device__ __forceinline__ void release(int b, int64_t s, int tid, int bar_id, int T) {
        group_sync(bar_id, T);
        if (tid == 0) {
            const uint32_t old = st_atom_add_acqrel(st_smem_addr(&ctl->count[b]), 1u);
            if ((old + 1) % (uint32_t)G == 0 && s + 1 < total) issue(b, s + 1);
        }
    }

    // Thread 0 after the step loop of an aborted CTA: wait (bounded) for the
    // last copy issued into each buffer, so none is in flight at exit.
    __device__ void drain() {
        for (int b = 0; b < 2; ++b) {
            const uint32_t n_issued = *(volatile uint32_t *)&ctl->issued[b];
            if (n_issued == 0) continue;
            const uint32_t bar = st_smem_addr(&ctl->full[b]);
            const uint32_t parity = (n_issued - 1) & 1u;
            const uint64_t t0 = st_globaltimer();
            for (uint32_t it = 0; it < (1u << 30); ++it) {
                if (st_mbar_try(bar, parity)) break;
                if (st_globaltimer() - t0 > wait_ns) break;
            }
        }
    }
};

// One CMux step of one gate (ACC += HP((X^-e - 1) ACC, BK_{i,j}), party i)
// with D and F read from the ring's shared buffers; the slot order and the
// transform pairing are those of cmux_step.  Returns false on abort.
template <class F, int LOGN, int NPF>
__device__ __forceinline__ bool staged_step(const LaunchShape &S, const typename F::E *keyA, const Gadget &Gd,
                                            KeyRing<typename F::E> &R, const typename F::E *kD,
                                            const typename F::E *kF, int64_t s, int i, uint32_t e, uint32_t *acc,
                                            typename F::E *xbuf, const typename F::Tw *twf,
                                            const typename F::Tw *twi, int g, int tid, int bar_id) {
    constexpr int EPT = 8;
    using NT = Ntt<F, LOGN, true, EPT>;
    using E = typename F::E;
    constexpr int N = NT::N, T = NT::T;
    const int k = (int)S.k;
    if (e == 0) {  // X^0 - 1 = 0: HP adds nothing, but the buffers of s are waited for and released
        if (!R.wait(0, s, g, tid, bar_id, T)) return false;
        R.release(0, s, tid, bar_id, T);
        if (!R.wait(1, s, g, tid, bar_id, T)) return false;
        R.release(1, s, tid, bar_id, T);
        return true;
    }
    E C0[EPT], CI[EPT], CJ[EPT], V[EPT];
    uint32_t vv[EPT];
#pragma unroll
    for (int c = 0; c < EPT; ++c) C0[c] = CI[c] = CJ[c] = V[c] = F::zero();
#pragma unroll 1
    for (int q = 0; q <= k + 1; ++q) {
        const int jj = (q == 0) ? 0 : (q == 1 ? i : (q - 1 < i ? q - 1 : q));  // q <= k only
        if (q >= 2 && q <= k) {
#pragma unroll
            for (int c = 0; c < EPT; ++c) CJ[c] = F::zero();
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
                    for (int p = 0; p < NPF; ++p) x[p][c] = F::from_digit(Gd.digit(D, l0 + p));
                }
            } else {
#pragma unroll
                for (int c = 0; c < EPT; ++c)
#pragma unroll
                    for (int p = 0; p < NPF; ++p) x[p][c] = F::from_digit(Gd.digit(vv[c], l0 + p));
            }
            NT::template forward<NPF>(x, tid, twf, xbuf, bar_id);
            if (l0 == 0 && (q == 0 || q == k + 1)) {  // the slot's first read of D (phase A) or F (phase B)
                if (!R.wait(q == 0 ? 0 : 1, s, g, tid, bar_id, T)) return false;
            }
            if (q <= k) {
                const E *kd = kD + l0 * N;                               // d_l0.. of BK_{i,j} (shared memory)
                const E *ka = keyA + ((size_t)jj * 3 + l0) * N;          // -a_l0.. or pk_jj[l0..]
                if (q == 0) mac_npf<F, LOGN, EPT, NPF, true>(C0, x, kd, tid);
                else if (q == 1) mac_npf<F, LOGN, EPT, NPF, true>(CI, x, kd, tid);
                else mac_npf<F, LOGN, EPT, NPF, true>(CJ, x, kd, tid);
                mac_npf<F, LOGN, EPT, NPF>(V, x, ka, tid);
            } else {
                mac_npf<F, LOGN, EPT, NPF, true>(C0, x, kF + l0 * N, tid);        // f0_l0..
                mac_npf<F, LOGN, EPT, NPF, true>(CI, x, kF + (3 + l0) * N, tid);  // f1_l0..
            }
        }
        if (q == k) R.release(0, s, tid, bar_id, T);      // the last read of D in this step
        if (q == k + 1) R.release(1, s, tid, bar_id, T);  // the last read of F
        const bool pair = (q == k && k >= 2) || q == k + 1;
        const bool single = (q >= 2 && q < k) || (q == k && k == 1);
        if (pair) {
            const bool last = (q == k + 1);
            E y[2][EPT];
#pragma unroll
            for (int c = 0; c < EPT; ++c) {
                y[0][c] = last ? C0[c] : CJ[c];
                y[1][c] = last ? CI[c] : V[c];
            }
            NT::template inverse<2>(y, tid, twi, xbuf, bar_id);
            uint32_t *d0 = acc + (last ? 0 : jj) * N;
#pragma unroll
            for (int c = 0; c < EPT; ++c) d0[tid + T * c] += F::to_u32(y[0][c]);
            if (last) {
                uint32_t *d1 = acc + i * N;
#pragma unroll
                for (int c = 0; c < EPT; ++c) d1[tid + T * c] += F::to_u32(y[1][c]);
            } else {
#pragma unroll
                for (int c = 0; c < EPT; ++c) vv[c] = F::to_u32(y[1][c]);
            }
        } else if (single) {
            const bool is_v = (q == k);
            E y[1][EPT];
#pragma unroll
            for (int c = 0; c < EPT; ++c) y[0][c] = is_v ? V[c] : CJ[c];
            NT::template inverse<1>(y, tid, twi, xbuf, bar_id);
            if (is_v) {
#pragma unroll
                for (int c = 0; c < EPT; ++c) vv[c] = F::to_u32(y[0][c]);
            } else {
                uint32_t *dst = acc + jj * N;
#pragma unroll
                for (int c = 0; c < EPT; ++c) dst[tid + T * c] += F::to_u32(y[0][c]);
            }
        }
    }
    return true;
}

// G gates per CTA (gates blockIdx.x * G + g; the groups past `count` in the
// last CTA repeat its last gate and write nothing).  Inputs and outputs as
// bootstrap_ntt_kernel.
template <class F, int LOGN, int NPF, int G>
__global__ void __launch_bounds__(G *((1 << LOGN) / 8), 1)
bootstrap_staged_kernel(LaunchShape S, DeviceKeys K, const GateDesc *__restrict__ desc,
                        const uint32_t *__restrict__ ct_a, const uint32_t *__restrict__ ct_b,
                        const uint32_t *__restrict__ abar_in, int64_t max_steps, uint32_t *__restrict__ ext,
                        uint32_t *__restrict__ acc_out, uint32_t count) {
    constexpr int N = 1 << LOGN, EPT = 8, T = N / EPT;
    using E = typename F::E;
    using Tw = typename F::Tw;
    extern __shared__ __align__(16) unsigned char smem[];
    const int g = threadIdx.x / T, tid = threadIdx.x % T, bar_id = 1 + g;
    const uint32_t gate_raw = blockIdx.x * G + g;
    const bool live = gate_raw < count;
    const uint32_t gate = live ? gate_raw : count - 1;
    const StagedLayout L = staged_layout<F, LOGN, NPF>(S.k, S.n, G);
    StagedCtl *ctl = reinterpret_cast<StagedCtl *>(smem + L.ctl);
    const E *kD = reinterpret_cast<const E *>(smem + L.keyD);
    const E *kF = reinterpret_cast<const E *>(smem + L.keyF);
    unsigned char *gbase = smem + L.group0 + (size_t)g * L.group_bytes;
    E *xbuf = reinterpret_cast<E *>(gbase + L.xbuf);
    uint32_t *acc = reinterpret_cast<uint32_t *>(gbase + L.acc);
    uint16_t *abar = reinterpret_cast<uint16_t *>(gbase + L.abar);
    const Tw *twf = static_cast<const Tw *>(K.tw_fwd);
    const Tw *twi = static_cast<const Tw *>(K.tw_inv);

    const int64_t all_steps = (int64_t)S.k * S.n;
    KeyRing<E> R;
    R.ctl = ctl;
    R.dst[0] = st_smem_addr(smem + L.keyD);
    R.dst[1] = st_smem_addr(smem + L.keyF);
    R.bytes[0] = (uint32_t)(sizeof(E) * 3 * N);
    R.bytes[1] = (uint32_t)(sizeof(E) * 6 * N);
    R.bk_all = static_cast<const E *>(K.bk);
    R.N = N;
    R.G = G;
    R.total = (max_steps >= 0 && max_steps < all_steps) ? max_steps : all_steps;
    R.skip_step = S.skip_key_step;
    R.wait_ns = S.wait_ns;
    R.status = K.status;

    if (threadIdx.x == 0) {
        st_mbar_init(st_smem_addr(&ctl->full[0]), 1);
        st_mbar_init(st_smem_addr(&ctl->full[1]), 1);
        ctl->count[0] = ctl->count[1] = 0;
        ctl->issued[0] = ctl->issued[1] = 0;
        ctl->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && R.total > 0) {
        R.issue(0, 0);
        R.issue(1, 0);
    }
    // Linear part + modulus switch and ACC init of this group's gate.
    if (abar_in) {
        const uint32_t W = S.k * S.n + 1;
        for (uint32_t x = tid; x < W; x += T) abar[x] = (uint16_t)abar_in[(size_t)gate * W + x];
    } else {
        lin_modswitch(S, desc[gate], ct_a, ct_b, abar, tid, T);
    }
    group_sync(bar_id, T);
    init_acc<LOGN, EPT>(acc, S.k, abar[S.k * S.n], tid);
    group_sync(bar_id, T);

    const Gadget Gd = make_gadget(S.bg_bit);
    const int n = (int)S.n;
    const E *keyA = static_cast<const E *>(K.keyA);
    bool ok = true;
#pragma unroll 1
    for (int64_t s = 0; ok && s < R.total; ++s) {
        const int i = (int)(s / n) + 1, j = (int)(s % n);
        const uint32_t e = abar[(i - 1) * n + j];
        ok = staged_step<F, LOGN, NPF>(S, keyA, Gd, R, kD, kF, s, i, e, acc, xbuf, twf, twi, g, tid, bar_id);
        if (!ok) break;
        group_sync(bar_id, T);  // ACC updates of the step are visible to the next rotation
    }
    __syncthreads();
    if (*(volatile uint32_t *)&ctl->abort) {
        if (threadIdx.x == 0) R.drain();
        return;
    }
    if (!live) return;
    if (acc_out) {
        uint32_t *dst = acc_out + (size_t)gate * (S.k + 1) * N;
        for (uint32_t x = tid; x < (S.k + 1) * N; x += T) dst[x] = acc[x];
    } else {
        sample_extract<LOGN, T>(S, acc, ext + (size_t)gate * (S.k * N + 1), tid);
    }
}

// G gates per CTA; the last CTA's groups past `count` repeat its last gate.
template <class F, int LOGN, int NPF, int G>
cudaError_t launch_staged_g(const LaunchShape &S, const DeviceKeys &K, const GateDesc *desc, const uint32_t *ct_a,
                            const uint32_t *ct_b, const uint32_t *abar_in, int64_t max_steps, uint32_t *ext,
                            uint32_t *acc_out, uint32_t count, cudaStream_t st) {
    const StagedLayout L = staged_layout<F, LOGN, NPF>(S.k, S.n, G);
    auto kern = bootstrap_staged_kernel<F, LOGN, NPF, G>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return e;
    const uint32_t blocks = (count + G - 1) / G;
    kern<<<blocks, G * ((1 << LOGN) / 8), L.total, st>>>(S, K, desc, ct_a, ct_b, abar_in, max_steps, ext, acc_out,
                                                        count);
    return cudaGetLastError();
}

constexpr size_t kStagedSmemMax = 227 * 1024;

// Up to 3 groups (about 170 registers a thread), 2 where 3 do not fit (large k).
template <class F, int LOGN, int NPF>
cudaError_t launch_staged(const LaunchShape &S, const DeviceKeys &K, const GateDesc *desc, const uint32_t *ct_a,
                          const uint32_t *ct_b, const uint32_t *abar_in, int64_t max_steps, uint32_t *ext,
                          uint32_t *acc_out, uint32_t count, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    if (K.status == nullptr) return cudaErrorInvalidValue;
    if (staged_layout<F, LOGN, NPF>(S.k, S.n, 3).total <= kStagedSmemMax)
        return launch_staged_g<F, LOGN, NPF, 3>(S, K, desc, ct_a, ct_b, abar_in, max_steps, ext, acc_out, count, st);
    if (staged_layout<F, LOGN, NPF>(S.k, S.n, 2).total <= kStagedSmemMax)
        return launch_staged_g<F, LOGN, NPF, 2>(S, K, desc, ct_a, ct_b, abar_in, max_steps, ext, acc_out, count, st);
    return cudaErrorInvalidValue;
}

}  // namespace br
}  // namespace mk
