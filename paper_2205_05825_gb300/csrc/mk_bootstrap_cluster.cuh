// mk_bootstrap_cluster.cuh -- the latency form of the blind rotation: one
// thread-block cluster per gate, one CTA per accumulator polynomial.
//
// The batched kernel (mk_bootstrap.cuh) gives each gate one CTA, which runs
// the (k+2)(d+1) transforms of every CMux step one after the other.  For a
// small batch that leaves most SMs idle and the gate's latency is that whole
// chain.  Here CTA jj of a cluster of k+1 owns ACC_jj (shared memory) and, per
// CMux step of the hybrid product (Sec. 3.2; u_jj = g^-1((X^-e - 1) ACC_jj),
// v = sum_jj <u_jj, A_jj>, w = g^-1(v), ACC_jj += <u_jj, d>, ACC_0 += <w, f0>,
// ACC_i += <w, f1>):
//   1. every CTA transforms the digits of its own (X^-e - 1) ACC_jj and
//      accumulates c'_jj = <u_jj, d> and its share v_jj = <u_jj, A_jj>; the
//      share goes to each of the first ND = min(d, k+1) CTAs through
//      distributed shared memory;
//   2. cluster barrier; each of those CTAs sums the shares, inverse-transforms
//      v (all get the same v), decomposes it and transforms its own digit
//      polynomials of w (digit l in CTA l mod ND), writing NTT(w_l) into CTAs
//      0 and i;
//   3. cluster barrier; CTAs 0 and i add <w, f0> / <w, f1> to c'_0 / c'_i;
//      every CTA inverse-transforms its c'_jj into ACC_jj.
// The critical path per step is one forward pass of d digit polynomials, one
// of a single digit polynomial (k >= 2) and two single inverse transforms.
//
// Key entries are staged in shared memory by the bulk-copy engine
// (cp.async.bulk, completion counted on an mbarrier): the CTA's own public-key
// polynomials A_jj (-a for jj = 0, pk_jj otherwise) once, and per active CMux
// step d_1..d_d of BK_{i,j} and, in CTAs 0 and i, f0 or f1.  A buffer's copy
// for the next active step is issued once every thread has read the current
// one, so it lands while the following transforms run.  Waits on the copies
// are bounded in global time (S.wait_ns): a wait that runs out sets the CTA's
// abort word and the context's status word, later waits return at once and no
// copy is issued after it, but the CTA keeps passing every cluster barrier
// (its results are then garbage; mk_sync reports MK_ETIMEOUT); before it
// exits, thread 0 waits (bounded) for the last copy issued into each buffer.
// The twiddle tables go into shared memory too where they fit (k <= 5 at
// N = 1024); beyond that the public keys are read through L1 instead to make
// room for them (k = 6, 7), and where even that does not fit, the twiddles.
// Results are bit-identical to the batched kernel (the same exact field
// arithmetic; sums mod p are order-independent).
#pragma once
#include <cooperative_groups.h>

#include "mk_bootstrap.cuh"
#include "mk_bulk.cuh"

namespace mk {
namespace br {

namespace cg = cooperative_groups;

// Field addition of two partial sums (each as left by mac).
__device__ __forceinline__ uint64_t fadd(const uint64_t &a, const uint64_t &b) { return add2(a, b); }
__device__ __forceinline__ uint2 fadd(const uint2 &a, const uint2 &b) {
    return make_uint2(red2p(a.x + b.x, TWO_P1), red2p(a.y + b.y, TWO_P2));
}

struct ClusterCtl {
    unsigned long long bar[3];  // mbarriers of the staged buffers: A (once), D, F
    uint32_t issued[3];         // copies issued into each (thread 0)
    uint32_t abort;             // a wait of this CTA ran out
};

// Shared memory of one CTA: the staged key buffers first (bulk-copy
// destinations, 16-byte aligned), then the exchange buffer, the shares of v
// (read in CTAs 0..ND-1), NTT(w_0..w_2) (read in CTAs 0 and i), ACC_jj, the
// twiddle tables (when staged), the control block and the mod-switched words.  vbuf and wbuf hold thread tid's
// element c at c * T + tid (T threads per CTA).
struct ClusterLayout {
    size_t keyA, keyD, keyF, xbuf, vbuf, wbuf, acc, twf, twi, ctl, abar, total;
};

// TWS: the forward and inverse twiddle tables copied into shared memory
// (padded, one entry in 4) instead of read through L1.  KAS: the CTA's public
// keys staged in shared memory instead of read through L1.
template <class F, int LOGN, bool TWS, bool KAS>
__host__ __device__ inline ClusterLayout cluster_layout(uint32_t k, uint32_t n) {
    constexpr size_t N = (size_t)1 << LOGN;
    using E = typename F::E;
    using Tw = typename F::Tw;
    constexpr size_t tw_bytes = TWS ? ((sizeof(Tw) * (N + N / 4) + 15) & ~size_t(15)) : 0;
    ClusterLayout L;
    L.keyA = 0;
    L.keyD = L.keyA + (KAS ? sizeof(E) * 3 * N : 0);
    L.keyF = L.keyD + sizeof(E) * 3 * N;
    L.xbuf = L.keyF + sizeof(E) * 3 * N;
    L.vbuf = L.xbuf + sizeof(E) * 3 * padded_len(N);  // three padded polynomials per forward pass
    L.wbuf = L.vbuf + sizeof(E) * (k + 1) * N;
    L.acc = L.wbuf + sizeof(E) * 3 * N;
    L.twf = L.acc + sizeof(uint32_t) * N;
    L.twi = L.twf + tw_bytes;
    L.ctl = L.twi + tw_bytes;
    L.abar = L.ctl + ((sizeof(ClusterCtl) + 15) & ~size_t(15));
    L.total = L.abar + ((sizeof(uint16_t) * (k * n + 1) + 15) & ~size_t(15));
    return L;
}

// Every thread: wait until mbarrier `bar` has completed its phase of parity
// `parity`, bounded in global time.  Nothing branches on the outcome: a wait
// that runs out only sets the abort and status words.
__device__ __forceinline__ void cl_wait(uint32_t bar, uint32_t parity, ClusterCtl *ctl, uint64_t wait_ns,
                                        uint32_t *status) {
    if (st_mbar_try(bar, parity)) return;
    if (*(volatile uint32_t *)&ctl->abort) return;
    const uint64_t t0 = st_globaltimer();
    for (uint32_t it = 0; it < (1u << 30); ++it) {
        if (st_mbar_try(bar, parity)) return;
        if (*(volatile uint32_t *)&ctl->abort) return;
        if (st_globaltimer() - t0 > wait_ns) break;
    }
    *(volatile uint32_t *)&ctl->abort = 1u;
    atomicOr(status, kStatusCluster);
}

// Thread 0: the first step s >= s0 below `limit` with a nonzero rotation
// (and, for the F buffer, one whose party i is this CTA's polynomial, or any
// step for CTA 0); `limit` if there is none.
__device__ __forceinline__ int64_t cl_next_step(const uint16_t *abar, int64_t s0, int64_t limit, bool for_f, int jj,
                                                int n) {
    for (int64_t s = s0; s < limit; ++s) {
        if (abar[s] == 0) continue;
        if (for_f && jj != 0 && jj != (int)(s / n) + 1) continue;
        return s;
    }
    return limit;
}

// Thread 0: bulk-copy `bytes` from src into the staged buffer b for step s
// (s < 0: the public keys, copied once), unless the CTA is aborting or the
// test hook skips step s.
__device__ __forceinline__ void cl_issue(ClusterCtl *ctl, int b, uint32_t dst, const void *src, uint32_t bytes,
                                         int64_t s, int64_t skip_step) {
    if (*(volatile uint32_t *)&ctl->abort || (s >= 0 && s == skip_step)) return;
    st_fence_proxy_async();
    st_bulk_load(dst, src, bytes, st_smem_addr(&ctl->bar[b]));
    ctl->issued[b] += 1;
}

template <class F, int LOGN, int EPT, bool TWS, bool KAS>
__global__ void __launch_bounds__((1 << LOGN) / EPT, 1)
bootstrap_cluster_kernel(LaunchShape S, DeviceKeys K, const GateDesc *__restrict__ desc,
                         const uint32_t *__restrict__ ct_a, const uint32_t *__restrict__ ct_b,
                         const uint32_t *__restrict__ abar_in, int64_t max_steps, uint32_t *__restrict__ ext,
                         uint32_t *__restrict__ acc_out) {
    constexpr int N = 1 << LOGN, T = N / EPT;
    using E = typename F::E;
    using Tw = typename F::Tw;
    using NT = Ntt<F, LOGN, !TWS, EPT>;
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cluster = cg::this_cluster();
    const int tid = threadIdx.x;
    const int k = (int)S.k, n = (int)S.n;
    const int jj = (int)cluster.block_rank();  // this CTA's accumulator polynomial
    const int ND = k + 1 < 3 ? k + 1 : 3;      // CTAs that transform the digits of w
    const uint32_t gate = blockIdx.x / (S.k + 1);
    const ClusterLayout L = cluster_layout<F, LOGN, TWS, KAS>(S.k, S.n);
    const E *keyA_s = reinterpret_cast<const E *>(smem + L.keyA);
    const E *keyD_s = reinterpret_cast<const E *>(smem + L.keyD);
    const E *keyF_s = reinterpret_cast<const E *>(smem + L.keyF);
    E *xbuf = reinterpret_cast<E *>(smem + L.xbuf);
    E *vbuf = reinterpret_cast<E *>(smem + L.vbuf);
    E *wbuf = reinterpret_cast<E *>(smem + L.wbuf);
    uint32_t *acc = reinterpret_cast<uint32_t *>(smem + L.acc);
    ClusterCtl *ctl = reinterpret_cast<ClusterCtl *>(smem + L.ctl);
    uint16_t *abar = reinterpret_cast<uint16_t *>(smem + L.abar);
    const Tw *twf, *twi;
    if constexpr (TWS) {
        twf = reinterpret_cast<const Tw *>(smem + L.twf);
        twi = reinterpret_cast<const Tw *>(smem + L.twi);
        load_twiddles<F, LOGN, EPT>(K, reinterpret_cast<Tw *>(smem + L.twf), reinterpret_cast<Tw *>(smem + L.twi),
                                    tid);
    } else {
        twf = static_cast<const Tw *>(K.tw_fwd);
        twi = static_cast<const Tw *>(K.tw_inv);
    }
    const E *bk_all = static_cast<const E *>(K.bk);
    const E *keyA = static_cast<const E *>(K.keyA);
    const Gadget G = make_gadget(S.bg_bit);
    const uint32_t key_bytes = (uint32_t)(sizeof(E) * 3 * N);
    const uint32_t barA = st_smem_addr(&ctl->bar[0]), barD = st_smem_addr(&ctl->bar[1]),
                   barF = st_smem_addr(&ctl->bar[2]);
    const int64_t all_steps = (int64_t)k * n;
    const int64_t limit = (max_steps >= 0 && max_steps < all_steps) ? max_steps : all_steps;

    if (tid == 0) {
        for (int b = 0; b < 3; ++b) {
            st_mbar_init(st_smem_addr(&ctl->bar[b]), 1);
            ctl->issued[b] = 0;
        }
        ctl->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    // Linear part + modulus switch (each CTA of the gate computes the same words).
    if (abar_in) {
        const uint32_t W = S.k * S.n + 1;
        for (uint32_t x = tid; x < W; x += T) abar[x] = (uint16_t)abar_in[(size_t)gate * W + x];
    } else {
        lin_modswitch(S, desc[gate], ct_a, ct_b, abar, tid, T);
    }
    __syncthreads();
    if (tid == 0) {  // A_jj once; d and f of the first active steps
        if (KAS) cl_issue(ctl, 0, st_smem_addr(keyA_s), keyA + (size_t)jj * 3 * N, key_bytes, -1, -1);
        const int64_t sd = cl_next_step(abar, 0, limit, false, jj, n);
        if (sd < limit) cl_issue(ctl, 1, st_smem_addr(keyD_s), bk_all + (size_t)sd * 9 * N, key_bytes, sd, S.skip_key_step);
        const int64_t sf = cl_next_step(abar, 0, limit, true, jj, n);
        if (sf < limit)
            cl_issue(ctl, 2, st_smem_addr(keyF_s), bk_all + ((size_t)sf * 9 + (jj == 0 ? 3 : 6)) * N, key_bytes, sf,
                     S.skip_key_step);
    }
    const uint32_t bbar = abar[S.k * S.n];
#pragma unroll
    for (int c = 0; c < EPT; ++c) {
        const uint32_t m = tid + T * c;
        uint32_t r = m + bbar;
        if (r >= 2 * N) r -= 2 * N;
        acc[m] = jj ? 0u : ((r >= (uint32_t)N) ? (0u - (1u << 29)) : (1u << 29));
    }
    E *vdst[3];  // the share buffers this CTA writes into (CTAs 0..ND-1)
#pragma unroll
    for (int r = 0; r < 3; ++r) vdst[r] = (r < ND) ? (r == jj ? vbuf : cluster.map_shared_rank(vbuf, r)) : nullptr;
    E *wbuf0 = jj == 0 ? wbuf : cluster.map_shared_rank(wbuf, 0);
    cluster.sync();  // every CTA of the cluster is running before remote accesses
    if (KAS) cl_wait(barA, 0, ctl, S.wait_ns, K.status);

    uint32_t nD = 0, nF = 0;  // waits done on the D and F buffers
#pragma unroll 1
    for (int64_t s = 0; s < limit; ++s) {
        const uint32_t e = abar[s];
        if (e == 0) continue;  // the same word in every CTA: the whole cluster skips
        const int i = (int)(s / n) + 1;
        const bool with_f = (jj == 0 || jj == i);
        // 1. digits of (X^-e - 1) ACC_jj, one forward pass, c'_jj and v_jj
        E C[EPT], V[EPT];
#pragma unroll
        for (int c = 0; c < EPT; ++c) C[c] = V[c] = F::zero();
        {
            E x[3][EPT];
#pragma unroll
            for (int c = 0; c < EPT; ++c) {
                const uint32_t m = tid + T * c;
                uint32_t r = m + e;
                if (r >= 2 * N) r -= 2 * N;
                uint32_t a = acc[r & (N - 1)];
                if (r >= (uint32_t)N) a = 0u - a;
                const uint32_t D = a - acc[m];
#pragma unroll
                for (int p = 0; p < 3; ++p) x[p][c] = F::from_digit(G.digit(D, p));
            }
            NT::template forward<3>(x, tid, twf, xbuf);
            cl_wait(barD, nD & 1u, ctl, S.wait_ns, K.status);
            ++nD;
            mac_npf<F, LOGN, EPT, 3, true>(C, x, keyD_s, tid);  // d_1..d_3
            if constexpr (KAS) mac_npf<F, LOGN, EPT, 3, true>(V, x, keyA_s, tid);  // -a or pk_jj
            else mac_npf<F, LOGN, EPT, 3, false>(V, x, keyA + (size_t)jj * 3 * N, tid);
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            if (r >= ND) break;
#pragma unroll
            for (int c = 0; c < EPT; ++c) vdst[r][(size_t)jj * N + c * T + tid] = V[c];
        }
        __syncthreads();  // every read of this step's d is done
        if (tid == 0) {
            const int64_t sd = cl_next_step(abar, s + 1, limit, false, jj, n);
            if (sd < limit)
                cl_issue(ctl, 1, st_smem_addr(keyD_s), bk_all + (size_t)sd * 9 * N, key_bytes, sd, S.skip_key_step);
        }
        cluster.sync();  // A: the shares of v are in CTAs 0..ND-1
        if (jj < ND) {
            // 2. v = sum of the shares, w = g^-1(v), NTT of this CTA's digits of w to CTAs 0 and i
            E *wbuf_i = jj == i ? wbuf : cluster.map_shared_rank(wbuf, i);
            E y[1][EPT];
#pragma unroll
            for (int c = 0; c < EPT; ++c) y[0][c] = vbuf[c * T + tid];
            for (int q = 1; q <= k; ++q)
#pragma unroll
                for (int c = 0; c < EPT; ++c) y[0][c] = fadd(y[0][c], vbuf[(size_t)q * N + c * T + tid]);
            NT::template inverse<1>(y, tid, twi, xbuf);
            uint32_t vv[EPT];
#pragma unroll
            for (int c = 0; c < EPT; ++c) vv[c] = F::to_u32(y[0][c]);
#pragma unroll 1
            for (int l = jj; l < 3; l += ND) {
                E x[1][EPT];
#pragma unroll
                for (int c = 0; c < EPT; ++c) x[0][c] = F::from_digit(G.digit(vv[c], l));
                NT::template forward<1>(x, tid, twf, xbuf);
#pragma unroll
                for (int c = 0; c < EPT; ++c) {
                    wbuf0[(size_t)l * N + c * T + tid] = x[0][c];
                    wbuf_i[(size_t)l * N + c * T + tid] = x[0][c];
                }
            }
        }
        cluster.sync();  // B: NTT(w) is in CTAs 0 and i
        if (with_f) {
            // 3a. c'_0 += <w, f0>, c'_i += <w, f1>
            cl_wait(barF, nF & 1u, ctl, S.wait_ns, K.status);
            ++nF;
            E w[3][EPT];
#pragma unroll
            for (int l = 0; l < 3; ++l)
#pragma unroll
                for (int c = 0; c < EPT; ++c) w[l][c] = wbuf[(size_t)l * N + c * T + tid];
            mac_npf<F, LOGN, EPT, 3, true>(C, w, keyF_s, tid);
            __syncthreads();  // every read of this step's f is done
            if (tid == 0) {
                const int64_t sf = cl_next_step(abar, s + 1, limit, true, jj, n);
                if (sf < limit)
                    cl_issue(ctl, 2, st_smem_addr(keyF_s), bk_all + ((size_t)sf * 9 + (jj == 0 ? 3 : 6)) * N,
                             key_bytes, sf, S.skip_key_step);
            }
        }
        // 3b. ACC_jj += c'_jj
        {
            E y[1][EPT];
#pragma unroll
            for (int c = 0; c < EPT; ++c) y[0][c] = C[c];
            NT::template inverse<1>(y, tid, twi, xbuf);
#pragma unroll
            for (int c = 0; c < EPT; ++c) acc[tid + T * c] += F::to_u32(y[0][c]);
        }
        __syncthreads();
    }
    if (tid == 0) {  // no copy of this CTA may be in flight when it exits
        for (int b = 0; b < 3; ++b) {
            const uint32_t cnt = ctl->issued[b];
            if (cnt == 0) continue;
            const uint32_t bar = st_smem_addr(&ctl->bar[b]);
            const uint64_t t0 = st_globaltimer();
            for (uint32_t it = 0; it < (1u << 30); ++it) {
                if (st_mbar_try(bar, (cnt - 1) & 1u)) break;
                if (st_globaltimer() - t0 > S.wait_ns) break;
            }
        }
    }
    __syncthreads();
    if (acc_out) {
        uint32_t *dst = acc_out + ((size_t)gate * (S.k + 1) + jj) * N;
        for (int x = tid; x < N; x += T) dst[x] = acc[x];
    } else {
        uint32_t *dst = ext + (size_t)gate * (S.k * N + 1);
        if (jj == 0) {
            if (tid == 0) dst[S.k * N] = acc[0] + (1u << 29);  // +1/8
        } else {
            uint32_t *ai = dst + (size_t)(jj - 1) * N;  // SampleExtract of ACC_jj
            for (int m = tid; m < N; m += T) ai[m] = (m == 0) ? acc[0] : 0u - acc[N - m];
        }
    }
    cluster.sync();  // no CTA leaves while another could still address its shared memory
}

// Elements of a polynomial per thread in the cluster kernel (N / kClusterEpt
// threads per CTA).  One CTA per SM runs here, so latency is hidden by warps
// rather than by other CTAs: 4 (eight warps, two butterfly stages per
// register pass) measured 10-12 % faster per gate than 8 on GB300.
constexpr int kClusterEpt = 4;
constexpr size_t kClusterSmemMax = 227 * 1024;

// What goes into shared memory besides the step's keys, by fit: the twiddle
// tables and the public keys (0), the twiddle tables only (1: large k), the
// public keys only (2); -1 if not even the step's keys fit (large k n).
template <class F, int LOGN>
__host__ __device__ inline int cluster_mode(uint32_t k, uint32_t n) {
    if (cluster_layout<F, LOGN, true, true>(k, n).total <= kClusterSmemMax) return 0;
    if (cluster_layout<F, LOGN, true, false>(k, n).total <= kClusterSmemMax) return 1;
    if (cluster_layout<F, LOGN, false, true>(k, n).total <= kClusterSmemMax) return 2;
    return -1;
}

template <class F, int LOGN, bool TWS, bool KAS>
cudaLaunchConfig_t cluster_config(uint32_t k, uint32_t n, uint32_t count, cudaStream_t st, cudaLaunchAttribute *attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(count * (k + 1), 1, 1);
    cfg.blockDim = dim3((1 << LOGN) / kClusterEpt, 1, 1);
    cfg.dynamicSmemBytes = cluster_layout<F, LOGN, TWS, KAS>(k, n).total;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = k + 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

template <class F, int LOGN, bool TWS, bool KAS>
int cluster_capacity_t(uint32_t k, uint32_t n) {
    auto kern = bootstrap_cluster_kernel<F, LOGN, kClusterEpt, TWS, KAS>;
    const size_t smem = cluster_layout<F, LOGN, TWS, KAS>(k, n).total;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = cluster_config<F, LOGN, TWS, KAS>(k, n, 1, nullptr, attr);
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess) return 0;
    return clusters;
}

// Clusters of this shape that can be resident at once (one wave of gates), or
// 0 if the device cannot run them.
template <class F, int LOGN>
int cluster_capacity(uint32_t k, uint32_t n) {
    if (k + 1 > 8) return 0;
    switch (cluster_mode<F, LOGN>(k, n)) {
        case 0: return cluster_capacity_t<F, LOGN, true, true>(k, n);
        case 1: return cluster_capacity_t<F, LOGN, true, false>(k, n);
        case 2: return cluster_capacity_t<F, LOGN, false, true>(k, n);
        default: return 0;
    }
}

template <class F, int LOGN, bool TWS, bool KAS>
cudaError_t launch_bootstrap_cluster_t(const LaunchShape &S, const DeviceKeys &K, const GateDesc *desc,
                                       const uint32_t *ct_a, const uint32_t *ct_b, const uint32_t *abar_in,
                                       int64_t max_steps, uint32_t *ext, uint32_t *acc_out, uint32_t count,
                                       cudaStream_t st) {
    auto kern = bootstrap_cluster_kernel<F, LOGN, kClusterEpt, TWS, KAS>;
    const size_t smem = cluster_layout<F, LOGN, TWS, KAS>(S.k, S.n).total;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = cluster_config<F, LOGN, TWS, KAS>(S.k, S.n, count, st, attr);
    return cudaLaunchKernelEx(&cfg, kern, S, K, desc, ct_a, ct_b, abar_in, max_steps, ext, acc_out);
}

template <class F, int LOGN>
cudaError_t launch_bootstrap_cluster(const LaunchShape &S, const DeviceKeys &K, const GateDesc *desc,
                                     const uint32_t *ct_a, const uint32_t *ct_b, const uint32_t *abar_in,
                                     int64_t max_steps, uint32_t *ext, uint32_t *acc_out, uint32_t count,
                                     cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    if (S.k + 1 > 8 || K.status == nullptr) return cudaErrorInvalidValue;
    switch (cluster_mode<F, LOGN>(S.k, S.n)) {
        case 0:
            return launch_bootstrap_cluster_t<F, LOGN, true, true>(S, K, desc, ct_a, ct_b, abar_in, max_steps, ext,
                                                                   acc_out, count, st);
        case 1:
            return launch_bootstrap_cluster_t<F, LOGN, true, false>(S, K, desc, ct_a, ct_b, abar_in, max_steps, ext,
                                                                    acc_out, count, st);
        case 2:
            return launch_bootstrap_cluster_t<F, LOGN, false, true>(S, K, desc, ct_a, ct_b, abar_in, max_steps, ext,
                                                                    acc_out, count, st);
        default:
            return cudaErrorInvalidConfiguration;  // the shape needs more shared memory than a CTA has
    }
}

}  // namespace br
}  // namespace mk
