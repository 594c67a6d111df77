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
//      accumulates c'_jj = <u_jj, d> and its share v_jj = <u_jj, A_jj>;
//      the shares go to CTA 0 through distributed shared memory;
//   2. cluster barrier; CTA 0 sums the shares, inverse-transforms v,
//      decomposes and transforms w, and hands NTT(w) to CTA i; the CTAs
//      jj not in {0, i} finish c'_jj and their step;
//   3. cluster barrier; CTAs 0 and i add <w, f0> / <w, f1> and finish.
// The critical path per step is two forward passes of d digit polynomials
// and two single inverse transforms, instead of (k+2)(d+1) transforms.
// Results are bit-identical to the batched kernel (the same exact field
// arithmetic; sums mod p are order-independent).
#pragma once
#include <cooperative_groups.h>

#include "mk_bootstrap.cuh"

namespace mk {
namespace br {

namespace cg = cooperative_groups;

// Field addition of two partial sums (each as left by mac).
__device__ __forceinline__ uint64_t fadd(const uint64_t &a, const uint64_t &b) { return add2(a, b); }
__device__ __forceinline__ uint2 fadd(const uint2 &a, const uint2 &b) {
    return make_uint2(red2p(a.x + b.x, TWO_P1), red2p(a.y + b.y, TWO_P2));
}

struct ClusterLayout {
    size_t acc, xbuf, vbuf, wbuf, abar, total;
};

template <class F, int LOGN>
__host__ __device__ inline ClusterLayout cluster_layout(uint32_t k, uint32_t n) {
    constexpr size_t N = (size_t)1 << LOGN;
    using E = typename F::E;
    ClusterLayout L;
    L.acc = 0;
    L.xbuf = L.acc + sizeof(uint32_t) * N;
    L.vbuf = L.xbuf + sizeof(E) * 3 * padded_len(N);  // three padded polynomials per forward pass
    L.wbuf = L.vbuf + sizeof(E) * (k + 1) * N;  // CTA 0: the k+1 shares of v
    L.abar = L.wbuf + sizeof(E) * 3 * N;        // CTA 0 and CTA i: NTT(w_l)
    L.total = L.abar + ((sizeof(uint16_t) * (k * n + 1) + 15) & ~size_t(15));
    return L;
}

template <class F, int LOGN>
__global__ void __launch_bounds__((1 << LOGN) / 8, 1)
bootstrap_cluster_kernel(LaunchShape S, DeviceKeys K, const GateDesc *__restrict__ desc,
                         const uint32_t *__restrict__ ct_a, const uint32_t *__restrict__ ct_b,
                         const uint32_t *__restrict__ abar_in, int64_t max_steps, uint32_t *__restrict__ ext,
                         uint32_t *__restrict__ acc_out) {
    constexpr int N = 1 << LOGN, T = N / 8;
    using E = typename F::E;
    using Tw = typename F::Tw;
    using NT = Ntt<F, LOGN, true>;
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cluster = cg::this_cluster();
    const int tid = threadIdx.x;
    const int k = (int)S.k, n = (int)S.n;
    const int jj = (int)cluster.block_rank();  // this CTA's accumulator polynomial
    const uint32_t gate = blockIdx.x / (S.k + 1);
    const ClusterLayout L = cluster_layout<F, LOGN>(S.k, S.n);
    uint32_t *acc = reinterpret_cast<uint32_t *>(smem + L.acc);
    E *xbuf = reinterpret_cast<E *>(smem + L.xbuf);
    E *vbuf = reinterpret_cast<E *>(smem + L.vbuf);
    E *wbuf = reinterpret_cast<E *>(smem + L.wbuf);
    uint16_t *abar = reinterpret_cast<uint16_t *>(smem + L.abar);
    const Tw *twf = static_cast<const Tw *>(K.tw_fwd);
    const Tw *twi = static_cast<const Tw *>(K.tw_inv);
    const E *bk_all = static_cast<const E *>(K.bk);
    const E *keyA = static_cast<const E *>(K.keyA);
    const Gadget G = make_gadget(S.bg_bit);

    // Linear part + modulus switch (each CTA of the gate computes the same words).
    if (abar_in) {
        const uint32_t W = S.k * S.n + 1;
        for (uint32_t x = tid; x < W; x += T) abar[x] = (uint16_t)abar_in[(size_t)gate * W + x];
    } else {
        lin_modswitch(S, desc[gate], ct_a, ct_b, abar, tid, T);
    }
    __syncthreads();
    const uint32_t bbar = abar[S.k * S.n];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint32_t m = tid + T * c;
        uint32_t r = m + bbar;
        if (r >= 2 * N) r -= 2 * N;
        acc[m] = jj ? 0u : ((r >= (uint32_t)N) ? (0u - (1u << 29)) : (1u << 29));
    }
    E *vbuf0 = cluster.map_shared_rank(vbuf, 0);  // CTA 0's share buffer
    cluster.sync();  // every CTA of the cluster is running before remote accesses

    int64_t steps = 0;
#pragma unroll 1
    for (int i = 1; i <= k; ++i) {
        E *wbuf_i = cluster.map_shared_rank(wbuf, i);  // CTA i receives NTT(w)
#pragma unroll 1
        for (int j = 0; j < n; ++j) {
            if (max_steps >= 0 && steps >= max_steps) break;
            ++steps;
            const uint32_t e = abar[(i - 1) * n + j];
            if (e == 0) continue;  // the same word in every CTA: the whole cluster skips
            const E *bk = bk_all + ((size_t)((i - 1) * n + j) * 9) * N;
            // 1. digits of (X^-e - 1) ACC_jj, one forward pass, c'_jj and v_jj
            E C[8], V[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) C[c] = V[c] = F::zero();
            {
                E x[3][8];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
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
                mac_npf<F, LOGN, 8, 3>(C, x, bk, tid);                             // d_1..d_3
                mac_npf<F, LOGN, 8, 3>(V, x, keyA + (size_t)jj * 3 * N, tid);      // -a or pk_jj
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) vbuf0[(size_t)jj * N + 8 * tid + c] = V[c];
            cluster.sync();  // A: the shares of v are in CTA 0
            if (jj == 0) {
                // 2. v = sum of the shares, w = g^-1(v), NTT(w) to CTA i
                E y[1][8];
#pragma unroll
                for (int c = 0; c < 8; ++c) y[0][c] = vbuf[8 * tid + c];
                for (int q = 1; q <= k; ++q)
#pragma unroll
                    for (int c = 0; c < 8; ++c) y[0][c] = fadd(y[0][c], vbuf[(size_t)q * N + 8 * tid + c]);
                NT::template inverse<1>(y, tid, twi, xbuf);
                E x[3][8];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const uint32_t vv = F::to_u32(y[0][c]);
#pragma unroll
                    for (int p = 0; p < 3; ++p) x[p][c] = F::from_digit(G.digit(vv, p));
                }
                NT::template forward<3>(x, tid, twf, xbuf);
#pragma unroll
                for (int l = 0; l < 3; ++l)
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        wbuf[(size_t)l * N + 8 * tid + c] = x[l][c];
                        wbuf_i[(size_t)l * N + 8 * tid + c] = x[l][c];
                    }
            }
            if (jj != 0 && jj != i) {  // c'_jj is complete
                E y[1][8];
#pragma unroll
                for (int c = 0; c < 8; ++c) y[0][c] = C[c];
                NT::template inverse<1>(y, tid, twi, xbuf);
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[tid + T * c] += F::to_u32(y[0][c]);
            }
            cluster.sync();  // B: NTT(w) is in CTA i
            if (jj == 0 || jj == i) {
                // 3. c'_0 += <w, f0>, c'_i += <w, f1>
                const E *f = bk + (jj == 0 ? 3 : 6) * (size_t)N;
                E w[3][8];
#pragma unroll
                for (int l = 0; l < 3; ++l)
#pragma unroll
                    for (int c = 0; c < 8; ++c) w[l][c] = wbuf[(size_t)l * N + 8 * tid + c];
                mac_npf<F, LOGN, 8, 3>(C, w, f, tid);
                E y[1][8];
#pragma unroll
                for (int c = 0; c < 8; ++c) y[0][c] = C[c];
                NT::template inverse<1>(y, tid, twi, xbuf);
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[tid + T * c] += F::to_u32(y[0][c]);
            }
            __syncthreads();
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

template <class F, int LOGN>
cudaError_t launch_bootstrap_cluster(const LaunchShape &S, const DeviceKeys &K, const GateDesc *desc,
                                     const uint32_t *ct_a, const uint32_t *ct_b, const uint32_t *abar_in,
                                     int64_t max_steps, uint32_t *ext, uint32_t *acc_out, uint32_t count,
                                     cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    if (S.k + 1 > 8) return cudaErrorInvalidValue;
    const ClusterLayout L = cluster_layout<F, LOGN>(S.k, S.n);
    auto kern = bootstrap_cluster_kernel<F, LOGN>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(count * (S.k + 1), 1, 1);
    cfg.blockDim = dim3((1 << LOGN) / 8, 1, 1);
    cfg.dynamicSmemBytes = L.total;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = S.k + 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, S, K, desc, ct_a, ct_b, abar_in, max_steps, ext, acc_out);
}

}  // namespace br
}  // namespace mk
