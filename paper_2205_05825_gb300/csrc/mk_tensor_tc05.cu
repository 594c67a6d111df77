// mk_tensor_tc05.cu -- the Toeplitz products of the tensor form on the
// fifth-generation tensor cores (tcgen05.mma kind::f16, accumulators in TMEM).
//
// Same contraction as tc_products_kernel (mk_tensor.cu): for one output
// polynomial of every gate of a wave, sum over nchunks key polynomials and
// the four signed byte planes b of the key
//   out[g][m] += 2^(8b) * sum_t T_b[m][t] * u[g][t],  T_b[m][t] = ext_b[m - t],
// with bf16 operands (signed bytes and 8-bit digits are exact in bf16) and
// fp32 accumulation, exact while every (chunk, plane) sum stays within 2^24.
//
// A CTA owns 128 output coefficients m0..m0+127 and 128 gates.  The MMA's row
// r' stands for coefficient m = m0 + 127 - r' (rows reversed), so element
// (r', t) of the A operand is R[t - m0 - 127 + r'] with R[y] = ext[-y]: a
// Hankel matrix, constant along anti-diagonals.  Shared memory holds, per
// plane, an array of 16-byte units where unit ui holds the eight elements
// R[ui - m0 - 127 .. ui - m0 - 120].  The 8x8 core matrix (row group g',
// column group kk) of the K-step at t0 is then the eight consecutive units
// starting at t0 + 8 (g' + kk): a K-major no-swizzle operand whose
// leading- and stride-dimension byte offsets are both 128, read straight
// from the unit array by the descriptor -- no per-tile copy of the matrix.
// The digits (B operand, gates x coefficients) are staged per 64-coefficient
// chunk with cp.async into core-matrix order, double buffered against the
// MMAs.  The four planes accumulate in four 128-column TMEM blocks (all 512
// columns); after each key polynomial every thread drains its own row
// (tcgen05.ld 32x32b) into integer sums.  Every wait on an mbarrier is
// bounded; on timeout the kernel records the fact and returns after
// releasing TMEM.
#include <cuda_bf16.h>

#include "mk_internal.h"

namespace mk {
namespace {

constexpr int T5_M = 128;       // output coefficients per CTA (TMEM lanes)
constexpr int T5_NG = 128;      // gates per CTA (MMA N)
constexpr int T5_KC = 64;       // coefficients per staged digit tile
constexpr int T5_STAGES = 4;    // digit tiles in flight: loads run two tiles ahead of the MMAs
constexpr int T5_THREADS = 128;
constexpr uint32_t T5_TMEM_COLS = 512;
constexpr uint32_t T5_WAIT_LIMIT = 1u << 26;

// Instruction descriptor, kind::f16: fp32 accumulator, bf16 A and B, both
// K-major, N = 128, M = 128.
constexpr uint32_t T5_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(T5_NG >> 3) << 17) |
                              ((uint32_t)(T5_M >> 4) << 24);

__device__ unsigned int g_tc05_error;  // nonzero: some wait of some CTA timed out

template <int LOGN>
struct T5Smem {
    static constexpr int N = 1 << LOGN;
    static constexpr int UNITS = N + 128;  // the K-steps read units [0, N + 120)
    static constexpr size_t plane_bytes = (size_t)UNITS * 16;
    static constexpr size_t stage_bytes = (size_t)T5_NG * T5_KC * 2;
    static constexpr size_t off_b = 4 * plane_bytes;
    static constexpr size_t off_key = off_b + T5_STAGES * stage_bytes;
    static constexpr size_t off_acc = off_key + (size_t)N * 4;  // integer sums [128 gates][128 rows]
    static constexpr size_t off_bar = off_acc + (size_t)T5_NG * T5_M * 4;  // T5_STAGES mbarriers, then the TMEM address
    static constexpr size_t used = off_bar + 8 * T5_STAGES + 16;
    // More than half of the SM's shared memory: one CTA per SM, so the 512
    // TMEM columns it allocates are always free.
    static constexpr size_t bytes = used < 120 * 1024 ? 120 * 1024 : used;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start, leading- and stride-dimension byte
// offsets (16-byte units), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t it = 0; it < T5_WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void mma_issue(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(T5_IDESC), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(g) : "memory");
}

// Grid (N / 128, G / 128, outputs), T5_THREADS threads.
template <int LOGN>
__global__ void __launch_bounds__(T5_THREADS, 1) tc05_products_kernel(TcArgs A, uint32_t G) {
    using L = T5Smem<LOGN>;
    constexpr int N = L::N, UNITS = L::UNITS;
    constexpr int KSTEPS = N / T5_KC;  // staged digit tiles per key polynomial
    extern __shared__ __align__(1024) unsigned char smem[];
    uint32_t *skey = reinterpret_cast<uint32_t *>(smem + L::off_key);
    uint32_t *sacc = reinterpret_cast<uint32_t *>(smem + L::off_acc);  // [gate][row]: row = tid, conflict-free
    const uint32_t bar0 = smem_addr(smem + L::off_bar);  // barrier of stage s at bar0 + 8 s
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + L::off_bar + 8 * T5_STAGES);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int type = blockIdx.z & 1, zi = blockIdx.z >> 1;
    const int m0 = blockIdx.x * T5_M;
    const uint32_t g0 = blockIdx.y * T5_NG;
    const uint32_t *keyz = type ? A.key[1] + zi * A.key_zstride[1] : A.key[0] + zi * A.key_zstride[0];
    const uint16_t *digz = A.dig + zi * A.dig_zstride + (size_t)g0 * N;
    const uint32_t a_base = smem_addr(smem), b_base = smem_addr(smem + L::off_b);

    if (tid == 0) {
        for (int q = 0; q < T5_STAGES; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar0 + 8 * q) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(tmem_slot)),
                     "r"(T5_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    for (int g = 0; g < T5_NG; ++g) sacc[g * T5_M + tid] = 0;
    bool ok = true;
    // Tile j (over all key polynomials) uses stage j % T5_STAGES; its MMAs
    // commit to that stage's barrier as the stage's (j / T5_STAGES)-th use.
    uint32_t j = 0;
    auto stage_bar = [&](uint32_t t) { return bar0 + 8 * (t % T5_STAGES); };
    auto wait_tile = [&](uint32_t t) { return mbar_wait(stage_bar(t), (t / T5_STAGES) & 1); };
    // digits of 128 gates x 64 coefficients into core-matrix order: core
    // (gate group ng, column group kg) at (ng * 8 + kg) * 128, row r at + r * 16
    auto load_tile = [&](const uint16_t *dig, int kc, uint32_t t) {
        const uint32_t sb = b_base + (t % T5_STAGES) * (uint32_t)L::stage_bytes;
        for (int q = tid; q < T5_NG * (T5_KC / 8); q += T5_THREADS) {
            const int gate = q >> 3, kg = q & 7;
            const uint32_t dst = sb + (uint32_t)(((gate >> 3) * 8 + kg) * 128 + (gate & 7) * 16);
            cp_async16(dst, dig + (size_t)gate * N + kc * T5_KC + kg * 8);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    for (int c = 0; c < A.nchunks && ok; ++c) {
        const uint32_t *key = keyz + (size_t)c * N;
        const uint16_t *dig = digz + (size_t)c * G * N;
        const uint32_t j0 = j;  // first tile of this key polynomial
        // start the first two digit tiles (their stages are free: every MMA
        // of the previous key polynomial has completed)
        load_tile(dig, 0, j0);
        load_tile(dig, 1, j0 + 1);
        // key words, then the four unit arrays: unit ui holds R_b[ui - m0 - 127 + e],
        // e = 0..7, with R_b[y] = ext_b[-y]
        for (int x = tid; x < N; x += T5_THREADS) skey[x] = key[x];
        __syncthreads();
        for (int ui = tid; ui < UNITS; ui += T5_THREADS) {
            uint32_t packed[4][4];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int x = m0 + 127 - ui - e;  // ext index
                uint32_t v = 0;
                bool neg = false;
                if (x >= 0 && x < N) v = skey[x];
                else if (x < 0 && x > -N) v = skey[x + N], neg = true;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int by = (int)(int8_t)(uint8_t)(v & 0xFFu);
                    v = (v - (uint32_t)by) >> 8;
                    const __nv_bfloat16 h = __int2bfloat16_rn(neg ? -by : by);
                    const uint32_t hb = (uint32_t)__bfloat16_as_ushort(h);
                    if (e & 1) packed[b][e >> 1] |= hb << 16;
                    else packed[b][e >> 1] = hb;
                }
            }
#pragma unroll
            for (int b = 0; b < 4; ++b)
                *reinterpret_cast<uint4 *>(smem + (size_t)b * L::plane_bytes + (size_t)ui * 16) =
                    make_uint4(packed[b][0], packed[b][1], packed[b][2], packed[b][3]);
        }

        for (int kc = 0; kc < KSTEPS; ++kc, ++j) {
            // tile j + 2 goes into the stage tile j - 2 used: its MMAs must be
            // done (for kc < 2 that stage held a tile of the previous key
            // polynomial, whose MMAs all completed before its drain)
            if (kc + 2 < KSTEPS) {
                if (kc >= 2 && !wait_tile(j - 2)) ok = false;
                if (__syncthreads_and(ok) == 0) {
                    ok = false;
                    break;
                }
                load_tile(dig, kc + 2, j + 2);
                asm volatile("cp.async.wait_group 2;\n" ::: "memory");  // tile j has landed
            } else if (kc + 1 < KSTEPS) {
                asm volatile("cp.async.wait_group 1;\n" ::: "memory");
            } else {
                asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t sb = b_base + (j % T5_STAGES) * (uint32_t)L::stage_bytes;
#pragma unroll
                for (int s = 0; s < T5_KC / 16; ++s) {
                    const int t0 = kc * T5_KC + s * 16;
                    const uint64_t bdesc = smem_desc(sb + (uint32_t)(2 * s * 128), 128, 8 * 128);
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const uint64_t adesc = smem_desc(a_base + (uint32_t)(b * L::plane_bytes + t0 * 16), 128, 128);
                        mma_issue(tmem + (uint32_t)(b * T5_NG), adesc, bdesc, (kc | s) ? 1u : 0u);
                    }
                }
                mma_commit(stage_bar(j));
            }
        }
        if (!ok) break;
        // the last two tiles' MMAs were not waited for above; the last commit
        // covers every earlier MMA of the key polynomial
        if (!wait_tile(j - 2) || !wait_tile(j - 1)) ok = false;
        if (__syncthreads_and(ok) == 0) {
            ok = false;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int q = 0; q < T5_NG / 32; ++q) {
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * T5_NG + q * 32), r);
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    sacc[(q * 32 + i) * T5_M + tid] += (uint32_t)__float2int_rn(__uint_as_float(r[i])) << (8 * b);
            }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();  // TMEM drained and units read: the next key polynomial may overwrite both
    }

    if (ok) {
        // row r' = tid holds coefficient m0 + 127 - tid of every gate
        int32_t *dst = (type ? A.dst[1] : A.dst[0]) + zi * A.dst_zstride;
        const int m = m0 + 127 - tid;
        for (int g = 0; g < T5_NG; ++g) {
            int32_t *d = dst + (size_t)(g0 + g) * A.dst_stride + m;
            const uint32_t v = sacc[g * T5_M + tid];
            *d = A.accumulate ? (int32_t)((uint32_t)*d + v) : (int32_t)v;
        }
    } else {
        asm volatile("cp.async.wait_all;\n" ::: "memory");  // no copy may land after the CTA exits
        if (tid == 0) {
            atomicCAS(&g_tc05_error, 0u, 1u + blockIdx.x + 1024u * blockIdx.y);
            // let MMAs still in flight finish before their TMEM goes away (bounded)
            mbar_wait(bar0, 0);
        }
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(T5_TMEM_COLS)
                     : "memory");
}

}  // namespace

template <int LOGN>
static cudaError_t launch_tc05(const TcArgs &A, uint32_t G, int outputs, cudaStream_t st) {
    constexpr int N = 1 << LOGN;
    if (G % T5_NG) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(tc05_products_kernel<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)T5Smem<LOGN>::bytes);
    if (e != cudaSuccess) return e;
    tc05_products_kernel<LOGN><<<dim3(N / T5_M, G / T5_NG, outputs), T5_THREADS, T5Smem<LOGN>::bytes, st>>>(A, G);
    return cudaGetLastError();
}

cudaError_t launch_products_tc05(const TcArgs &A, uint32_t N, uint32_t G, int outputs, cudaStream_t st) {
    if (N == 256) return launch_tc05<8>(A, G, outputs, st);
    if (N == 1024) return launch_tc05<10>(A, G, outputs, st);
    return cudaErrorInvalidValue;
}

cudaError_t tc05_error(unsigned int *code, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(code, g_tc05_error, sizeof(unsigned int));
    if (e == cudaSuccess && clear) {
        const unsigned int zero = 0;
        e = cudaMemcpyToSymbol(g_tc05_error, &zero, sizeof(unsigned int));
    }
    return e;
}

}  // namespace mk
