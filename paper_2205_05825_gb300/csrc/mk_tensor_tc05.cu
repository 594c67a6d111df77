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
// A work item is 128 output coefficients m0..m0+127 of 128 gates; one
// persistent CTA per SM loops over items.  The MMA's row
// r' stands for coefficient m = m0 + 127 - r' (rows reversed), so element
// (r', t) of the A operand is R[t - m0 - 127 + r'] with R[y] = ext[-y]: a
// Hankel matrix, constant along anti-diagonals.  Shared memory holds, per
// plane, an array of 16-byte units where unit ui holds the eight elements
// R[ui - m0 - 127 .. ui - m0 - 120].  The 8x8 core matrix (row group g',
// column group kk) of the K-step at t0 is then the eight consecutive units
// starting at t0 + 8 (g' + kk): a K-major no-swizzle operand whose
// leading- and stride-dimension byte offsets are both 128, read straight
// from the unit array by the descriptor -- no per-tile copy of the matrix.
// The digits (B operand, 128 gates x 64 coefficients per tile) arrive by TMA
// (a 3-D tiled tensor map over [chunk][gate][coefficient], 128-byte swizzle)
// into four stages: warp 5 produces tiles (expect-tx on the stage's full
// barrier, wait on its empty barrier), warp 4 issues the MMAs (wait full,
// commit empty) -- no block-wide barrier inside the K loop.  Each key
// polynomial is two passes over K, one per pair of byte planes, into the two
// 256-column halves of TMEM (plane b in columns 128 b .. 128 b + 127): while
// the MMAs of one pass run, warps 0-3 drain the other half (tcgen05.ld
// 32x32b, one row per thread, into integer sums) and build the unit arrays
// of the pass after, then signal it through that half's ready barrier.
// Every wait on an mbarrier is bounded in global time (TcArgs::wait_ns).  A
// wait that runs out sets the CTA's abort word; every role then leaves at its
// next wait (the other roles do not wait out their own limits), the producer
// waits for its copies still in flight and the MMA warp for its last commit
// (waits on the engine's own work, bounded but not cut short by the abort
// word), the CTA records the timeout and releases TMEM on every path.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "mk_internal.h"

namespace mk {
namespace {

constexpr int T5_M = 128;       // output coefficients per CTA (TMEM lanes)
constexpr int T5_NG = 128;      // gates per CTA (MMA N)
constexpr int T5_KC = 64;       // coefficients per staged digit tile
constexpr int T5_STAGES = 4;    // digit tiles in flight: loads run two tiles ahead of the MMAs
constexpr int T5_WORKERS = 128;               // warps 0-3: TMEM drain (one row each), unit arrays, planes
constexpr int T5_THREADS = T5_WORKERS + 64;   // + warp 4 (MMA issue) + warp 5 (TMA producer)
constexpr uint32_t T5_TMEM_COLS = 512;
constexpr uint32_t T5_SPIN_LIMIT = 1u << 30;        // backstop on the polls of one wait
constexpr uint64_t T5_DRAIN_NS = 1000000000ull;      // bound on waits for the CTA's own copies and MMAs

// Instruction descriptor, kind::f16: fp32 accumulator, bf16 A and B, both
// K-major, N = 128, M = 128.
constexpr uint32_t T5_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(T5_NG >> 3) << 17) |
                              ((uint32_t)(T5_M >> 4) << 24);

__device__ unsigned int g_tc05_error;  // nonzero: some wait of some CTA timed out
// Test hook, one shot: 1 + the index (within its CTA) of one digit-tile load
// that the first producer reaching it does not issue; 0: none.
__device__ unsigned int g_tc05_skip;

template <int LOGN>
struct T5Smem {
    static constexpr int N = 1 << LOGN;
    static constexpr int UNITS = N + 128;  // the K-steps read units [0, N + 120)
    static constexpr int RLEN = UNITS + 8;  // R elements a plane's units cover (+ slack)
    static constexpr size_t plane_bytes = (size_t)UNITS * 16;
    static constexpr size_t stage_bytes = (size_t)T5_NG * T5_KC * 2;  // one TMA tile, 1024-byte aligned
    // offsets from the 1024-byte aligned base
    static constexpr size_t off_b = 0;
    static constexpr size_t off_a = off_b + T5_STAGES * stage_bytes;
    static constexpr size_t off_r = off_a + 4 * plane_bytes;              // [4 planes][2 copies][RLEN] bf16
    static constexpr size_t off_acc = off_r + (size_t)4 * 2 * RLEN * 2;  // integer sums [128 gates][128 rows]
    static constexpr size_t off_bar = off_acc + (size_t)T5_NG * T5_M * 4;  // mbarriers, then the TMEM address
    static constexpr int NBARS = 2 * T5_STAGES + 5;  // full[S], empty[S], done[2], ready[2], fin
    static constexpr size_t off_abort = off_bar + 8 * NBARS + 4;  // after the TMEM address word
    static constexpr size_t used = off_bar + 8 * NBARS + 8;
    // + 1 KB to align the base; more than half of the SM: one CTA per SM,
    // so the 512 TMEM columns it allocates are always free
    static constexpr size_t bytes = used + 1024 < 120 * 1024 ? 120 * 1024 : used + 1024;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start, leading- and stride-dimension byte
// offsets (16-byte units), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// K-major, 128-byte swizzle (TMA's CU_TENSOR_MAP_SWIZZLE_128B layout): rows
// of 128 bytes, 8-row atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// Wait for the phase of parity `parity` of `bar`, at most wait_ns of global
// time.  With an abort word: give up as soon as it is set, and set it on a
// timeout (so the CTA's other roles give up too); without one (waits on the
// CTA's own copies and MMAs, which complete by themselves): only the bound.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t wait_ns, volatile uint32_t *abort) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 0; it < T5_SPIN_LIMIT; ++it) {
        if (mbar_try(bar, parity)) return true;
        if (abort && *abort) return false;
        if (globaltimer() - t0 > wait_ns) break;
    }
    if (abort) *abort = 1;
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

__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// The four byte planes of R_b[y] = ext_b[-y] for y = i - m0 - 127, i in
// [0, RLEN), each in two copies one element apart (copy 1 holds element
// i + 1 at i), so that any eight consecutive elements are four aligned
// 32-bit words of one copy.  Threads [t0, t0 + nt) of the CTA take part.
template <int LOGN>
__device__ __forceinline__ void build_planes(const uint32_t *__restrict__ key, int m0, uint16_t *rpl, int t, int nt) {
    using L = T5Smem<LOGN>;
    constexpr int N = L::N;
    for (int i = t; i < L::RLEN; i += nt) {
        const int x = m0 + 127 - i;  // ext index
        uint32_t v = 0;
        bool neg = false;
        if (x >= 0 && x < N) v = __ldg(key + x);
        else if (x < 0 && x > -N) v = __ldg(key + x + N), neg = true;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int by = (int)(int8_t)(uint8_t)(v & 0xFFu);
            v = (v - (uint32_t)by) >> 8;
            const uint16_t hb = __bfloat16_as_ushort(__int2bfloat16_rn(neg ? -by : by));
            rpl[(2 * b) * L::RLEN + i] = hb;
            if (i > 0) rpl[(2 * b + 1) * L::RLEN + i - 1] = hb;
        }
    }
}

// Unit ui of plane b = R_b elements [ui, ui + 8), for planes b0 and b0 + 1,
// by the worker threads.
template <int LOGN>
__device__ __forceinline__ void build_units(unsigned char *a, const uint16_t *rpl, int b0, int t) {
    using L = T5Smem<LOGN>;
    for (int ui = t; ui < L::UNITS; ui += T5_WORKERS) {
        const int cp = ui & 1;
        const int w0 = (ui - cp) >> 1;  // first word of the window in copy cp
#pragma unroll
        for (int b = b0; b < b0 + 2; ++b) {
            const uint32_t *wp = reinterpret_cast<const uint32_t *>(rpl + (2 * b + cp) * L::RLEN) + w0;
            *reinterpret_cast<uint4 *>(a + (size_t)b * L::plane_bytes + (size_t)ui * 16) =
                make_uint4(wp[0], wp[1], wp[2], wp[3]);
        }
    }
}

__device__ __forceinline__ void workers_sync() { asm volatile("bar.sync 1, %0;\n" ::"n"(T5_WORKERS) : "memory"); }

// Barrier of the worker warps that also ANDs their flags, so that all of them
// take the same branch after a bounded wait.
__device__ __forceinline__ bool workers_all(bool ok) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)ok), "n"(T5_WORKERS)
        : "memory");
    return r != 0;
}

// One work item: 128 output coefficients (m-tile) x 128 gates (g-tile) of
// one output; m-tiles vary fastest so that CTAs running at the same time
// share digit tiles in L2.
struct T5Item {
    int m0;
    uint32_t g0;
    int chunk0;  // first digit polynomial of the output in the tensor map
    int type;
    int zi;
    const uint32_t *key;  // key polynomial 0 of the output
};

template <int LOGN>
__device__ __forceinline__ T5Item item_of(const TcArgs &A, uint32_t G, int it) {
    constexpr int N = 1 << LOGN, MT = N / T5_M;
    const int GT = (int)(G / T5_NG);
    T5Item r;
    r.m0 = (it % MT) * T5_M;
    const int rest = it / MT;
    r.g0 = (uint32_t)(rest % GT) * T5_NG;
    const int z = rest / GT;
    r.type = z & 1;
    r.zi = z >> 1;
    r.chunk0 = (int)(r.zi * (A.dig_zstride / ((size_t)G * N)));
    r.key = r.type ? A.key[1] + r.zi * A.key_zstride[1] : A.key[0] + r.zi * A.key_zstride[0];
    return r;
}

// Persistent: grid min(items, SMs), T5_THREADS threads; CTA b takes items
// b, b + gridDim.x, ...  Its passes form one sequence gp = 0, 1, ...: pass
// gp belongs to item gp / (2 nchunks) of the CTA, key polynomial
// (gp / 2) % nchunks, planes 2 (gp % 2) and 2 (gp % 2) + 1, TMEM half gp % 2,
// so the prologue and the last drain of an item overlap the MMAs of its
// neighbours.  dmap: the digits as a [chunks][G][N] bf16 tensor, tile box
// 64 x 128 x 1, 128-byte swizzle.
template <int LOGN>
__global__ void __launch_bounds__(T5_THREADS, 1)
    tc05_products_kernel(TcArgs A, uint32_t G, int items, const __grid_constant__ CUtensorMap dmap) {
    using L = T5Smem<LOGN>;
    constexpr int N = L::N;
    constexpr int KSTEPS = N / T5_KC;  // digit tiles per key polynomial
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024 - (smem_addr(smem_raw) & 1023)) & 1023);
    uint16_t *rpl = reinterpret_cast<uint16_t *>(smem + L::off_r);      // plane b, copy c at (2 b + c) * RLEN
    uint32_t *sacc = reinterpret_cast<uint32_t *>(smem + L::off_acc);  // [gate][row]: row = tid, conflict-free
    const uint32_t full0 = smem_addr(smem + L::off_bar);  // full[s] = full0 + 8 s
    const uint32_t empty0 = full0 + 8 * T5_STAGES;        // empty[s] = empty0 + 8 s
    const uint32_t done0 = empty0 + 8 * T5_STAGES;        // done[h]: every MMA of a pass on half h
    const uint32_t ready0 = done0 + 16;                   // ready[h]: half h drained, the units of its next pass built
    const uint32_t fin = ready0 + 16;                     // the MMA warp's last commit
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + L::off_bar + 8 * L::NBARS);
    volatile uint32_t *abort = reinterpret_cast<volatile uint32_t *>(smem + L::off_abort);
    const uint64_t wait_ns = A.wait_ns;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nch = A.nchunks, PI = 2 * nch;  // passes per item
    const int my_items = (items - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    const int PT = my_items * PI;             // passes of this CTA
    unsigned char *abuf = smem + L::off_a;
    const uint32_t a_base = smem_addr(abuf), b_base = smem_addr(smem + L::off_b);

    if (tid == 0) {
        for (int q = 0; q < 2 * T5_STAGES + 2; ++q)  // full, empty, done
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(full0 + 8 * q) : "memory");
        for (int h = 0; h < 2; ++h)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(ready0 + 8 * h), "n"(T5_WORKERS) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(fin) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        *abort = 0;
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
    bool ok = true;

    if (warp == 5) {
        // producer: tile j = gp * KSTEPS + kc into stage j % S once the MMAs
        // of tile j - S (same stage) have committed
        uint32_t issued = 0, skipped = 0xFFFFFFFFu;
        for (int gp = 0; gp < PT && ok; ++gp) {
            const T5Item I = item_of<LOGN>(A, G, (int)blockIdx.x + (gp / PI) * (int)gridDim.x);
            const int c = (gp >> 1) % nch;
            for (int kc = 0; kc < KSTEPS; ++kc) {
                const uint32_t j = (uint32_t)(gp * KSTEPS + kc), st = j % T5_STAGES;
                if (j >= T5_STAGES && !mbar_wait(empty0 + 8 * st, ((j / T5_STAGES) - 1) & 1, wait_ns, abort))
                    ok = false;
                if (!__all_sync(0xFFFFFFFFu, ok)) {
                    ok = false;
                    break;
                }
                if (lane == 0) {
                    if (g_tc05_skip == j + 1 && atomicCAS(&g_tc05_skip, j + 1, 0u) == j + 1) {
                        skipped = j;  // test hook: this tile's copy is never issued
                    } else {
                        mbar_expect_tx(full0 + 8 * st, (uint32_t)L::stage_bytes);
                        tma_load_3d(b_base + st * (uint32_t)L::stage_bytes, &dmap, kc * T5_KC, (int)I.g0,
                                    I.chunk0 + c, full0 + 8 * st);
                    }
                }
                issued = j + 1;
                __syncwarp();
            }
        }
        // every copy issued has landed before shared memory can be released
        // (in the normal course the MMAs consumed them all; a stage's newest
        // tile is the only one of it that can still be in flight)
        if (lane == 0)
            for (uint32_t j = issued > T5_STAGES ? issued - T5_STAGES : 0; j < issued; ++j)
                if (j != skipped) mbar_wait(full0 + 8 * (j % T5_STAGES), (j / T5_STAGES) & 1, T5_DRAIN_NS, nullptr);
        __syncwarp();
    } else if (warp == 4) {
        // MMA issuer: pass gp starts once its TMEM half is drained and its
        // unit arrays are built (ready), then follows the digit tiles (full)
        const uint64_t adesc0 = smem_desc(a_base, 128, 128);
        for (int gp = 0; gp < PT && ok; ++gp) {
            const int h = gp & 1;
            if (!mbar_wait(ready0 + 8 * h, (gp >> 1) & 1, wait_ns, abort)) ok = false;
            if (!__all_sync(0xFFFFFFFFu, ok)) {
                ok = false;
                break;
            }
            for (int kc = 0; kc < KSTEPS; ++kc) {
                const uint32_t j = (uint32_t)(gp * KSTEPS + kc), st = j % T5_STAGES;
                if (!mbar_wait(full0 + 8 * st, (j / T5_STAGES) & 1, wait_ns, abort)) ok = false;
                if (!__all_sync(0xFFFFFFFFu, ok)) {
                    ok = false;
                    break;
                }
                if (lane == 0) {
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const uint64_t bdesc0 = smem_desc_sw128(b_base + st * (uint32_t)L::stage_bytes);
#pragma unroll
                    for (int s4 = 0; s4 < T5_KC / 16; ++s4) {
                        const int t0 = kc * T5_KC + s4 * 16;
                        const uint64_t bdesc = bdesc0 + (uint64_t)(s4 * 32 / 16);  // 32 bytes per K-step of 16
#pragma unroll
                        for (int bb = 0; bb < 2; ++bb) {
                            const int b = 2 * h + bb;
                            const uint64_t adesc = adesc0 + (uint64_t)((b * L::plane_bytes + t0 * 16) / 16);
                            mma_issue(tmem + (uint32_t)(b * T5_NG), adesc, bdesc, (kc | s4) ? 1u : 0u);
                        }
                    }
                    mma_commit(empty0 + 8 * st);
                }
                __syncwarp();
            }
            if (!ok) break;
            if (lane == 0) mma_commit(done0 + 8 * h);  // every MMA of pass gp
            __syncwarp();
        }
        // no MMA of this CTA is in flight past this point (the commit arrives
        // once every earlier MMA of this thread has completed)
        if (lane == 0) {
            mma_commit(fin);
            mbar_wait(fin, 0, T5_DRAIN_NS, nullptr);
        }
        __syncwarp();
    } else {
        // workers.  Prologue: the unit arrays of passes 0 and 1.  Step gp:
        // once pass gp - 1 has completed, drain its half into the integer
        // sums (and write the outputs of its item after its last pass); then
        // build the units of pass gp + 1 (same half: its previous MMAs were
        // pass gp - 1) and release it.  The planes of key polynomial s + 1
        // (s = gp / 2 counts the CTA's key polynomials) are built once both
        // halves of polynomial s have their units.
        {
            const T5Item I = item_of<LOGN>(A, G, (int)blockIdx.x);
            build_planes<LOGN>(I.key, I.m0, rpl, tid, T5_WORKERS);
            workers_sync();
            for (int h = 0; h < 2 && h < PT; ++h) {
                build_units<LOGN>(abuf, rpl, 2 * h, tid);
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(ready0 + 8 * h) : "memory");
            }
        }
        for (int gp = 0; gp <= PT; ++gp) {
            if (gp >= 1) {
                const int pp = gp - 1, hp = pp & 1, lp = pp % PI;  // the drained pass, its half, its index in the item
                ok = workers_all(mbar_wait(done0 + 8 * hp, (pp >> 1) & 1, wait_ns, abort));
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll 1
                for (int q = 0; q < T5_NG / 32; ++q) {  // gates 32 q .. 32 q + 31, planes 2 hp and 2 hp + 1
                    uint32_t r0[32], r1[32];
                    const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(2 * hp * T5_NG + q * 32);
                    tmem_ld32_nowait(ta, r0);
                    tmem_ld32_nowait(ta + T5_NG, r1);
                    tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const uint32_t v = ((uint32_t)__float2int_rn(__uint_as_float(r0[i])) +
                                            ((uint32_t)__float2int_rn(__uint_as_float(r1[i])) << 8))
                                           << (16 * hp);
                        uint32_t &a = sacc[(q * 32 + i) * T5_M + tid];
                        a = lp == 0 ? v : a + v;
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                if (lp == PI - 1) {
                    // row r' = tid holds coefficient m0 + 127 - tid of every gate
                    const T5Item I = item_of<LOGN>(A, G, (int)blockIdx.x + (pp / PI) * (int)gridDim.x);
                    int32_t *dst = (I.type ? A.dst[1] : A.dst[0]) + I.zi * A.dst_zstride + (I.m0 + 127 - tid) +
                                   (size_t)I.g0 * A.dst_stride;
#pragma unroll 1
                    for (int g = 0; g < T5_NG; g += 16) {
                        uint32_t old[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            old[i] = A.accumulate ? (uint32_t)dst[(size_t)(g + i) * A.dst_stride] : 0u;
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            dst[(size_t)(g + i) * A.dst_stride] = (int32_t)(old[i] + sacc[(g + i) * T5_M + tid]);
                    }
                }
            }
            const int q = gp + 1, s = q >> 1, hq = q & 1;
            if (q >= 2 && q < PT) {
                workers_sync();  // the planes of key polynomial s are complete
                build_units<LOGN>(abuf, rpl, 2 * hq, tid);
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(ready0 + 8 * hq) : "memory");
            }
            if (hq == 1 && 2 * (s + 1) < PT) {
                workers_sync();  // every unit of key polynomial s is built: the planes may be replaced
                const T5Item I = item_of<LOGN>(A, G, (int)blockIdx.x + ((s + 1) / nch) * (int)gridDim.x);
                build_planes<LOGN>(I.key + (size_t)((s + 1) % nch) * N, I.m0, rpl, tid, T5_WORKERS);
            }
        }
    }
    if (!__syncthreads_and(ok) && tid == 0) atomicCAS(&g_tc05_error, 0u, 1u + blockIdx.x);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(T5_TMEM_COLS)
                     : "memory");
}

}  // namespace

namespace {
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}
}  // namespace

template <int LOGN>
static cudaError_t launch_tc05(const TcArgs &A, uint32_t G, int outputs, cudaStream_t st) {
    constexpr int N = 1 << LOGN;
    if (G % T5_NG || A.dig_chunks <= 0) return cudaErrorInvalidValue;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    // digits: [dig_chunks][G][N] bf16; a box of 64 coefficients x 128 gates x 1 polynomial
    CUtensorMap map;
    const cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)G, (cuuint64_t)A.dig_chunks};
    const cuuint64_t strides[2] = {(cuuint64_t)N * 2, (cuuint64_t)G * N * 2};
    const cuuint32_t box[3] = {(cuuint32_t)T5_KC, (cuuint32_t)T5_NG, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<uint16_t *>(A.dig), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(tc05_products_kernel<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)T5Smem<LOGN>::bytes);
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // one CTA per SM (its shared memory and TMEM take the SM), each looping over items
    const int items = (N / T5_M) * (int)(G / T5_NG) * outputs;
    const int grid = items < sms ? items : sms;
    tc05_products_kernel<LOGN><<<grid, T5_THREADS, T5Smem<LOGN>::bytes, st>>>(A, G, items, map);
    return cudaGetLastError();
}

cudaError_t launch_products_tc05(const TcArgs &A, uint32_t N, uint32_t G, int outputs, cudaStream_t st) {
    if (N == 256) return launch_tc05<8>(A, G, outputs, st);
    if (N == 1024) return launch_tc05<10>(A, G, outputs, st);
    return cudaErrorInvalidValue;
}

cudaError_t tc05_arm_skip(uint32_t tile_plus_one) {
    return cudaMemcpyToSymbol(g_tc05_skip, &tile_plus_one, sizeof(tile_plus_one));
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
