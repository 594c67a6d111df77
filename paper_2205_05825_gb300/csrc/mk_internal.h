// Internal interface between the host runtime (mk_host.cpp) and the CUDA
// kernels (mk_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "../../include/mk_tfhe.h"

namespace mk {

// Goldilocks prime 2^64 - 2^32 + 1: the NTT modulus of the exact product form
// MK_FORM_NTT.
constexpr uint64_t kGoldilocks = 0xFFFFFFFF00000001ull;
// The two 28-bit primes of MK_FORM_NTT2 (both = 1 mod 8192): residues mod p1
// and p2, recombined by CRT.  p1 p2 = 7.20e16 exceeds twice the largest
// product sum of any supported parameter set, (k+1) d N 2^(bg_bit-1) 2^31
// <= 9 * 3 * 1024 * 2^9 * 2^31 = 3.04e16 (k <= 8, bg_bit <= 10, N <= 1024,
// keys as signed 32-bit values).
constexpr uint32_t kP1 = 268369921u;  // 0x0fff0001
constexpr uint32_t kP2 = 268361729u;  // 0x0ffee001

// Per-gate record consumed by the fused linear + blind-rotation kernel.
struct GateDesc {
    uint32_t ia, ib;   // row indices into the a / b ciphertext arrays
    uint32_t cst;      // torus constant of the linear part
    int32_t s1, s2;    // integer scalars of the linear part
    uint32_t out;      // row index of the output ciphertext
};

// Device-resident key material of one context, in the layouts the kernels read.
// Element type of the NTT-domain arrays by form: MK_FORM_NTT uint64 (mod
// Goldilocks); MK_FORM_NTT2 uint2 (residues mod kP1, kP2, Montgomery form);
// MK_FORM_FFT double2 (N/2 folded complex points, times 2/N).
// Twiddle entries: uint64 (NTT) or uint4 {w1, w2, w1', w2'} with Shoup
// companions w' = floor(w * 2^32 / p) (NTT2).
struct DeviceKeys {
    const void *tw_fwd;   // [N] psi^bitrev(m); FFT form: [3][N/2] forward, inverse, twist
    const void *tw_inv;   // [N] psi^-bitrev(m)
    const void *bk;       // [k][n][3][d][N] NTT domain, bit-reversed order, times N^-1
    const void *keyA;     // [(k+1)][d][N]: [0] = NTT(-a), [j] = NTT(pk_j), times N^-1
    const uint32_t *ks;   // [k][N][t][B'-1][n+1] torus32
    // MK_FORM_TC: bk and keyA hold torus32 words in the same order ([0] = -a);
    // the wave workspace holds tc_ws_gates gates (a multiple of 64).
    void *tc_ws;
    uint32_t tc_ws_gates;
    // The context's status word (device): a kernel whose bounded wait ran out
    // sets its bit (kStatusStaged, kStatusNetlist, kStatusCluster); mk_sync reports it as
    // MK_ETIMEOUT and clears it.
    uint32_t *status;
    // MK_FORM_NTT2: per-prime twiddles [2 directions][2 primes][N] uint2
    // {w, w'} for the split-prime kernel (nullptr for the other forms).
    const void *tw_split;
};

constexpr uint32_t kStatusStaged = 1u, kStatusNetlist = 2u, kStatusCluster = 4u;

struct LaunchShape {
    uint32_t n, N, logN, k, d, bg_bit, ks_bit, t;
    int variant;  // blind-rotation variant (see kVariantNpf)
    int form;     // MK_FORM_*
    // Batches of at most this many gates run the cluster (latency) kernel of
    // the NTT forms: one CTA per accumulator polynomial (0: never).
    uint32_t cluster_max;
    // Bound on each wait of the staged kernel for a key copy, in ns of global
    // time, and a test hook: the key copies of this CMux step are never
    // issued, so the waits for them run out (-1: none).
    uint64_t wait_ns;
    int64_t skip_key_step;
};

// Clusters of the latency form that fit on the device at once for this
// shape (NTT forms, k + 1 <= 8), or 0.
int cluster_capacity(const LaunchShape &S);

// a1-a8: linear part, window shift, modulus switch, blind rotation (NTT form),
// SampleExtract, +1/8.  ext: [count][k*N + 1].  If abar_out != nullptr the
// kernel stops after the modulus switch and writes it there instead.
cudaError_t launch_bootstrap_ntt(const LaunchShape &S, const DeviceKeys &K, const GateDesc *desc,
                                 const uint32_t *ct_a, const uint32_t *ct_b, uint32_t *ext,
                                 uint32_t count, cudaStream_t st);

// Mod switch only (stage output).
cudaError_t launch_modswitch(const LaunchShape &S, const GateDesc *desc, const uint32_t *ct_a,
                             const uint32_t *ct_b, uint32_t *abar, uint32_t count, cudaStream_t st);

// Blind rotation from precomputed abar with a step limit (stage output).
cudaError_t launch_blind_rotate_ntt(const LaunchShape &S, const DeviceKeys &K, const uint32_t *abar,
                                    uint32_t count, int64_t max_steps, uint32_t *acc,
                                    cudaStream_t st);

// Blind-rotation variants: digit polynomials per forward transform (1 or 3),
// the minimum resident CTAs per SM the register allocation is capped for,
// where the twiddles live (0: a shared-memory copy per CTA, 1: global memory
// through the read-only cache), and the elements each thread holds per
// polynomial (8: N/8 threads per gate, three stages per register pass; 4:
// N/4 threads, two stages per pass, fewer registers per thread).  Kinds:
// 0 gives each gate its own CTA (mk_bootstrap.cuh); 1 is the staged kernel
// (mk_bootstrap_staged.cuh: G gates per CTA share each step's key entry,
// bulk-copied into shared memory once); 2 is the split-prime kernel
// (mk_bootstrap_split.cuh, MK_FORM_NTT2: one half of a gate's threads per
// prime; MK_FORM_NTT runs variant 2's kernel for these numbers).  All give
// identical results.
constexpr int kNumVariants = 9;
constexpr int kVariantNpf[kNumVariants] = {3, 1, 3, 3, 3, 3, 3, 3, 3};
constexpr int kVariantMinBlocks[kNumVariants] = {3, 4, 3, 4, 2, 3, 1, 2, 3};
constexpr int kVariantTwg[kNumVariants] = {0, 1, 1, 1, 1, 1, 1, 1, 1};
constexpr int kVariantEpt[kNumVariants] = {8, 8, 8, 8, 4, 4, 8, 8, 8};
constexpr int kVariantKind[kNumVariants] = {0, 0, 0, 0, 0, 0, 1, 2, 2};
static_assert(kNumVariants == MK_NUM_VARIANTS, "variant count of the ABI");

// Per-(ring dimension, variant) blind-rotation launchers, one translation unit
// each (mk_br.cu built with -DMK_LOGN -DMK_VARIANT).  abar_in == nullptr: the
// gate's linear part and modulus switch come from desc/ct_a/ct_b;
// acc_out == nullptr: the extracted LWE goes to ext, otherwise the raw
// accumulator to acc_out.
#define MK_DECLARE_BOOTSTRAP(LOGN, F, V)                                                                      \
    cudaError_t launch_bootstrap_logn##LOGN##_f##F##_v##V(const LaunchShape &S, const DeviceKeys &K,           \
                                                          const GateDesc *desc, const uint32_t *ct_a,         \
                                                          const uint32_t *ct_b, const uint32_t *abar_in,      \
                                                          int64_t max_steps, uint32_t *ext, uint32_t *acc_out, \
                                                          uint32_t count, cudaStream_t st);
#define MK_DECLARE_BOOTSTRAP_F(LOGN, F)                                                                       \
    MK_DECLARE_BOOTSTRAP(LOGN, F, 0) MK_DECLARE_BOOTSTRAP(LOGN, F, 1) MK_DECLARE_BOOTSTRAP(LOGN, F, 2)          \
    MK_DECLARE_BOOTSTRAP(LOGN, F, 3) MK_DECLARE_BOOTSTRAP(LOGN, F, 4) MK_DECLARE_BOOTSTRAP(LOGN, F, 5)          \
    MK_DECLARE_BOOTSTRAP(LOGN, F, 6) MK_DECLARE_BOOTSTRAP(LOGN, F, 7) MK_DECLARE_BOOTSTRAP(LOGN, F, 8)
MK_DECLARE_BOOTSTRAP_F(8, 0)
MK_DECLARE_BOOTSTRAP_F(8, 1)
MK_DECLARE_BOOTSTRAP_F(10, 0)
MK_DECLARE_BOOTSTRAP_F(10, 1)
MK_DECLARE_BOOTSTRAP(8, 2, 0)
MK_DECLARE_BOOTSTRAP(10, 2, 0)

// Cluster (latency) form of the NTT blind rotation, one translation unit per
// (ring dimension, field): mk_brc.cu built with -DMK_LOGN -DMK_FIELD.  Same
// arguments as the launchers above; needs k + 1 <= 8.  cluster_capacity_*:
// the clusters of k + 1 CTAs that fit on the device at once (0: none).
#define MK_DECLARE_CLUSTER(LOGN, F)                                                                            \
    cudaError_t launch_cluster_logn##LOGN##_f##F(const LaunchShape &S, const DeviceKeys &K, const GateDesc *desc, \
                                                 const uint32_t *ct_a, const uint32_t *ct_b,                    \
                                                 const uint32_t *abar_in, int64_t max_steps, uint32_t *ext,     \
                                                 uint32_t *acc_out, uint32_t count, cudaStream_t st);          \
    int cluster_capacity_logn##LOGN##_f##F(uint32_t k, uint32_t n);
MK_DECLARE_CLUSTER(8, 0)
MK_DECLARE_CLUSTER(8, 1)
MK_DECLARE_CLUSTER(10, 0)
MK_DECLARE_CLUSTER(10, 1)

// A whole operator netlist in one persistent launch (mk_netlist.cuh): every
// (gate, pair) item of the plan, taken by CTAs in topological order, each
// waiting for its input rows to be marked ready.  NTT forms only; built in
// the variant-2 translation unit of each (ring dimension, field).
struct NetlistArgs {
    const GateDesc *desc;  // items in topological order; ia, ib, out are pool rows
    uint32_t count;        // items
    uint32_t *pool;        // [rows][k n + 1] ciphertext rows
    uint32_t input_rows;   // rows below this (inputs and constants) are ready from the start
    uint32_t *ready;       // [rows]: the epoch of the call that wrote the row
    uint32_t epoch;        // this call's epoch (never 0)
    uint32_t *next;        // item counter (0 at launch)
    uint32_t *abort;       // set when some wait ran out (0 at launch)
    uint32_t *done;        // items finished (0 at launch): the progress the waits watch
    int64_t skip_item;     // test hook: this item never marks its output ready (-1: none)
};
#define MK_DECLARE_NETLIST(LOGN, F)                                                                          \
    cudaError_t launch_netlist_logn##LOGN##_f##F(const LaunchShape &S, const DeviceKeys &K, const NetlistArgs &A, \
                                                 uint32_t sm_count, cudaStream_t st);
MK_DECLARE_NETLIST(8, 0)
MK_DECLARE_NETLIST(8, 1)
MK_DECLARE_NETLIST(10, 0)
MK_DECLARE_NETLIST(10, 1)
cudaError_t launch_netlist(const LaunchShape &S, const DeviceKeys &K, const NetlistArgs &A, uint32_t sm_count,
                           cudaStream_t st);

// MK_FORM_TC (mk_tensor.cu): the blind rotation of a batch as a wave of
// tensor-core Toeplitz products.  Same arguments as the launchers above;
// count is processed in waves of K.tc_ws_gates gates.
cudaError_t launch_bootstrap_tc(const LaunchShape &S, const DeviceKeys &K, const GateDesc *desc, const uint32_t *ct_a,
                                const uint32_t *ct_b, const uint32_t *abar_in, int64_t max_steps, uint32_t *ext,
                                uint32_t *acc_out, uint32_t count, cudaStream_t st);
bool tc_shape_supported(const LaunchShape &S);
// One launch of a Toeplitz product kernel of the tensor form: output z
// (0 <= z < outputs) is dst[type] + (z >> 1) * dst_zstride (row g at
// g * dst_stride words), type = z & 1, the sum over nchunks products of
// key[type] + (z >> 1) * key_zstride[type] + c * N (torus32 words) with the
// digits dig + (z >> 1) * dig_zstride + c * G * N ([G][N] bf16 bit patterns).
struct TcArgs {
    int32_t *dst[2];
    size_t dst_zstride;
    uint32_t dst_stride;
    int accumulate;
    const uint32_t *key[2];
    size_t key_zstride[2];
    const uint16_t *dig;
    size_t dig_zstride;
    int nchunks;
    int dig_chunks;  // digit polynomials in the whole dig array (for the tcgen05 engine's tensor map)
    uint64_t wait_ns;  // bound on each mbarrier wait of the tcgen05 engine (global time)
};
// The tcgen05 engine of those products (mk_tensor_tc05.cu): G a multiple of
// 128; one persistent CTA per SM over (coefficient tile, gate tile, output)
// items of 128 x 128.  tc05_error reads (and optionally clears) the timeout record of its
// bounded waits (0: none).
cudaError_t launch_products_tc05(const TcArgs &A, uint32_t N, uint32_t G, int outputs, cudaStream_t st);
cudaError_t tc05_error(unsigned int *code, bool clear);
// Test hook: the next launch's first producer reaching its digit tile
// tile_plus_one - 1 skips that tile's copy (0 disarms).
cudaError_t tc05_arm_skip(uint32_t tile_plus_one);
constexpr uint32_t kTcWaveGates = 4096;  // gates per wave of the context's workspace
size_t tc_workspace_bytes(const LaunchShape &S, uint32_t gates);
uint32_t tc_wave_granularity();
// out[g] = sum_c keys[c] * digits[c][g] (negacyclic, mod 2^32); work holds
// nchunks * G * N bf16.
cudaError_t launch_negacyclic_tc(uint32_t N, uint32_t G, uint32_t nchunks, const uint32_t *keys, const int8_t *digits,
                                 int32_t *out, void *work, int engine, cudaStream_t st);
// Register-resident bf16 m16n8k16 MMA loop: 8 MMAs per warp and iteration.
cudaError_t launch_mma_peak(uint32_t blocks, uint32_t threads, uint32_t iters, float *sink, cudaStream_t st);

// a9: per-party key switch of ext [count][k*N+1] into out rows desc[g].out
// (or row g when desc == nullptr).  From kKeyswitchBatchMin gates on (and for
// 2-bit digits) a CTA serves a group of gates from each key row it reads.
constexpr uint32_t kKeyswitchBatchMin = 64;
cudaError_t launch_keyswitch(const LaunchShape &S, const DeviceKeys &K, const GateDesc *desc,
                             const uint32_t *ext, uint32_t *out, uint32_t count, cudaStream_t st);

// Eq. 8: out = (0, 1/4) - in.
cudaError_t launch_not(const LaunchShape &S, const uint32_t *in, uint32_t *out, size_t count,
                       cudaStream_t st);

// Build GateDesc records on the device from gate types (uint8) or mk_lin.
cudaError_t launch_desc_from_types(const uint8_t *types, GateDesc *desc, uint32_t base,
                                   uint32_t count, cudaStream_t st);
cudaError_t launch_desc_from_lin(const mk_lin *lin, GateDesc *desc, uint32_t base, uint32_t count,
                                 cudaStream_t st);
cudaError_t launch_desc_uniform(int type, GateDesc *desc, uint32_t base, uint32_t count, cudaStream_t st);

// Fixed device scratch of mk_gates_noalloc (mk_noalloc.cu): its size, and
// the device address on `device` (current), looked up on first use per device.
constexpr size_t kNoAllocScratchBytes = MK_NOALLOC_SCRATCH_BYTES;
cudaError_t noalloc_scratch(int device, void **ptr);

// ------------------------------------------------------------ circuits
struct Wire {
    int32_t w;
    int neg;
};
struct Netlist {
    uint32_t ka = 0, kb = 0;
    std::vector<mk_gate_rec> gates;
    std::vector<Wire> outputs;
};
bool build_netlist(int op, uint32_t k, int style, Netlist &out);
mk_lin gate_lin(const mk_gate_rec &g);
std::vector<uint32_t> netlist_levels(const Netlist &net);

// Wire buffer helpers: rows are ciphertexts of W words, wire w of pair p at row w*P + p.
cudaError_t launch_circuit_consts(uint32_t *pool, uint32_t P, uint32_t W, cudaStream_t st);
cudaError_t launch_circuit_inputs(uint32_t *pool, const uint32_t *src, uint32_t kbits, uint32_t P, uint32_t wire0,
                                  uint32_t W, cudaStream_t st);
cudaError_t launch_circuit_outputs(uint32_t *dst, const uint32_t *pool, const int32_t *outs, uint32_t nout,
                                   uint32_t P, uint32_t W, cudaStream_t st);

// Register-resident Goldilocks butterfly loop (ALU ceiling measurement).
// Each thread performs iters * 8 butterflies; sink receives one word per block.
cudaError_t launch_butterfly_peak(uint32_t blocks, uint32_t threads, uint32_t iters, uint64_t *sink,
                                  cudaStream_t st);
// Same for Harvey/Shoup butterflies modulo a 30-bit prime (MK_FORM_NTT2).
cudaError_t launch_butterfly_peak2(uint32_t blocks, uint32_t threads, uint32_t iters, uint32_t *sink,
                                   cudaStream_t st);
// Same for complex FP64 butterflies (MK_FORM_FFT).
cudaError_t launch_butterfly_peak_fft(uint32_t blocks, uint32_t threads, uint32_t iters, double *sink,
                                      cudaStream_t st);

}  // namespace mk
