/*
 * mk_tfhe.h -- C ABI of the GB300 multi-key TFHE gate-bootstrapping library.
 *
 * The calls follow the paper's statement of the problem (Jiang et al.,
 * "Privacy-Preserving Distributed Machine Learning Made Faster",
 * arXiv 2205.05825): MKTFHE.Setup / KeyGen / SymEnc / SymDec (Sec. 3.2),
 * the bootstrapped gates of Sec. 4.1 (Eq. 6-11 and the NAND of Sec. 3.2),
 * MKNOT (Eq. 8) and the k-bit two's-complement operators of Sec. 4.3-4.5
 * (Algorithms 3-6).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Torus elements are uint32 (x stands for x / 2^32).
 *  - A multi-key LWE ciphertext is one row uint32[k*n + 1] laid out as
 *    (a_1 | a_2 | ... | a_k | b): party blocks of n words, then b.  Its phase
 *    is b + sum_i <a_i, s_i>; a bit m is encoded as m/4 (Sec. 3.2, SymEnc).
 *  - Batches are row-major [count][k*n + 1].  k-bit integers are LSB-first
 *    rows of bit ciphertexts, two's complement: [pairs][kbits][k*n + 1].
 *  - Pointers named d_* are device pointers on the context's device, owned by
 *    the caller, 16-byte aligned.  Pointers named h_* are host pointers owned
 *    by the caller.  The library owns the keys and its scratch space.
 *  - Device work is enqueued on the context's stream and returns without
 *    waiting, except where a call says it synchronises.  A context is not
 *    thread-safe: one host thread per context at a time.
 *  - Every call returns MK_OK (0) or a negative error code; mk_last_error()
 *    gives a message for the last failure on that context.  Errors never
 *    leave the device in a faulted state: arguments are checked on the host
 *    before any launch.
 */
#ifndef MK_TFHE_H
#define MK_TFHE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- errors */
#define MK_OK 0
#define MK_EINVAL (-1)   /* bad argument (null pointer, size, party index) */
#define MK_ENOMEM (-2)   /* host or device allocation failed */
#define MK_EPARAMS (-3)  /* parameter set not supported */
#define MK_ETIMEOUT (-4) /* a device-side wait gave up (watchdog) */
#define MK_EDEVICE (-5)  /* CUDA error, or a device call on a host-only context */
#define MK_ESTATE (-6)   /* keys missing for the requested operation */
#define MK_EFORMAT (-7)  /* key blob has a bad header, size or checksum */

/* ---------------------------------------------------------------- params */
/* mkparams (Sec. 3.1, Table 7): LWE dimension n, ring dimension N, party
 * count k, bootstrapping gadget base B = 2^bg_bit of length d, key-switching
 * base B' = 2^ks_bit of length t (Table 7's d'), and the Gaussian noise
 * standard deviations (torus units) of LWE and RLWE samples. */
typedef struct mk_params {
    uint32_t n, N, k, bg_bit, d, ks_bit, t, reserved;
    double sigma_lwe, sigma_rlwe;
} mk_params;

enum {
    MK_PRESET_TOY = 0,   /* n=64,  N=256,  B=2^8, d=3, B'=4, t=8, sigma 2^-25 / 2^-25 */
    MK_PRESET_FULL = 1,  /* n=560, N=1024, B=2^8, d=3, B'=4, t=8, sigma 2^-15 / per k */
    MK_PRESET_PAPER = 2  /* Table 7 verbatim: B=2^9, alpha=3.05e-5, beta=3.72e-9 */
};

/* Fill *out with a preset for k parties.  FULL's RLWE sigma depends on k:
 * 2^-28 (k=1), 2^-30 (k=2,3), 2^-32 (k>=4) -- the stated 2^-25 exceeds the
 * decision margin of the bootstrap at N=1024.  Returns MK_EINVAL for an
 * unknown preset or k == 0. */
int mk_params_preset(int preset, uint32_t k, mk_params *out);

/* ---------------------------------------------------------------- context */
typedef struct mk_ctx mk_ctx;

/* MKTFHE.Setup (Sec. 3.2): create a context for `params`, derive the common
 * reference string a in T_N[X]^d from crs_seed, bind CUDA device `device`
 * and stream `stream` (a cudaStream_t; NULL = the legacy default stream).
 * device = -1 makes a host-only context: key generation, encryption,
 * decryption and key export work, device calls return MK_EDEVICE.
 * Supported: N in {256, 1024}, d*bg_bit <= 32, ks_bit*t <= 31,
 * 1 <= k <= 8.  The context is released with mk_ctx_destroy. */
int mk_ctx_create(const mk_params *params, uint64_t crs_seed, int device, void *stream, mk_ctx **out);
int mk_ctx_destroy(mk_ctx *ctx);
int mk_ctx_set_stream(mk_ctx *ctx, void *stream);
int mk_ctx_get_params(const mk_ctx *ctx, mk_params *out);

/* Negacyclic-product form used by the blind rotation.  The two NTT forms and
 * the tensor form are exact (the product sums are recovered as integers and
 * reduced mod 2^32), so they give bit-identical ciphertexts.  The FP64 FFT form rounds each
 * product to the nearest integer; its error per product is small (well
 * below 2^12 torus32 units) but not zero, so its ciphertexts differ from the
 * exact ones in low bits and, rarely, more (a flipped gadget digit), while
 * decrypting to the same bits.  Changing the form rebuilds the device keys
 * on the next gate call.  Default: MK_FORM_NTT2. */
enum {
    MK_FORM_NTT = 0,  /* NTT over the prime 2^64 - 2^32 + 1 */
    MK_FORM_NTT2 = 1, /* NTTs over the primes 0x0fff0001 and 0x0ffee001, CRT */
    MK_FORM_FFT = 2,  /* FP64 FFT of N/2 folded complex points */
    MK_FORM_TC = 3    /* tensor cores: Toeplitz products of key byte planes and
                         gadget digits, bf16 operands, fp32 sums (exact) */
};
/* MK_FORM_TC runs the blind rotation of a batch as a wave: every CMux step is
 * a few launches over all gates of the batch, with the accumulators and
 * digits in a device workspace the context allocates with the keys (about
 * 4 (3 (k+1) N + k n) + 6 (k+2) N bytes per gate, for up to 4096 gates at a
 * time).  It needs N in {256, 1024}, d = 3 and bg_bit <= 8 (the exactness
 * bound |digit| * |key byte| * N <= 2^24); mk_ctx_set_form returns
 * MK_EPARAMS otherwise. */
int mk_ctx_set_form(mk_ctx *ctx, int form);
int mk_ctx_get_form(const mk_ctx *ctx, int *form);

/* Largest number of gates bootstrapped by one launch (default 4096; the
 * scratch space grows with it).  1 gives the one-gate-per-launch form. */
int mk_ctx_set_batch(mk_ctx *ctx, uint32_t max_gates_per_launch);

/* Latency (cluster) form of the NTT blind rotation: one thread-block cluster
 * of k+1 CTAs per gate, CTA j owning accumulator polynomial j, so one gate
 * runs two to four times faster than in the batched kernel (k = 2 to 7)
 * while the GPU has SMs to spare.  MK_CLUSTER_AUTO (default) uses it for launches of at most
 * max(1, floor(k/2)) waves of gates, a wave being the clusters the device
 * can hold at once (queried when the keys are laid out for the form); _ON
 * for every launch, _OFF never.  Only the NTT forms with k <= 7; results are
 * bit-identical either way.  No paper counterpart: a scheduling choice. */
enum { MK_CLUSTER_AUTO = 0, MK_CLUSTER_OFF = 1, MK_CLUSTER_ON = 2 };
int mk_ctx_set_cluster(mk_ctx *ctx, int mode);

/* Test hook for the kernels' bounded waits (no paper counterpart).  Every
 * wait of the staged blind rotation (variant 6) for a key copy and of the
 * tcgen05 product engine (MK_FORM_TC, variant 1) gives up after wait_ns of
 * global time (0: the default, 1 s); a kernel whose wait gave up stops its
 * work, lets its own copies and tensor-core operations finish, and returns
 * without its outputs; the next mk_sync reports MK_ETIMEOUT, and the context
 * stays usable.  kind MK_FAULT_SKIP_KEY_STEP: until the next call, the staged
 * kernel and the cluster latency kernel never copy the key entry of CMux step
 * `arg` (0-based), so the waits for it run out.  kind MK_FAULT_SKIP_DIGIT_TILE: in the next tcgen05
 * launch, the first CTA that reaches its digit tile `arg` does not load it
 * (one shot).  kind MK_FAULT_SKIP_WIRE_READY: until the next call, the
 * persistent operator launch never marks the output of its work item `arg`
 * (0-based, in the plan's level order) ready, so once every other gate has
 * finished, the gates that read it give up after the bound.  MK_FAULT_NONE clears all three.  Nothing here
 * faults the device: a skipped copy or mark is one that is never issued. */
enum { MK_FAULT_NONE = 0, MK_FAULT_SKIP_KEY_STEP = 1, MK_FAULT_SKIP_DIGIT_TILE = 2, MK_FAULT_SKIP_WIRE_READY = 3 };
int mk_debug_fault(mk_ctx *ctx, int kind, int64_t arg, uint64_t wait_ns);

/* The k-bit operators evaluate their netlist level by level.  With graphs on
 * (the default) the level loop of each (operator, width, pairs) plan is
 * captured once as a CUDA graph on a stream the context owns and replayed on
 * the context's stream; it is captured again when the form, the variant or
 * the key buffers change.  Graphs are not used while timing is enabled
 * (mk_timing_enable) or with MK_FORM_TC.  No paper counterpart: launch
 * overhead only, results are identical either way. */
int mk_ctx_set_graphs(mk_ctx *ctx, int on);

/* How the operators (mk_*_kbit) run their netlists on the NTT forms.
 * MK_EXEC_LEVELS: one batched bootstrap + key-switch launch pair per netlist
 * level (the cluster latency kernel for narrow levels).  MK_EXEC_PERSISTENT:
 * one launch over every (gate, pair) of the netlist: CTAs take gates in the
 * netlist's level order, wait (bounded, MK_ETIMEOUT through mk_sync) until
 * the gate's input wires are ready (giving up when no gate of the launch
 * finishes for the wait bound of mk_debug_fault), and run the gate's blind
 * rotation and key switch, so a gate starts as soon as its own inputs exist
 * instead of after the whole previous level.  MK_EXEC_AUTO (default): the
 * level loop, which measured faster on every operator (their pairs advance
 * in step, and the persistent launch switches keys one gate at a time).
 * Results are identical.  No paper counterpart (Alg. 3-6 define the
 * circuits, not their schedule). */
enum { MK_EXEC_AUTO = 0, MK_EXEC_LEVELS = 1, MK_EXEC_PERSISTENT = 2 };
int mk_ctx_set_circuit_exec(mk_ctx *ctx, int mode);

/* Construction family of the operator netlists (same functions, same
 * quotient and remainder rules).  MK_CIRCUIT_ARRAY (default): the paper's
 * array constructions (Sec. 4.3-4.5) -- ripple-carry adder and subtractor,
 * Baugh-Wooley array multiplier with a ripple final addition, CAS-array
 * divider: O(k) levels per addition, the fewest gates.  MK_CIRCUIT_SHALLOW:
 * every carry chain replaced by a parallel-prefix (Sklansky) carry network
 * and the multiplier's partial products reduced by Dadda stages: O(log k)
 * levels per addition, for 10-25 % more gates in the multiplier and divider
 * and up to 60 % more in the adders (levels at 8 / 16 bits: add 17 / 33 -> 7 / 9, mul 35 / 75 -> 19 / 26, div 236 / 852 ->
 * 100 / 223).  Each level is one batched launch whatever its width, so an
 * evaluation with few pairs per level (latency-bound) runs faster with the
 * shallow family and one that fills every level (throughput-bound) with the
 * array family.  Two more families reproduce the paper's own constructions
 * for comparison: MK_CIRCUIT_PAPER, the array family with the multiplier
 * built from the paper's 0-, 1- and 2-adders (Sec. 3.3, Alg. 4: k rows of
 * k-1 typed full adders over sign-weighted partial products, k^2 + 5k(k-1)
 * gates against the paper's 7k(k-1)); MK_CIRCUIT_NAND, Table 2's naive
 * scheme: the array family with every gate composed of bootstrapped NANDs
 * (NOT included).  Applies to the operator calls and server requests made
 * after the change; MK_EINVAL for another value.  No paper counterpart
 * (ARRAY and PAPER are the paper's constructions). */
enum { MK_CIRCUIT_ARRAY = 0, MK_CIRCUIT_SHALLOW = 1, MK_CIRCUIT_PAPER = 2, MK_CIRCUIT_NAND = 3 };
int mk_ctx_set_circuit_style(mk_ctx *ctx, int style);
int mk_ctx_get_circuit_style(const mk_ctx *ctx, int *style);

/* Blind-rotation kernel variants (same results, different register/occupancy
 * trade-offs): 0..MK_NUM_VARIANTS-1.  0-5: one CTA per gate, with different
 * digit polynomials per forward pass, register caps, twiddle placement and
 * elements per thread; 6: several gates per CTA sharing each CMux step's
 * bootstrapping-key entry, bulk-copied once into shared memory; 7, 8
 * (MK_FORM_NTT2): the two primes' transforms on separate warps, recombined
 * by CRT through shared memory (MK_FORM_NTT runs variant 2's kernel for 7
 * and 8).  mk_autotune times every variant on
 * `sample_gates` random ciphertexts on the context's device, keeps the
 * fastest for the context and stores it in *best (and, if ms_out is not
 * NULL, each variant's milliseconds in ms_out[0..MK_NUM_VARIANTS-1]).  It
 * synchronises the stream.  MK_FORM_FFT and MK_FORM_TC have one kernel for
 * every variant number: there it times nothing, reports 0 ms and keeps the
 * variant.  No paper counterpart: a tuning aid. */
#define MK_NUM_VARIANTS 9
int mk_ctx_set_variant(mk_ctx *ctx, int variant);
int mk_ctx_get_variant(const mk_ctx *ctx, int *variant);
int mk_autotune(mk_ctx *ctx, uint32_t sample_gates, int *best, float *ms_out);

/* Product-form autotuner.  forms: a set of bits (1 << MK_FORM_*).  For each
 * form in the set that the parameters support, the call builds that form's
 * device keys, autotunes its variants (mk_autotune) and times one launch of
 * min(sample_gates, batch) random ciphertexts; it keeps the fastest form and
 * variant for the context and stores the form in *best_form (if not NULL)
 * and each tried form's milliseconds in ms_out[MK_FORM_*] (0 for the rest;
 * ms_out may be NULL).  Leave MK_FORM_FFT out of the set to choose among the
 * exact forms only.  It synchronises the stream.  MK_EPARAMS if no form in
 * the set supports the parameters.  No paper counterpart: a tuning aid. */
#define MK_NUM_FORMS 4
int mk_autotune_form(mk_ctx *ctx, uint32_t sample_gates, uint32_t forms, int *best_form, float *ms_out);

/* Message of the last failed call on ctx (never NULL). */
const char *mk_last_error(const mk_ctx *ctx);

/* Wait for all work enqueued on the context's stream; reports any
 * asynchronous CUDA error as MK_EDEVICE, and MK_ETIMEOUT if a bounded
 * device-side wait of the tensor form's tcgen05 engine gave up since the
 * last check (its results are then invalid). */
int mk_sync(mk_ctx *ctx);

/* ---------------------------------------------------------------- keys */
/* MKTFHE.KeyGen (Sec. 3.2) for party `party` (0-based) from `seed`: the TLWE
 * secret s in {0,1}^n, the RLWE secret z in {0,1}^N, the public key
 * b = -z*a + e, the bootstrapping key BK = {UniEnc(s_j; z)}_j and the
 * key-switching key KS.  Secrets stay in host memory of the context; public
 * material is uploaded on first use.  Deterministic in (params, crs_seed,
 * seed): every random number comes from Philox4x32-10 streams. */
int mk_keygen(mk_ctx *ctx, uint32_t party, uint64_t seed);

/* Key material in host memory, uint32 torus words, row-major:
 *   crs [d][N];  s [n] (0/1);  z [N] (0/1);  pk [d][N];
 *   bk  [n][3][d][N]       UniEnc(s_j; z) = (d-vector, f0, f1) for j < n;
 *   ks  [N][t][B'-1][n+1]  row (a_0..a_{n-1}, b) = LWE_s(delta*z_j*2^(32-ks_bit*(l+1)))
 *                          at [j][l][delta-1].
 * mk_import_crs replaces the CRS; mk_import_party copies one party's keys in
 * (s and z may be NULL for a party whose secrets this context must not hold).
 * mk_export_* copy out; any output pointer may be NULL to skip that part. */
int mk_import_crs(mk_ctx *ctx, const uint32_t *h_crs);
int mk_import_party(mk_ctx *ctx, uint32_t party, const uint32_t *h_s, const uint32_t *h_z,
                    const uint32_t *h_pk, const uint32_t *h_bk, const uint32_t *h_ks);
int mk_export_crs(const mk_ctx *ctx, uint32_t *h_crs);
int mk_export_party(const mk_ctx *ctx, uint32_t party, uint32_t *h_s, uint32_t *h_z, uint32_t *h_pk,
                    uint32_t *h_bk, uint32_t *h_ks);

/* Serialised key set: header (magic, version, params, party mask, secret
 * flag), CRS, each party's keys, FNV-1a 64 checksum.  mk_save_keys with
 * h_blob == NULL stores the needed size in *len.  include_secrets = 0 writes
 * the public material only.  mk_load_keys returns MK_EFORMAT on a bad magic,
 * parameter mismatch, truncated blob or checksum. */
int mk_save_keys(const mk_ctx *ctx, int include_secrets, void *h_blob, size_t cap, size_t *len);
int mk_load_keys(mk_ctx *ctx, const void *h_blob, size_t len);

/* ---------------------------------------------------------------- enc/dec */
/* MKTFHE.SymEnc (Sec. 3.2) by party `party` of count bits (0/1 bytes) into
 * h_ct [count][k*n + 1], extended to the multi-key layout (other parties'
 * blocks zero).  b = -<a, s> + m/4 + e; a and e from Philox streams of seed. */
int mk_encrypt(mk_ctx *ctx, uint32_t party, const uint8_t *h_bits, size_t count, uint64_t seed,
               uint32_t *h_ct);
/* Encryption under the joint key (every party block uniform); needs every
 * party's secret.  Used to make all k*n blind-rotation steps active. */
int mk_encrypt_joint(mk_ctx *ctx, const uint8_t *h_bits, size_t count, uint64_t seed, uint32_t *h_ct);

/* A noiseless ciphertext of each public bit: zero mask, zero noise, b = m/4
 * (the encoding of SymEnc, Sec. 3.2).  It decrypts to the bit under every
 * set of keys and needs no secret: the operator circuits use it for their
 * constant wires, and a server for public operands of the encrypted
 * application (a data count, a learning rate, a zoom factor; Sec. 4.6).
 * Only the lowest bit of each h_bits byte is read; h_ct: host
 * [count][k*n + 1]. */
int mk_trivial(mk_ctx *ctx, const uint8_t *h_bits, size_t count, uint32_t *h_ct);

/* MKTFHE.SymDec (Sec. 3.2): with every party's secret, the bit m minimising
 * |b + sum_i <a_i, s_i> - m/4|.  `ct` is a host pointer if on_device == 0,
 * else a device pointer (copied back, synchronising the stream). */
int mk_decrypt(mk_ctx *ctx, const uint32_t *ct, size_t count, int on_device, uint8_t *h_bits);
/* Phases b + sum_i <a_i, s_i> of count ciphertexts (same pointer rule). */
int mk_phase(mk_ctx *ctx, const uint32_t *ct, size_t count, int on_device, uint32_t *h_phase);

/* ---------------------------------------------------------------- gates */
enum { MK_AND = 0, MK_OR = 1, MK_NAND = 2, MK_NOR = 3, MK_XOR = 4, MK_XNOR = 5 };

/* Multi-key bootstrapped gates (Sec. 4.1): for g < count,
 *   d_out[g] = KeySwitch(GB(lin(type, d_a[g], d_b[g])))
 * with the linear part of Eq. 6 (AND), Eq. 7 (OR), Sec. 3.2 (NAND: 5/8 - c1 - c2),
 * Eq. 9 (NOR, constant 3/8), Eq. 10 (XOR), Eq. 11 (XNOR: 1/2 + 2(c1 - c2)).
 * mk_gate applies one type to every gate; mk_gates reads a per-gate type
 * (uint8, device).  d_out may not alias d_a or d_b.  Needs every party's
 * public keys. */
int mk_gate(mk_ctx *ctx, int type, const uint32_t *d_a, const uint32_t *d_b, uint32_t *d_out,
            size_t count);
int mk_gates(mk_ctx *ctx, const uint8_t *d_types, const uint32_t *d_a, const uint32_t *d_b,
             uint32_t *d_out, size_t count);

/* General linear gate: d_out[g] = KeySwitch(GB((0, cst[g]) + s1[g]*a[g] + s2[g]*b[g]))
 * where d_lin holds count records {uint32 cst; int32 s1; int32 s2} (device). */
typedef struct mk_lin { uint32_t cst; int32_t s1, s2; } mk_lin;
int mk_gates_lin(mk_ctx *ctx, const mk_lin *d_lin, const uint32_t *d_a, const uint32_t *d_b,
                 uint32_t *d_out, size_t count);

/* The linear record of one bootstrapped gate type (MK_AND..MK_XNOR) into
 * *out (host memory): AND Eq. 6 (-1/8, 1, 1), OR Eq. 7 (1/8, 1, 1), NAND
 * Sec. 3.2 (5/8, -1, -1), NOR (3/8, -1, -1), XOR Eq. 10 (0, 2, -2), XNOR
 * (1/2, 2, -2); the NOR and XNOR constants are this library's readings of
 * Eq. 9 and Eq. 11 (the printed ones fail their truth tables).  neg_a /
 * neg_b nonzero fold a NOT (Eq. 8: 1/4 - c) of that input into the record.
 * Needs no context.  MK_EINVAL for another type or a NULL out. */
int mk_gate_lin(int type, int neg_a, int neg_b, mk_lin *out);

/* MKNOT (Eq. 8): d_out[g] = (0, 1/4) - d_a[g]; no bootstrapping, no key
 * switching.  d_out may alias d_a. */
int mk_not(mk_ctx *ctx, const uint32_t *d_a, uint32_t *d_out, size_t count);

/* ---------------------------------------------------------------- operators */
/* k-bit two's-complement operators (Sec. 3.3, Sec. 4.3-4.5, Algorithms 3-6)
 * as netlists of the bootstrapped gates, evaluated level by level: every
 * level of the netlist is one batched bootstrap + key-switch launch over all
 * its gates of all `pairs` operand pairs (gates of one level are
 * independent).  Operands are LSB-first rows of bit ciphertexts:
 * d_a, d_b [pairs][kbits][k*n+1].  Outputs:
 *   mk_add_kbit / mk_sub_kbit: d_out [pairs][kbits]     (a + b, a - b mod 2^kbits)
 *   mk_mul_kbit:               d_out [pairs][2*kbits]   (the full product)
 *   mk_div_kbit:               d_q, d_r [pairs][kbits]  (truncating quotient,
 *                              remainder with a's sign; b = 0 and
 *                              (-2^(kbits-1)) / (-1) give unspecified bits)
 * 2 <= kbits <= 64.  The context keeps a plan per (operator, kbits, pairs):
 * gate descriptors and a wire buffer of (gates + 2 + 2*kbits) * pairs
 * ciphertexts, allocated on first use. */
enum { MK_OP_ADD = 0, MK_OP_SUB = 1, MK_OP_MUL = 2, MK_OP_DIV = 3 };
int mk_add_kbit(mk_ctx *ctx, uint32_t kbits, const uint32_t *d_a, const uint32_t *d_b, uint32_t *d_out,
                size_t pairs);
int mk_sub_kbit(mk_ctx *ctx, uint32_t kbits, const uint32_t *d_a, const uint32_t *d_b, uint32_t *d_out,
                size_t pairs);
int mk_mul_kbit(mk_ctx *ctx, uint32_t kbits, const uint32_t *d_a, const uint32_t *d_b, uint32_t *d_out,
                size_t pairs);
int mk_div_kbit(mk_ctx *ctx, uint32_t kbits, const uint32_t *d_a, const uint32_t *d_b, uint32_t *d_q,
                uint32_t *d_r, size_t pairs);

/* The netlist of an operator in a construction family (MK_CIRCUIT_*), for
 * inspection: gate records (output wire of
 * gate g = 2 + 2*kbits + g; wires 0/1 = constants 0/1, then a's bits, then
 * b's bits), outputs encoded as 2*wire + negated, and the number of levels.
 * Any output pointer may be NULL (counts only); caps bound the copies. */
typedef struct mk_gate_rec {
    uint8_t op;           /* MK_AND .. MK_XNOR */
    uint8_t neg_a, neg_b; /* input negated (MKNOT folded into the gate) */
    uint8_t reserved;
    int32_t a, b;         /* input wires */
} mk_gate_rec;
int mk_circuit_netlist(int op, uint32_t kbits, int style, mk_gate_rec *gates, uint32_t gate_cap,
                       uint32_t *n_gates, int32_t *outputs, uint32_t out_cap, uint32_t *n_outputs,
                       uint32_t *n_levels);

/* ---------------------------------------------------------------- serving */
/* Continuous batching of operator requests from several clients (the paper's
 * cloud server evaluating participants' circuits, Sec. 5.5).  Every admitted
 * request keeps its wire ciphertexts in one device pool of `pool_rows`
 * ciphertext rows; mk_server_step runs one wave: one batched bootstrap +
 * key-switch launch over at most `wave_gates` ready gates of all running
 * requests (each contributes the gates of its current netlist level; a level
 * is split across waves when it does not fit), after admitting queued
 * requests, in arrival order, while the pool has room.  Requests therefore
 * join while others are on the GPU, and their gates share launches.  Results
 * are the same alone and in any mix (every gate touches only its own
 * request's wires; the NTT forms are exact).
 *
 * mk_server_submit queues a request: operator MK_OP_*, kbits, pairs and the
 * operand/output device buffers of mk_*_kbit (d_out2 = remainder for
 * MK_OP_DIV, NULL otherwise).  The operands must stay valid until the request
 * is running, the outputs are written when it is done.  mk_server_step
 * synchronises the context's stream before returning; *n_done = requests
 * finished by this wave.  mk_server_poll: *state = 0 queued, 1 running,
 * 2 done. */
typedef struct mk_server mk_server;
int mk_server_create(mk_ctx *ctx, uint32_t wave_gates, uint64_t pool_rows, mk_server **out);
int mk_server_destroy(mk_server *srv);
int mk_server_submit(mk_server *srv, int op, uint32_t kbits, const uint32_t *d_a, const uint32_t *d_b,
                     uint32_t *d_out, uint32_t *d_out2, uint32_t pairs, uint64_t *ticket);
int mk_server_step(mk_server *srv, uint32_t *n_done);
int mk_server_poll(const mk_server *srv, uint64_t ticket, int *state);
int mk_server_stats(const mk_server *srv, uint64_t *waves, uint64_t *gates, uint32_t *running, uint32_t *queued);

/* ---------------------------------------------------------------- stages */
/* The stages of one bootstrapped gate, for stage-by-stage comparison.
 * mk_stage_modswitch: d_abar[g] = mod-switched words of lin(...) with the
 *   -1/4 window shift on b (values in [0, 2N)), layout as a ciphertext.
 * mk_stage_blind_rotate: accumulator (k+1 polynomials of N words) after the
 *   first max_steps CMux steps (-1 = all k*n), from d_abar.
 * mk_stage_bootstrap: d_ext[g] = SampleExtract(blind rotation) + 1/8, an LWE
 *   of dimension k*N + 1 under (z_1..z_k).
 * mk_stage_keyswitch: MKKeySwitch (Sec. 3.2) of d_ext into d_out. */
int mk_stage_modswitch(mk_ctx *ctx, const mk_lin *d_lin, const uint32_t *d_a, const uint32_t *d_b,
                       uint32_t *d_abar, size_t count);
int mk_stage_blind_rotate(mk_ctx *ctx, const uint32_t *d_abar, size_t count, int64_t max_steps,
                          uint32_t *d_acc);
int mk_stage_bootstrap(mk_ctx *ctx, const mk_lin *d_lin, const uint32_t *d_a, const uint32_t *d_b,
                       uint32_t *d_ext, size_t count);
int mk_stage_keyswitch(mk_ctx *ctx, const uint32_t *d_ext, uint32_t *d_out, size_t count);

/* ---------------------------------------------------------------- no allocation */
/* mk_gates_noalloc: the same gates as mk_gates, for callers that cannot let
 * the library allocate device memory while they run -- for example a serving
 * process that reserves all device memory at start-up and forbids later
 * cudaMalloc, or a latency-critical loop where an allocation could stall or
 * fail.  The paper has no counterpart; this is an integration aid.
 *
 *  - It calls no cudaMalloc, cudaFree or other allocating routine.  Its
 *    scratch (gate descriptors and the extracted samples between blind
 *    rotation and key switch) is a fixed device array of
 *    MK_NOALLOC_SCRATCH_BYTES that every GPU which loads the library holds
 *    until the process exits.
 *  - Capacity: a call takes at most
 *      floor((MK_NOALLOC_SCRATCH_BYTES - 256) / (4 * (k*N + 1) + 24))
 *    gates (510 for k = 2, N = 1024; 127 for k = 8).  Larger counts return
 *    MK_EINVAL before any device work.
 *  - The context's keys must already be on the device: make one ordinary
 *    gate call (or mk_autotune) on this context first, otherwise MK_ESTATE.
 *  - The first call on a device looks up the scratch array's device address
 *    (cudaGetSymbolAddress, with that device current) and keeps it for the
 *    process; make that first call before any stream capture.  The kept
 *    address does not survive cudaDeviceReset (or any other teardown of the
 *    device's primary context): do not call this entry point after one.
 *  - Under MK_FORM_TC the blind rotation works in the context's tensor-form
 *    workspace, which the context allocated together with its device keys
 *    (so no allocation happens in the call either); the fixed array still
 *    holds the descriptors and the extracted samples.
 *  - Every call shares the one array and it keeps the previous call's
 *    contents; the kernels write every scratch word before reading it, so
 *    nothing needs clearing.  Calls whose device work overlaps (different
 *    streams or contexts on the same GPU) race on the scratch: serialise
 *    them, e.g. by using one stream. */
#define MK_NOALLOC_SCRATCH_BYTES (4u << 20)
int mk_gates_noalloc(mk_ctx *ctx, const uint8_t *d_types, const uint32_t *d_a, const uint32_t *d_b,
                     uint32_t *d_out, size_t count);

/* ---------------------------------------------------------------- measurement */
/* Per-kernel timing with CUDA events recorded on the context's stream around
 * every launch of the given kernel class while enabled.  mk_timing_read
 * synchronises the stream and returns the summed device milliseconds and the
 * launch count since the last reset. */
enum { MK_KERNEL_BOOTSTRAP = 0, MK_KERNEL_KEYSWITCH = 1 };
int mk_timing_enable(mk_ctx *ctx, int on);
int mk_timing_reset(mk_ctx *ctx);
int mk_timing_read(mk_ctx *ctx, int kernel, double *ms_total, uint64_t *launches);

/* ALU ceiling of a product form: run a register-resident loop of independent
 * butterflies on every SM of `device`; *per_s receives butterflies per
 * second.  form = MK_FORM_NTT: Goldilocks butterflies (one 64-bit modular
 * multiply, add and subtract); MK_FORM_NTT2: Harvey butterflies modulo a
 * 28-bit prime (one Shoup multiply, one conditional subtraction, add, sub);
 * MK_FORM_FFT: complex FP64 butterflies (one complex multiply, two complex
 * additions); MK_FORM_TC: multiply-accumulates per second of independent
 * warp-level bf16 m16n8k16 MMAs (the instruction of the tensor form).
 * No paper counterpart: a measurement aid for the roofline of the blind
 * rotation. */
int mk_measure_butterfly_rate(int device, void *stream, int form, uint32_t iters, double *per_s);

/* The product kernel of MK_FORM_TC on its own, for exactness checks:
 *   out[g] = sum_{c < nchunks} keys[c] * digits[c][g]   in Z[X]/(X^N + 1) mod 2^32
 * for g < G.  keys: device uint32 [nchunks][N] (torus32 words); digits:
 * device int8 [nchunks][G][N], each in [-128, 127]; out: device int32
 * [G][N] (the torus32 words, as int32).  engine 0: warp-level mma.sync, G a
 * positive multiple of 64; engine 1: tcgen05 with TMEM accumulators, G a
 * positive multiple of 128.  N in {256, 1024}, 1 <= nchunks <= 3; otherwise
 * MK_EINVAL.  MK_ETIMEOUT if a bounded wait of the tcgen05 kernel gave up.
 * The call allocates a bf16 copy of the digits, runs on `stream` and
 * synchronises it.  The same engine numbers select the tensor form's engine
 * as its variant (mk_ctx_set_variant; mk_autotune times both).
 * No paper counterpart: the negacyclic product of Sec. 3.1-3.2 (the hybrid
 * product's inner step) isolated for testing the tensor form. */
int mk_tc_negacyclic(int device, void *stream, uint32_t N, uint32_t G, uint32_t nchunks, const uint32_t *keys,
                     const int8_t *digits, int32_t *out, int engine);

#ifdef __cplusplus
}
#endif
#endif /* MK_TFHE_H */
