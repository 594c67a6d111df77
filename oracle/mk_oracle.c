/*
 * mk_oracle.c -- plain, slow CPU oracle for multi-key TFHE gate bootstrapping.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference the GPU
 * library is compared against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  The product library never
 * links, imports or calls it, and it shares no source with the product.
 *
 * Everything here follows the paper (Jiang et al., "Privacy-Preserving
 * Distributed Machine Learning Made Faster", arXiv 2205.05825) and the MKTFHE
 * scheme it builds on, step by step, with no blocking, fusion or reordering:
 *   - notation, torus T = R/Z, T_N[X] = R[X]/(X^N+1) mod 1: Sec. 3.1
 *   - MKTFHE.Setup / KeyGen / SymEnc / SymDec / MKKeySwitch / NAND: Sec. 3.2
 *   - TFHE gate constants: Sec. 3.2 (bullet list of TFHE.Boots*)
 *   - multi-key gates: Sec. 4.1, Eq. 6-11; LweAdd Algorithm 1, LweMul
 *     Algorithm 2; operation matrix Table 1
 *   - parameters: Table 7
 * Torus elements are held as uint32 (x stands for x / 2^32); all arithmetic
 * wraps mod 2^32.  Bootstrapping is deterministic; randomness enters only in
 * key generation and encryption, through a counter-based generator
 * (Philox4x32-10) keyed by explicit seeds.
 *
 * Readings of points the paper leaves open (the paper names UniEnc, the
 * hybrid product and the multi-key key switch but does not define them):
 *   R1  phase convention: phi = b + sum_i <a_i, s_i> (Sec. 3.2, SymEnc/SymDec);
 *       the same "+" sign for RLWE: phi = c_0 + sum_j c_j z_j.
 *   R2  bit m is encoded as m/4 (SymEnc, scaling factor 1/4).  The bootstrap
 *       maps input phase in [1/4, 3/4) to 1/4 and the rest to 0: a -1/4 shift
 *       of b, a sign test by the test vector of constant 1/8, then +1/8.
 *       This is the only window under which the NAND constant 5/8 (Sec. 3.2),
 *       AND (Eq. 6), OR (Eq. 7), XOR (Eq. 10) and NOT (Eq. 8) are all correct.
 *   R3  NOR and XNOR as printed (Eq. 9: 1/8 - c1 - c2; Eq. 11:
 *       1/4 - 2(c1 - c2)) fail their truth tables under R2; this oracle uses
 *       NOR = 3/8 - c1 - c2 and XNOR = 1/2 + 2(c1 - c2).
 *   R4  UniEnc(mu; z): r binary, d = r*a + mu*g + e1, f1 uniform,
 *       f0 = -z*f1 + r*g + e2, with the CRS a and g_l = 2^(32 - Bgbit*l).
 *   R5  hybrid product HP(c, (d, f0, f1), i): u_j = g^-1(c_j);
 *       v = -<u_0, a> + sum_{j>=1} <u_j, pk_j>; w = g^-1(v);
 *       c'_j = <u_j, d>; c'_0 += <w, f0>; c'_i += <w, f1>.
 *   R6  signed gadget digits in [-B/2, B/2) with round-to-nearest at the
 *       last digit (offset 2^(32 - Bgbit*d - 1)).
 *   R7  key switch: per party, round each coefficient to ks_bit*t bits, take
 *       t digits base 2^ks_bit, add the key rows LWE_s(delta*z_j*2^(32-ks_bit*l))
 *       for every nonzero digit delta.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Parameters (Table 7 notation: n, N, B = 2^bg_bit, d, B' = 2^ks_bit, d' = t) */
/* ------------------------------------------------------------------------- */
typedef struct {
    uint32_t n;       /* LWE dimension per party */
    uint32_t N;       /* ring dimension */
    uint32_t k;       /* number of parties */
    uint32_t bg_bit;  /* log2 of the bootstrapping gadget base B */
    uint32_t d;       /* bootstrapping gadget length */
    uint32_t ks_bit;  /* log2 of the key-switching base B' */
    uint32_t t;       /* key-switching length d' */
    uint32_t pad;
    double sigma_lwe;  /* LWE noise standard deviation (torus units) */
    double sigma_rlwe; /* RLWE noise standard deviation (torus units) */
} orc_params;

static uint32_t log2u(uint32_t x) { uint32_t l = 0; while ((1u << l) < x) ++l; return l; }

int orc_params_check(const orc_params *p) {
    if (!p) return -1;
    if (p->n == 0 || p->k == 0 || p->d == 0 || p->t == 0) return -1;
    if (p->N < 4 || (p->N & (p->N - 1))) return -1;
    if (p->bg_bit == 0 || p->bg_bit * p->d > 32) return -1;
    if (p->ks_bit == 0 || p->ks_bit * p->t > 31) return -1;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC 2011), written from its published definition.        */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Word q of the stream (seed, tag): counter = (q/4 low, q/4 high, tag, 0),
 * key = (seed low, seed high), word q%4 of the output block. */
uint32_t orc_word(uint64_t seed, uint32_t tag, uint64_t q) {
    uint64_t blk = q >> 2;
    uint32_t ctr[4] = {(uint32_t)blk, (uint32_t)(blk >> 32), tag, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[q & 3];
}

/* Standard normal number q of stream (seed, tag): Box-Muller (cosine branch)
 * on words 2q and 2q+1: u1 = (w0 + 1)/2^32 in (0,1], u2 = w1/2^32. */
double orc_normal(uint64_t seed, uint32_t tag, uint64_t q) {
    double u1 = ((double)orc_word(seed, tag, 2 * q) + 1.0) / 4294967296.0;
    double u2 = (double)orc_word(seed, tag, 2 * q + 1) / 4294967296.0;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * 3.14159265358979323846 * u2);
}

/* Gaussian torus32 noise: round(sigma * 2^32 * g) as a wrapping uint32. */
uint32_t orc_gauss32(uint64_t seed, uint32_t tag, uint64_t q, double sigma) {
    if (sigma == 0.0) return 0u;
    double g = orc_normal(seed, tag, q);
    long long e = llround(sigma * 4294967296.0 * g);
    return (uint32_t)(uint64_t)e;
}

/* Stream tags (shared numbering with the library's key generator). */
enum {
    TAG_CRS = 0x01,
    TAG_S = 0x10, TAG_Z = 0x11, TAG_PK_E = 0x12,
    TAG_BK_R = 0x20, TAG_BK_F1 = 0x21, TAG_BK_E1 = 0x22, TAG_BK_E2 = 0x23,
    TAG_KS_A = 0x30, TAG_KS_E = 0x31,
    TAG_ENC_A = 0x40, TAG_ENC_E = 0x41
};

/* ------------------------------------------------------------------------- */
/* Polynomials in T_N[X] = R[X]/(X^N + 1) mod 1 (Sec. 3.1), coefficients     */
/* held as uint32 (torus32) or as small integers cast to uint32.              */
/* ------------------------------------------------------------------------- */

/* out = p * q in Z[X]/(X^N+1), coefficients mod 2^32 (schoolbook):
 * out_m = sum_{i+j=m} p_i q_j - sum_{i+j=m+N} p_i q_j. */
void orc_negacyclic_mul(uint32_t N, const uint32_t *p, const uint32_t *q, uint32_t *out) {
    uint32_t *r = (uint32_t *)calloc(N, sizeof(uint32_t));
    for (uint32_t i = 0; i < N; ++i) {
        uint32_t pi = p[i];
        if (pi == 0) continue;
        for (uint32_t j = 0; j < N - i; ++j) r[i + j] += pi * q[j];
        for (uint32_t j = N - i; j < N; ++j) r[i + j - N] -= pi * q[j];
    }
    memcpy(out, r, N * sizeof(uint32_t));
    free(r);
}

/* acc += p * q (negacyclic, mod 2^32). */
static void negacyclic_muladd(uint32_t N, const uint32_t *p, const uint32_t *q, uint32_t *acc) {
    for (uint32_t i = 0; i < N; ++i) {
        uint32_t pi = p[i];
        if (pi == 0) continue;
        for (uint32_t j = 0; j < N - i; ++j) acc[i + j] += pi * q[j];
        for (uint32_t j = N - i; j < N; ++j) acc[i + j - N] -= pi * q[j];
    }
}

/* out = X^e * p for e in [0, 2N): X^N = -1 makes the shift negacyclic. */
void orc_monomial_mul(uint32_t N, uint32_t e, const uint32_t *p, uint32_t *out) {
    uint32_t *r = (uint32_t *)malloc(N * sizeof(uint32_t));
    e %= 2 * N;
    for (uint32_t m = 0; m < N; ++m) {
        uint32_t pos = m + e; /* X^m * X^e = X^(m+e) */
        uint32_t v = p[m];
        if (pos >= 2 * N) pos -= 2 * N;
        if (pos >= N) { pos -= N; v = 0u - v; }
        r[pos] = v;
    }
    memcpy(out, r, N * sizeof(uint32_t));
    free(r);
}

/* ------------------------------------------------------------------------- */
/* Gadget decomposition g^-1 (reading R6).  g_l = 2^(32 - bg_bit*l), l=1..d.  */
/* Returns d signed digits u_l in [-B/2, B/2) with sum_l u_l g_l equal to x   */
/* rounded to the nearest multiple of 2^(32 - bg_bit*d).                      */
/* ------------------------------------------------------------------------- */
void orc_gadget_decompose(const orc_params *P, uint32_t x, int32_t *digits) {
    uint32_t B = 1u << P->bg_bit, half = B >> 1;
    uint32_t offset = 0;
    for (uint32_t l = 1; l <= P->d; ++l) offset += half << (32 - P->bg_bit * l);
    if (P->bg_bit * P->d < 32) offset += 1u << (32 - P->bg_bit * P->d - 1); /* rounding */
    uint32_t xp = x + offset;
    for (uint32_t l = 1; l <= P->d; ++l) {
        uint32_t raw = (xp >> (32 - P->bg_bit * l)) & (B - 1);
        digits[l - 1] = (int32_t)raw - (int32_t)half;
    }
}

/* Decompose every coefficient of a polynomial: digits[l][m] (as uint32). */
static void gadget_decompose_poly(const orc_params *P, const uint32_t *c, uint32_t *digits) {
    int32_t dg[32];
    for (uint32_t m = 0; m < P->N; ++m) {
        orc_gadget_decompose(P, c[m], dg);
        for (uint32_t l = 0; l < P->d; ++l) digits[(size_t)l * P->N + m] = (uint32_t)dg[l];
    }
}

/* ------------------------------------------------------------------------- */
/* Key generation: MKTFHE.Setup / MKTFHE.KeyGen (Sec. 3.2), readings R4, R7.  */
/* Layouts (uint32):                                                          */
/*   crs  [d][N]                     the common reference string a            */
/*   s    [n]  (0/1), z [N] (0/1)    TLWE and RLWE secrets of one party       */
/*   pk   [d][N]                     b = -z*a + e                             */
/*   bk   [n][3][d][N]               UniEnc(s_j; z) = (d-vector, f0, f1)      */
/*   ks   [N][t][B'-1][n+1]          LWE_s(delta*z_j*2^(32-ks_bit*(l+1)))     */
/*                                   row = (a_0..a_{n-1}, b)                  */
/* ------------------------------------------------------------------------- */
void orc_keygen_crs(const orc_params *P, uint64_t crs_seed, uint32_t *crs) {
    for (uint32_t l = 0; l < P->d; ++l)
        for (uint32_t m = 0; m < P->N; ++m)
            crs[(size_t)l * P->N + m] = orc_word(crs_seed, TAG_CRS, (uint64_t)l * P->N + m);
}

static uint32_t gadget_g(const orc_params *P, uint32_t l0 /* 0-based */) {
    return 1u << (32 - P->bg_bit * (l0 + 1));
}

void orc_keygen_party(const orc_params *P, const uint32_t *crs, uint64_t seed, uint32_t *s,
                      uint32_t *z, uint32_t *pk, uint32_t *bk, uint32_t *ks, int nthreads) {
    const uint32_t n = P->n, N = P->N, d = P->d, t = P->t;
    const uint32_t Bks = 1u << P->ks_bit;
    for (uint32_t j = 0; j < n; ++j) s[j] = orc_word(seed, TAG_S, j) & 1u;
    for (uint32_t m = 0; m < N; ++m) z[m] = orc_word(seed, TAG_Z, m) & 1u;
    /* public key: b_l = -z * a_l + e_l */
    uint32_t *tmp = (uint32_t *)malloc(N * sizeof(uint32_t));
    for (uint32_t l = 0; l < d; ++l) {
        orc_negacyclic_mul(N, z, crs + (size_t)l * N, tmp);
        for (uint32_t m = 0; m < N; ++m)
            pk[(size_t)l * N + m] = (0u - tmp[m]) + orc_gauss32(seed, TAG_PK_E, (uint64_t)l * N + m, P->sigma_rlwe);
    }
    free(tmp);
    /* bootstrapping key: BK_j = UniEnc(s_j; z) for j = 0..n-1 */
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic)
#endif
    for (int64_t jj = 0; jj < (int64_t)n; ++jj) {
        uint32_t j = (uint32_t)jj;
        uint32_t *r = (uint32_t *)malloc(N * sizeof(uint32_t));
        uint32_t *prod = (uint32_t *)malloc(N * sizeof(uint32_t));
        for (uint32_t m = 0; m < N; ++m) r[m] = orc_word(seed, TAG_BK_R, (uint64_t)j * N + m) & 1u;
        uint32_t *ent = bk + (size_t)j * 3 * d * N;
        uint32_t *dv = ent, *f0 = ent + (size_t)d * N, *f1 = ent + (size_t)2 * d * N;
        for (uint32_t l = 0; l < d; ++l) {
            uint64_t qbase = ((uint64_t)j * d + l) * N;
            uint32_t g = gadget_g(P, l);
            /* d_l = r * a_l + s_j * g_l + e1 */
            orc_negacyclic_mul(N, r, crs + (size_t)l * N, prod);
            for (uint32_t m = 0; m < N; ++m)
                dv[(size_t)l * N + m] = prod[m] + orc_gauss32(seed, TAG_BK_E1, qbase + m, P->sigma_rlwe);
            dv[(size_t)l * N + 0] += s[j] * g; /* constant polynomial s_j * g_l */
            /* f1_l uniform; f0_l = -z * f1_l + r * g_l + e2 */
            for (uint32_t m = 0; m < N; ++m) f1[(size_t)l * N + m] = orc_word(seed, TAG_BK_F1, qbase + m);
            orc_negacyclic_mul(N, z, f1 + (size_t)l * N, prod);
            for (uint32_t m = 0; m < N; ++m)
                f0[(size_t)l * N + m] = (0u - prod[m]) + r[m] * g + orc_gauss32(seed, TAG_BK_E2, qbase + m, P->sigma_rlwe);
        }
        free(r);
        free(prod);
    }
    /* key-switching key (reading R7) */
    const size_t rows = (size_t)N * t * (Bks - 1);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t rr = 0; rr < (int64_t)rows; ++rr) {
        uint64_t row = (uint64_t)rr;
        uint32_t delta = (uint32_t)(row % (Bks - 1)) + 1;
        uint32_t l = (uint32_t)((row / (Bks - 1)) % t);
        uint32_t j = (uint32_t)(row / ((uint64_t)(Bks - 1) * t));
        uint32_t *dst = ks + row * (n + 1);
        uint32_t dot = 0;
        for (uint32_t x = 0; x < n; ++x) {
            dst[x] = orc_word(seed, TAG_KS_A, row * n + x);
            dot += dst[x] * s[x];
        }
        uint32_t msg = delta * z[j] * (1u << (32 - P->ks_bit * (l + 1)));
        dst[n] = (0u - dot) + msg + orc_gauss32(seed, TAG_KS_E, row, P->sigma_lwe);
    }
}

/* ------------------------------------------------------------------------- */
/* MKTFHE.SymEnc / SymDec (Sec. 3.2).  A multi-key ciphertext is laid out as  */
/* uint32[k*n + 1] = (a_1 | a_2 | ... | a_k | b); ciphertext extension of a   */
/* single-key ciphertext of party p zero-fills every other block.             */
/* ------------------------------------------------------------------------- */
void orc_encrypt(const orc_params *P, uint32_t party, const uint32_t *s, uint64_t seed,
                 const uint8_t *bits, size_t count, uint32_t *ct) {
    const uint32_t n = P->n, k = P->k;
    const size_t W = (size_t)k * n + 1;
    for (size_t c = 0; c < count; ++c) {
        uint32_t *row = ct + c * W;
        memset(row, 0, W * sizeof(uint32_t));
        uint32_t dot = 0;
        for (uint32_t x = 0; x < n; ++x) {
            uint32_t a = orc_word(seed, TAG_ENC_A, (uint64_t)c * n + x);
            row[(size_t)party * n + x] = a;
            dot += a * s[x];
        }
        uint32_t mu = (bits[c] & 1u) ? (1u << 30) : 0u; /* bit m -> m/4 */
        row[(size_t)k * n] = (0u - dot) + mu + orc_gauss32(seed, TAG_ENC_E, c, P->sigma_lwe);
    }
}

/* Joint-key encryption (test helper): every party block uniform, so that all
 * k*n blind-rotation steps are active: b = -sum_i <a_i, s_i> + m/4 + e. */
void orc_encrypt_joint(const orc_params *P, const uint32_t *s_all, uint64_t seed,
                       const uint8_t *bits, size_t count, uint32_t *ct) {
    const uint32_t n = P->n, k = P->k;
    const size_t W = (size_t)k * n + 1;
    for (size_t c = 0; c < count; ++c) {
        uint32_t *row = ct + c * W;
        uint32_t dot = 0;
        for (size_t x = 0; x < (size_t)k * n; ++x) {
            uint32_t a = orc_word(seed, TAG_ENC_A, (uint64_t)c * k * n + x);
            row[x] = a;
            dot += a * s_all[x];
        }
        uint32_t mu = (bits[c] & 1u) ? (1u << 30) : 0u;
        row[(size_t)k * n] = (0u - dot) + mu + orc_gauss32(seed, TAG_ENC_E, c, P->sigma_lwe);
    }
}

/* phase = b + sum_i <a_i, s_i>   (s_all = [k][n]) */
uint32_t orc_phase(const orc_params *P, const uint32_t *s_all, const uint32_t *ct) {
    const size_t kn = (size_t)P->k * P->n;
    uint32_t ph = ct[kn];
    for (size_t x = 0; x < kn; ++x) ph += ct[x] * s_all[x];
    return ph;
}

/* SymDec: the bit m in {0,1} minimising |phase - m/4| on the torus, i.e.
 * m = 1 iff phase lies in [1/8, 5/8). */
void orc_decrypt(const orc_params *P, const uint32_t *s_all, const uint32_t *ct, size_t count,
                 uint8_t *bits) {
    const size_t W = (size_t)P->k * P->n + 1;
    for (size_t c = 0; c < count; ++c) {
        uint32_t ph = orc_phase(P, s_all, ct + c * W);
        bits[c] = (uint8_t)(((ph - (1u << 29)) & 0xFFFFFFFFu) < (1u << 31));
    }
}

/* ------------------------------------------------------------------------- */
/* Ciphertext-level linear operations (Sec. 4.2).                             */
/* ------------------------------------------------------------------------- */
/* ModToT: a fraction num/den of the torus as torus32 (den a power of two). */
uint32_t orc_mod_to_t(int32_t num, uint32_t den) {
    uint32_t sh = 32 - log2u(den);
    return (uint32_t)num << sh;
}

/* Algorithm 1 (LweAdd): a_{i,j} = a1_{i,j} + a2_{i,j}, b = b1 + b2. */
void orc_lwe_add(const orc_params *P, const uint32_t *c1, const uint32_t *c2, uint32_t *out) {
    const size_t W = (size_t)P->k * P->n + 1;
    for (size_t x = 0; x < W; ++x) out[x] = c1[x] + c2[x];
}

/* LweSub (provided by MKTFHE, Sec. 4.1): c1 - c2 element by element. */
void orc_lwe_sub(const orc_params *P, const uint32_t *c1, const uint32_t *c2, uint32_t *out) {
    const size_t W = (size_t)P->k * P->n + 1;
    for (size_t x = 0; x < W; ++x) out[x] = c1[x] - c2[x];
}

/* Algorithm 2 (LweMul): c = c1 + kk * c2 for an integer scalar kk. */
void orc_lwe_mul(const orc_params *P, const uint32_t *c1, int32_t kk, const uint32_t *c2, uint32_t *out) {
    const size_t W = (size_t)P->k * P->n + 1;
    for (size_t x = 0; x < W; ++x) out[x] = c1[x] + (uint32_t)kk * c2[x];
}

/* Trivial ciphertext (0, ..., 0, mu) of a torus constant. */
static void lwe_trivial(const orc_params *P, uint32_t mu, uint32_t *out) {
    const size_t W = (size_t)P->k * P->n + 1;
    memset(out, 0, W * sizeof(uint32_t));
    out[W - 1] = mu;
}

/* Gate identifiers. */
enum { ORC_AND = 0, ORC_OR = 1, ORC_NAND = 2, ORC_NOR = 3, ORC_XOR = 4, ORC_XNOR = 5 };

/* The linear part of each bootstrapped gate (Table 1 lists the operations):
 *   AND  (Eq. 6):  (0,-1/8) + c1 + c2                 LweAdd, ModToT
 *   OR   (Eq. 7):  (0, 1/8) + c1 + c2                 LweAdd, ModToT
 *   NAND (Sec. 3.2, TFHE.BootsNAND): (0, 5/8) - c1 - c2   LweSub, ModToT
 *   NOR  (Eq. 9, constant per reading R3): (0, 3/8) - c1 - c2
 *   XOR  (Eq. 10): 2 * (c1 - c2)                      LweSub, LweMul
 *   XNOR (Eq. 11, per reading R3): (0, 1/2) + 2 * (c1 - c2)
 */
int orc_gate_linear(const orc_params *P, int type, const uint32_t *c1, const uint32_t *c2, uint32_t *out) {
    const size_t W = (size_t)P->k * P->n + 1;
    uint32_t *tr = (uint32_t *)malloc(W * sizeof(uint32_t));
    uint32_t *tmp = (uint32_t *)malloc(W * sizeof(uint32_t));
    int rc = 0;
    switch (type) {
    case ORC_AND:
        lwe_trivial(P, orc_mod_to_t(-1, 8), tr);
        orc_lwe_add(P, tr, c1, tmp);
        orc_lwe_add(P, tmp, c2, out);
        break;
    case ORC_OR:
        lwe_trivial(P, orc_mod_to_t(1, 8), tr);
        orc_lwe_add(P, tr, c1, tmp);
        orc_lwe_add(P, tmp, c2, out);
        break;
    case ORC_NAND:
        lwe_trivial(P, orc_mod_to_t(5, 8), tr);
        orc_lwe_sub(P, tr, c1, tmp);
        orc_lwe_sub(P, tmp, c2, out);
        break;
    case ORC_NOR:
        lwe_trivial(P, orc_mod_to_t(3, 8), tr);
        orc_lwe_sub(P, tr, c1, tmp);
        orc_lwe_sub(P, tmp, c2, out);
        break;
    case ORC_XOR:
        orc_lwe_sub(P, c1, c2, tmp);           /* c1 - c2 */
        lwe_trivial(P, 0u, tr);
        orc_lwe_mul(P, tr, 2, tmp, out);       /* 0 + 2 * (c1 - c2) */
        break;
    case ORC_XNOR:
        orc_lwe_sub(P, c1, c2, tmp);
        lwe_trivial(P, orc_mod_to_t(1, 2), tr);
        orc_lwe_mul(P, tr, 2, tmp, out);       /* 1/2 + 2 * (c1 - c2) */
        break;
    default:
        rc = -1;
    }
    free(tr);
    free(tmp);
    return rc;
}

/* Linear combination with explicit constant and integer scalars:
 * out = (0, cst) + s1 * c1 + s2 * c2 (Algorithms 1-2 composed). */
void orc_lin_comb(const orc_params *P, uint32_t cst, int32_t s1, const uint32_t *c1, int32_t s2,
                  const uint32_t *c2, uint32_t *out) {
    const size_t W = (size_t)P->k * P->n + 1;
    uint32_t *tr = (uint32_t *)malloc(W * sizeof(uint32_t));
    uint32_t *tmp = (uint32_t *)malloc(W * sizeof(uint32_t));
    lwe_trivial(P, cst, tr);
    orc_lwe_mul(P, tr, s1, c1, tmp);
    orc_lwe_mul(P, tmp, s2, c2, out);
    free(tr);
    free(tmp);
}

/* MKNOT (Eq. 8): (0, 1/4) - c; no bootstrapping, no key switching. */
void orc_not(const orc_params *P, const uint32_t *c, uint32_t *out) {
    const size_t W = (size_t)P->k * P->n + 1;
    uint32_t *tr = (uint32_t *)malloc(W * sizeof(uint32_t));
    lwe_trivial(P, orc_mod_to_t(1, 4), tr);
    orc_lwe_sub(P, tr, c, out);
    free(tr);
}

/* ------------------------------------------------------------------------- */
/* Gate bootstrapping GB (Sec. 3.2): evaluate the decryption circuit.         */
/* ------------------------------------------------------------------------- */

/* Modulus switch of every word to Z_{2N}: round(x * 2N / 2^32) mod 2N. */
uint32_t orc_mod_switch(const orc_params *P, uint32_t x) {
    uint32_t sh = 32 - (log2u(P->N) + 1);
    return (uint32_t)((((uint64_t)x + (1ull << (sh - 1))) >> sh) & (2u * P->N - 1));
}

/* Hybrid product (reading R5) of the MK RLWE ciphertext c = (c_0, ..., c_k)
 * with the uni-encryption bk_ij = (d, f0, f1) of party `party` (1..k):
 * returns c' with <c', (1, z_1..z_k)> ~ mu * <c, (1, z_1..z_k)>. */
void orc_hybrid_product(const orc_params *P, const uint32_t *c, const uint32_t *bk_ij,
                        const uint32_t *crs, const uint32_t *const *pks, uint32_t party,
                        uint32_t *out) {
    const uint32_t N = P->N, d = P->d, k = P->k;
    const uint32_t *dv = bk_ij, *f0 = bk_ij + (size_t)d * N, *f1 = bk_ij + (size_t)2 * d * N;
    uint32_t *u = (uint32_t *)malloc((size_t)d * N * sizeof(uint32_t));
    uint32_t *v = (uint32_t *)calloc(N, sizeof(uint32_t));
    uint32_t *negu = (uint32_t *)malloc((size_t)N * sizeof(uint32_t));
    memset(out, 0, (size_t)(k + 1) * N * sizeof(uint32_t));
    for (uint32_t j = 0; j <= k; ++j) {
        gadget_decompose_poly(P, c + (size_t)j * N, u); /* u_j = g^-1(c_j) */
        for (uint32_t l = 0; l < d; ++l) {
            const uint32_t *ul = u + (size_t)l * N;
            /* c'_j = <u_j, d> */
            negacyclic_muladd(N, ul, dv + (size_t)l * N, out + (size_t)j * N);
            if (j == 0) {
                /* v -= <u_0, a> */
                for (uint32_t m = 0; m < N; ++m) negu[m] = 0u - ul[m];
                negacyclic_muladd(N, negu, crs + (size_t)l * N, v);
            } else {
                /* v += <u_j, pk_j> */
                negacyclic_muladd(N, ul, pks[j - 1] + (size_t)l * N, v);
            }
        }
    }
    gadget_decompose_poly(P, v, u); /* w = g^-1(v) */
    for (uint32_t l = 0; l < d; ++l) {
        negacyclic_muladd(N, u + (size_t)l * N, f0 + (size_t)l * N, out);                       /* c'_0 += <w, f0> */
        negacyclic_muladd(N, u + (size_t)l * N, f1 + (size_t)l * N, out + (size_t)party * N);   /* c'_i += <w, f1> */
    }
    free(u);
    free(v);
    free(negu);
}

/* Blind rotation.  abar = mod-switched (k*n + 1) words, b last, after the
 * -1/4 window shift.  acc[(k+1)][N] on return.  Steps are taken for party
 * i = 1..k and j = 0..n-1 in ascending order; `max_steps` (or -1 for all)
 * truncates the loop for stage-by-stage comparison. */
void orc_blind_rotate(const orc_params *P, const uint32_t *abar, const uint32_t *crs,
                      const uint32_t *const *pks, const uint32_t *const *bks, int64_t max_steps,
                      uint32_t *acc) {
    const uint32_t n = P->n, N = P->N, k = P->k, d = P->d;
    const size_t A = (size_t)(k + 1) * N;
    uint32_t *tv = (uint32_t *)malloc(N * sizeof(uint32_t));
    uint32_t *rot = (uint32_t *)malloc(A * sizeof(uint32_t));
    uint32_t *hp = (uint32_t *)malloc(A * sizeof(uint32_t));
    /* ACC = (X^{-b} * v, 0, ..., 0) with test vector v = sum_m (1/8) X^m */
    for (uint32_t m = 0; m < N; ++m) tv[m] = 1u << 29;
    memset(acc, 0, A * sizeof(uint32_t));
    uint32_t bbar = abar[(size_t)k * n];
    orc_monomial_mul(N, (2 * N - bbar) % (2 * N), tv, acc);
    int64_t steps = 0;
    for (uint32_t i = 1; i <= k; ++i) {
        for (uint32_t j = 0; j < n; ++j) {
            if (max_steps >= 0 && steps >= max_steps) goto done;
            ++steps;
            uint32_t e = abar[(size_t)(i - 1) * n + j];
            /* CMux: ACC <- ACC + HP((X^{-e} - 1) * ACC, BK_{i,j}) */
            for (uint32_t p = 0; p <= k; ++p) {
                orc_monomial_mul(N, (2 * N - e) % (2 * N), acc + (size_t)p * N, rot + (size_t)p * N);
                for (uint32_t m = 0; m < N; ++m) rot[(size_t)p * N + m] -= acc[(size_t)p * N + m];
            }
            orc_hybrid_product(P, rot, bks[i - 1] + (size_t)j * 3 * d * N, crs, pks, i, hp);
            for (size_t x = 0; x < A; ++x) acc[x] += hp[x];
        }
    }
done:
    free(tv);
    free(rot);
    free(hp);
}

/* SampleExtract of coefficient 0: the LWE (a_1..a_k, b) of dimension k*N
 * with phase under (z_1..z_k) equal to coefficient 0 of the RLWE phase:
 * b = c_0[0]; a_i[0] = c_i[0]; a_i[m] = -c_i[N - m]. */
void orc_sample_extract(const orc_params *P, const uint32_t *acc, uint32_t *lwe) {
    const uint32_t N = P->N, k = P->k;
    for (uint32_t i = 1; i <= k; ++i) {
        const uint32_t *ci = acc + (size_t)i * N;
        uint32_t *ai = lwe + (size_t)(i - 1) * N;
        ai[0] = ci[0];
        for (uint32_t m = 1; m < N; ++m) ai[m] = 0u - ci[N - m];
    }
    lwe[(size_t)k * N] = acc[0];
}

/* GB: window shift -1/4, modulus switch, blind rotation, SampleExtract, +1/8.
 * Output: LWE of dimension k*N under (z_1..z_k), phase ~ 1/4 iff the input
 * phase lies in [1/4, 3/4), ~ 0 otherwise (reading R2). */
void orc_bootstrap(const orc_params *P, const uint32_t *c, const uint32_t *crs,
                   const uint32_t *const *pks, const uint32_t *const *bks, uint32_t *lwe_out) {
    const size_t W = (size_t)P->k * P->n + 1;
    uint32_t *abar = (uint32_t *)malloc(W * sizeof(uint32_t));
    uint32_t *acc = (uint32_t *)malloc((size_t)(P->k + 1) * P->N * sizeof(uint32_t));
    for (size_t x = 0; x + 1 < W; ++x) abar[x] = orc_mod_switch(P, c[x]);
    abar[W - 1] = orc_mod_switch(P, c[W - 1] - (1u << 30)); /* -1/4 window shift */
    orc_blind_rotate(P, abar, crs, pks, bks, -1, acc);
    orc_sample_extract(P, acc, lwe_out);
    lwe_out[(size_t)P->k * P->N] += 1u << 29; /* +1/8 */
    free(abar);
    free(acc);
}

/* MKTFHE.MKKeySwitch (Sec. 3.2, reading R7): LWE of dimension k*N under
 * (z_1..z_k) -> LWE of dimension k*n under (s_1..s_k). */
void orc_keyswitch(const orc_params *P, const uint32_t *const *kss, const uint32_t *lwe_in,
                   uint32_t *out) {
    const uint32_t n = P->n, N = P->N, k = P->k, t = P->t;
    const uint32_t Bks = 1u << P->ks_bit;
    const uint32_t prec = P->ks_bit * t;
    const uint32_t round_off = 1u << (32 - prec - 1);
    memset(out, 0, ((size_t)k * n + 1) * sizeof(uint32_t));
    out[(size_t)k * n] = lwe_in[(size_t)k * N];
    for (uint32_t i = 0; i < k; ++i) {
        const uint32_t *ksi = kss[i];
        uint32_t *oa = out + (size_t)i * n;
        for (uint32_t j = 0; j < N; ++j) {
            uint32_t abar = lwe_in[(size_t)i * N + j] + round_off;
            for (uint32_t l = 0; l < t; ++l) {
                uint32_t delta = (abar >> (32 - P->ks_bit * (l + 1))) & (Bks - 1);
                if (delta == 0) continue;
                const uint32_t *row = ksi + (((size_t)j * t + l) * (Bks - 1) + (delta - 1)) * (n + 1);
                for (uint32_t x = 0; x < n; ++x) oa[x] += row[x];
                out[(size_t)k * n] += row[n];
            }
        }
    }
}

/* One multi-key bootstrapped gate (MKTFHE.NAND pattern, Sec. 3.2 / 3.1):
 * linear combination -> GB -> MKKeySwitch. */
int orc_gate(const orc_params *P, int type, const uint32_t *c1, const uint32_t *c2,
             const uint32_t *crs, const uint32_t *const *pks, const uint32_t *const *bks,
             const uint32_t *const *kss, uint32_t *out) {
    const size_t W = (size_t)P->k * P->n + 1;
    uint32_t *lin = (uint32_t *)malloc(W * sizeof(uint32_t));
    uint32_t *ext = (uint32_t *)malloc(((size_t)P->k * P->N + 1) * sizeof(uint32_t));
    int rc = orc_gate_linear(P, type, c1, c2, lin);
    if (rc == 0) {
        orc_bootstrap(P, lin, crs, pks, bks, ext);
        orc_keyswitch(P, kss, ext, out);
    }
    free(lin);
    free(ext);
    return rc;
}

/* Batch of independent gates, OpenMP across gates only (each gate runs the
 * plain single-gate path above). */
int orc_gates(const orc_params *P, const int32_t *types, const uint32_t *c1, const uint32_t *c2,
              size_t count, const uint32_t *crs, const uint32_t *pk_all, const uint32_t *bk_all,
              const uint32_t *ks_all, uint32_t *out, int nthreads) {
    const uint32_t k = P->k;
    const size_t W = (size_t)k * P->n + 1;
    const uint32_t **pks = (const uint32_t **)malloc(k * sizeof(void *));
    const uint32_t **bks = (const uint32_t **)malloc(k * sizeof(void *));
    const uint32_t **kss = (const uint32_t **)malloc(k * sizeof(void *));
    const size_t pk_sz = (size_t)P->d * P->N, bk_sz = (size_t)P->n * 3 * P->d * P->N;
    const size_t ks_sz = (size_t)P->N * P->t * ((1u << P->ks_bit) - 1) * (P->n + 1);
    for (uint32_t i = 0; i < k; ++i) {
        pks[i] = pk_all + i * pk_sz;
        bks[i] = bk_all + i * bk_sz;
        kss[i] = ks_all + i * ks_sz;
    }
    int bad = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
#endif
    for (int64_t g = 0; g < (int64_t)count; ++g) {
        if (orc_gate(P, types[g], c1 + g * W, c2 + g * W, crs, pks, bks, kss, out + g * W) != 0) bad |= 1;
    }
    free(pks);
    free(bks);
    free(kss);
    return bad ? -1 : 0;
}

/* Blind rotation of a batch with a step limit (stage comparison). */
void orc_blind_rotate_batch(const orc_params *P, const uint32_t *abar, size_t count,
                            const uint32_t *crs, const uint32_t *pk_all, const uint32_t *bk_all,
                            int64_t max_steps, uint32_t *acc_out, int nthreads) {
    const uint32_t k = P->k;
    const size_t W = (size_t)k * P->n + 1, A = (size_t)(k + 1) * P->N;
    const uint32_t **pks = (const uint32_t **)malloc(k * sizeof(void *));
    const uint32_t **bks = (const uint32_t **)malloc(k * sizeof(void *));
    const size_t pk_sz = (size_t)P->d * P->N, bk_sz = (size_t)P->n * 3 * P->d * P->N;
    for (uint32_t i = 0; i < k; ++i) {
        pks[i] = pk_all + i * pk_sz;
        bks[i] = bk_all + i * bk_sz;
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t g = 0; g < (int64_t)count; ++g)
        orc_blind_rotate(P, abar + g * W, crs, pks, bks, max_steps, acc_out + g * A);
    free(pks);
    free(bks);
}

/* Single hybrid product with explicit pointers (for identity tests). */
void orc_hybrid_product_flat(const orc_params *P, const uint32_t *c, const uint32_t *bk_ij,
                             const uint32_t *crs, const uint32_t *pk_all, uint32_t party,
                             uint32_t *out) {
    const uint32_t k = P->k;
    const uint32_t **pks = (const uint32_t **)malloc(k * sizeof(void *));
    for (uint32_t i = 0; i < k; ++i) pks[i] = pk_all + (size_t)i * P->d * P->N;
    orc_hybrid_product(P, c, bk_ij, crs, pks, party, out);
    free(pks);
}

/* Bootstrap (without key switch) of a batch: out [count][k*N + 1]. */
void orc_bootstrap_batch(const orc_params *P, const uint32_t *c, size_t count, const uint32_t *crs,
                         const uint32_t *pk_all, const uint32_t *bk_all, uint32_t *out, int nthreads) {
    const uint32_t k = P->k;
    const size_t W = (size_t)k * P->n + 1, E = (size_t)k * P->N + 1;
    const uint32_t **pks = (const uint32_t **)malloc(k * sizeof(void *));
    const uint32_t **bks = (const uint32_t **)malloc(k * sizeof(void *));
    const size_t pk_sz = (size_t)P->d * P->N, bk_sz = (size_t)P->n * 3 * P->d * P->N;
    for (uint32_t i = 0; i < k; ++i) {
        pks[i] = pk_all + i * pk_sz;
        bks[i] = bk_all + i * bk_sz;
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t g = 0; g < (int64_t)count; ++g) orc_bootstrap(P, c + g * W, crs, pks, bks, out + g * E);
    free(pks);
    free(bks);
}

/* Key switch of a batch: in [count][k*N + 1] -> out [count][k*n + 1]. */
void orc_keyswitch_batch(const orc_params *P, const uint32_t *ks_all, const uint32_t *in, size_t count,
                         uint32_t *out, int nthreads) {
    const uint32_t k = P->k;
    const size_t W = (size_t)k * P->n + 1, E = (size_t)k * P->N + 1;
    const uint32_t **kss = (const uint32_t **)malloc(k * sizeof(void *));
    const size_t ks_sz = (size_t)P->N * P->t * ((1u << P->ks_bit) - 1) * (P->n + 1);
    for (uint32_t i = 0; i < k; ++i) kss[i] = ks_all + i * ks_sz;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t g = 0; g < (int64_t)count; ++g) orc_keyswitch(P, kss, in + g * E, out + g * W);
    free(kss);
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
