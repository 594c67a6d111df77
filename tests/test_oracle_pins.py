"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every check here compares the oracle with something other than itself:
published known-answer vectors, closed forms, exact algebraic identities,
brute force on tiny inputs, or the truth tables the paper's gates must
implement.  A plausible mistake anywhere in the oracle (a dropped term, a
wrong sign, index or operand) fails at least one of them.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from polyref import negacyclic, rlwe_phase, signed32, torus_dist

o = pytest.importorskip("oracle.oracle")
from paper_2205_05825_gb300 import workloads as W  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TRUTH = {0: lambda a, b: a & b, 1: lambda a, b: a | b, 2: lambda a, b: 1 - (a & b),
         3: lambda a, b: 1 - (a | b), 4: lambda a, b: a ^ b, 5: lambda a, b: 1 - (a ^ b)}


# ----------------------------------------------------------------------------- randomness
def test_philox_known_answers():
    """Philox4x32-10 against the Random123 known-answer vectors."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = o.philox(v[0:4], v[4:6])
        assert list(out) == v[6:10]


def test_stream_word_layout():
    """word(seed, tag, q) is word q%4 of the block with counter (q/4, 0, tag, 0)."""
    seed, tag = 0x0123456789ABCDEF, 0x21
    for q in (0, 1, 2, 3, 4, 7, 1 << 33):
        blk = q >> 2
        out = o.philox([blk & 0xFFFFFFFF, blk >> 32, tag, 0], [seed & 0xFFFFFFFF, seed >> 32])
        assert o.word(seed, tag, q) == int(out[q & 3])


def test_normal_moments_and_zero_sigma():
    """Box-Muller output: mean 0, variance 1, symmetric tails; sigma 0 gives 0."""
    x = np.array([o.normal(99, 0x12, q) for q in range(20000)])
    assert abs(x.mean()) < 0.03 and abs(x.var() - 1) < 0.05
    assert 0.035 < np.mean(np.abs(x) > 2) < 0.056  # 2-sided P(|Z|>2) = 0.0455
    assert all(o.gauss32(5, 0x12, q, 0.0) == 0 for q in range(10))
    e = signed32([o.gauss32(5, 0x12, q, 2.0 ** -15) for q in range(5000)])
    assert abs(e.std() / 2 ** 17 - 1) < 0.05  # sigma * 2^32 = 2^17 torus32 units


# ----------------------------------------------------------------------------- polynomials
@pytest.mark.parametrize("N", [4, 8, 16, 64])
def test_negacyclic_product_brute_force(N):
    """Schoolbook product equals the full product reduced by X^N = -1."""
    rng = np.random.default_rng(N)
    for _ in range(4):
        p = rng.integers(0, 1 << 32, N, dtype=np.uint64).astype(np.uint32)
        q = rng.integers(0, 1 << 32, N, dtype=np.uint64).astype(np.uint32)
        assert np.array_equal(o.negacyclic_mul(p, q), negacyclic(p, q))
    # X^N = -1: X^(N-1) * X = -1
    xa = np.zeros(N, np.uint32)
    xa[N - 1] = 1
    x1 = np.zeros(N, np.uint32)
    x1[1] = 1
    minus_one = np.zeros(N, np.uint32)
    minus_one[0] = 0xFFFFFFFF
    assert np.array_equal(o.negacyclic_mul(xa, x1), minus_one)


def test_monomial_product():
    """X^e * p equals the product with the monomial; exponents add mod 2N."""
    N = 16
    rng = np.random.default_rng(3)
    p = rng.integers(0, 1 << 32, N, dtype=np.uint64).astype(np.uint32)
    for e in range(2 * N):
        mono = np.zeros(N, np.uint32)
        mono[e % N] = 1 if e < N else 0xFFFFFFFF
        assert np.array_equal(o.monomial_mul(e, p), negacyclic(mono, p)), e
    assert np.array_equal(o.monomial_mul(N, p), (-p.astype(np.int64)).astype(np.uint32))
    assert np.array_equal(o.monomial_mul(5, o.monomial_mul(30, p)), o.monomial_mul(35 % 32, p))


def test_gadget_decomposition_closed_form():
    """Digits in [-B/2, B/2), sum u_l 2^(32-8l) = x rounded to a multiple of 2^8
    (round half up), g^-1(0) = 0."""
    P = W.toy_params(2)
    rng = np.random.default_rng(11)
    xs = list(rng.integers(0, 1 << 32, 3000, dtype=np.uint64)) + \
        [0, 1, 0x7F, 0x80, 0x81, 0xFF, 0x7FFFFF80, 0x80000000, 0xFFFFFF7F, 0xFFFFFF80, 0xFFFFFFFF]
    for x in xs:
        x = int(x)
        u = o.gadget_decompose(P, x)
        assert all(-128 <= v < 128 for v in u)
        rec = sum(int(v) << (32 - 8 * (l + 1)) for l, v in enumerate(u)) & 0xFFFFFFFF
        assert rec == (((x + 0x80) >> 8) << 8) & 0xFFFFFFFF, hex(x)
    assert list(o.gadget_decompose(P, 0)) == [0, 0, 0]


def test_gadget_decomposition_base_9():
    """Table 7's base 2^9 (d = 3): precision 27 bits, digits in [-256, 256)."""
    P = W.paper_params(2)
    rng = np.random.default_rng(12)
    for x in rng.integers(0, 1 << 32, 2000, dtype=np.uint64):
        x = int(x)
        u = o.gadget_decompose(P, x)
        assert all(-256 <= v < 256 for v in u)
        rec = sum(int(v) << (32 - 9 * (l + 1)) for l, v in enumerate(u)) & 0xFFFFFFFF
        assert rec == (((x + 0x10) >> 5) << 5) & 0xFFFFFFFF


@pytest.mark.parametrize("N", [256, 1024])
def test_mod_switch_closed_form(N):
    """x -> round(x * 2N / 2^32) mod 2N, checked with exact rationals."""
    P = dict(W.toy_params(2), N=N)
    rng = np.random.default_rng(N)
    xs = list(rng.integers(0, 1 << 32, 2000, dtype=np.uint64))
    step = (1 << 32) // (2 * N)
    xs += [0, 0xFFFFFFFF, step // 2 - 1, step // 2, step // 2 + 1, 3 * step + step // 2]
    for x in xs:
        x = int(x)
        exact = Fraction(x * 2 * N, 1 << 32)
        want = int(exact + Fraction(1, 2)) % (2 * N)  # floor(v + 1/2): ties round up
        assert o.mod_switch(P, x) == want


# ----------------------------------------------------------------------------- LWE layer
def tiny(sigma=0.0, k=2):
    return W.tiny_params(k=k, sigma=sigma)


@pytest.fixture(scope="module")
def tiny_keys():
    P = tiny(0.0)
    return P, o.keygen(P, W.CRS_SEED, W.party_seeds(2))


def test_public_key_relation_noiseless(tiny_keys):
    """With sigma = 0, pk = -z * a exactly, and UniEnc satisfies
    f0 + z * f1 = r * g (the F part encrypts r * g) for some binary r that
    also gives d - s_j g = r * a."""
    P, K = tiny_keys
    N, d = P["N"], P["d"]
    for i in range(2):
        for l in range(d):
            assert np.array_equal(K.pk[i, l], negacyclic(K.z[i], (-K.crs[l].astype(np.int64)).astype(np.uint32)))
        for j in (0, 7, P["n"] - 1):
            dv, f0, f1 = K.bk[i, j, 0], K.bk[i, j, 1], K.bk[i, j, 2]
            # recover r from d_1: d_1 = r * a_1 + s_j * g_1 (constant term); a is random so solve by brute force
            # is not needed: check consistency across digits instead.
            gl = [1 << (32 - 8 * (l + 1)) for l in range(d)]
            lhs = [(f0[l].astype(np.int64) + negacyclic(K.z[i], f1[l]).astype(np.int64)) & 0xFFFFFFFF
                   for l in range(d)]
            # r * g_l for consecutive l differ by the factor 2^8: r * g_0 = 2^8 * (r * g_1)
            assert np.array_equal(lhs[0], (lhs[1] << 8) & 0xFFFFFFFF)
            r = (lhs[d - 1] >> (32 - 8 * d)).astype(np.uint32)
            assert set(np.unique(r)) <= {0, 1}
            for l in range(d):
                want = negacyclic(r, K.crs[l]).astype(np.int64)
                want[0] += int(K.s[i, j]) * gl[l]
                assert np.array_equal(dv[l], (want & 0xFFFFFFFF).astype(np.uint32))


def test_encrypt_decrypt_noiseless(tiny_keys):
    """SymEnc with sigma = 0: phase exactly m/4; SymDec returns m."""
    P, K = tiny_keys
    bits = np.array([0, 1, 1, 0, 1], np.uint8)
    for party in (0, 1):
        c = o.encrypt(P, K, party, bits, 77 + party)
        assert np.array_equal(o.phase(P, K, c), bits.astype(np.uint32) << 30)
        assert np.array_equal(o.decrypt(P, K, c), bits)
        other = c[:, (1 - party) * P["n"]:(2 - party) * P["n"]]
        assert not other.any()  # ciphertext extension zero-fills the other block


def test_linear_ops_are_exact_on_phases(tiny_keys):
    """LweAdd / LweSub / LweMul (Algorithms 1-2) act linearly on phases, and
    MKNOT (Eq. 8) is exactly (0, 1/4) - c."""
    P, K = tiny_keys
    rng = np.random.default_rng(5)
    c1 = rng.integers(0, 1 << 32, o.ct_width(P), dtype=np.uint64).astype(np.uint32)
    c2 = rng.integers(0, 1 << 32, o.ct_width(P), dtype=np.uint64).astype(np.uint32)
    p1, p2 = int(o.phase(P, K, c1)[0]), int(o.phase(P, K, c2)[0])
    M = 0xFFFFFFFF
    assert int(o.phase(P, K, o.lwe_add(P, c1, c2))[0]) == (p1 + p2) & M
    assert int(o.phase(P, K, o.lwe_sub(P, c1, c2))[0]) == (p1 - p2) & M
    for kk in (-2, -1, 2, 3):
        assert int(o.phase(P, K, o.lwe_mul(P, c1, kk, c2))[0]) == (p1 + kk * p2) & M
    n = o.mk_not(P, c1)
    assert n[-1] == ((1 << 30) - int(c1[-1])) & M
    assert np.array_equal(n[:-1], (-c1[:-1].astype(np.int64)).astype(np.uint32))
    assert int(o.phase(P, K, n)[0]) == ((1 << 30) - p1) & M
    assert o.mod_to_t(1, 8) == 1 << 29 and o.mod_to_t(-1, 8) == 0xE0000000 and o.mod_to_t(5, 8) == 0xA0000000


def _window_bit(phase):
    """The bootstrap's decision (reading of Sec. 3.2 with the 1/4 encoding):
    1 iff the phase lies in [1/4, 3/4)."""
    return int(((phase - (1 << 30)) & 0xFFFFFFFF) < (1 << 31))


def test_gate_constants_against_truth_tables(tiny_keys):
    """The linear part of every gate (Eq. 6-11, NAND of Sec. 3.2) puts the
    phase of noiseless inputs inside the window [1/4, 3/4) exactly when the
    gate's truth table says 1, at distance >= 1/8 from the window edges."""
    P, K = tiny_keys
    for gi in range(6):
        for m1 in (0, 1):
            for m2 in (0, 1):
                c1 = o.encrypt(P, K, 0, np.array([m1], np.uint8), 1)[0]
                c2 = o.encrypt(P, K, 1, np.array([m2], np.uint8), 2)[0]
                ph = int(o.phase(P, K, o.gate_linear(P, gi, c1, c2))[0])
                assert _window_bit(ph) == TRUTH[gi](m1, m2), (gi, m1, m2)
                edge = min(int(torus_dist(ph, 1 << 30)), int(torus_dist(ph, 3 << 30)))
                assert edge >= 1 << 29


def test_printed_nor_xnor_constants_fail():
    """Eq. 9 (1/8 - c1 - c2) and Eq. 11 (1/4 - 2(c1 - c2)) as printed do not
    implement NOR / XNOR under the same window: the reading in the oracle
    replaces them (NOR 3/8, XNOR 1/2 + 2(c1 - c2))."""
    q = 1 << 30
    nor_printed = {(a, b): ((1 << 29) - a * q - b * q) & 0xFFFFFFFF for a in (0, 1) for b in (0, 1)}
    assert _window_bit(nor_printed[(0, 0)]) != 1  # NOR(0,0) must be 1
    xnor_printed = {(a, b): (q - 2 * (a * q - b * q)) & 0xFFFFFFFF for a in (0, 1) for b in (0, 1)}
    # every input pair lands exactly on a window edge: no noise margin at all
    assert all(min(int(torus_dist(v, q)), int(torus_dist(v, 3 * q))) == 0 for v in xnor_printed.values())


# ----------------------------------------------------------------------------- bootstrapping
def test_sample_extract_identity():
    """Phase of SampleExtract under z equals coefficient 0 of the RLWE phase, exactly."""
    P = dict(tiny(), N=64)
    rng = np.random.default_rng(21)
    for _ in range(5):
        acc = rng.integers(0, 1 << 32, (3, 64), dtype=np.uint64).astype(np.uint32)
        z = rng.integers(0, 2, (2, 64)).astype(np.uint32)
        lwe = o.sample_extract(P, acc)
        ph = (int(lwe[-1]) + sum(int(lwe[i * 64 + m]) * int(z[i, m]) for i in range(2) for m in range(64))) \
            & 0xFFFFFFFF
        assert ph == int(rlwe_phase(acc, z)[0])


def _hp_error_bound(P):
    # mu * sum_j t_j (rounded c_j - c_j) + r * (rounded v - v): each rounding <= 2^7
    return (1 << 7) * (1 + (P["k"] + 1) * P["N"])


def test_hybrid_product_noiseless_bound(tiny_keys):
    """HP(c, UniEnc(mu)) has phase mu * phase(c) up to the gadget rounding terms
    only (sigma = 0), for every party and both values of mu."""
    P, K = tiny_keys
    rng = np.random.default_rng(31)
    bound = _hp_error_bound(P)
    seen_mu = set()
    for party in (1, 2):
        for j in range(0, P["n"], 3):
            c = rng.integers(0, 1 << 32, (3, P["N"]), dtype=np.uint64).astype(np.uint32)
            mu = int(K.s[party - 1, j])
            seen_mu.add(mu)
            out = o.hybrid_product(P, K, c, party, j)
            want = (rlwe_phase(c, K.z).astype(np.int64) * mu) & 0xFFFFFFFF
            err = torus_dist(rlwe_phase(out, K.z), want)
            assert err.max() <= bound, (party, j, int(err.max()))
    assert seen_mu == {0, 1}


def test_blind_rotation_noiseless(tiny_keys):
    """With sigma = 0 the accumulator's phase is X^-phi * v (v = 1/8 sum X^m)
    up to the accumulated gadget rounding, where phi = b + sum a_ij s_ij mod 2N
    is computed from the mod-switched input directly."""
    P, K = tiny_keys
    N, n = P["N"], P["n"]
    rng = np.random.default_rng(41)
    abar = rng.integers(0, 2 * N, (6, 2 * n + 1)).astype(np.uint32)
    acc = o.blind_rotate(P, K, abar)
    bound = 2 * n * _hp_error_bound(P)
    for g in range(len(abar)):
        phi = (int(abar[g, -1]) + sum(int(abar[g, x]) * int(K.s_all[x]) for x in range(2 * n))) % (2 * N)
        want = np.array([(1 << 29) if (m + phi) % (2 * N) < N else (-(1 << 29)) & 0xFFFFFFFF for m in range(N)],
                        dtype=np.uint32)
        err = torus_dist(rlwe_phase(acc[g], K.z), want)
        assert err.max() <= bound


def test_blind_rotation_step_limit(tiny_keys):
    """Stopping after 0 steps leaves ACC = (X^-b v, 0, ...)."""
    P, K = tiny_keys
    N = P["N"]
    abar = np.zeros((1, 2 * P["n"] + 1), np.uint32)
    abar[0, -1] = 5
    acc = o.blind_rotate(P, K, abar, max_steps=0)[0]
    want0 = np.array([(1 << 29) if (m + 5) < N else (-(1 << 29)) & 0xFFFFFFFF for m in range(N)], np.uint32)
    assert np.array_equal(acc[0], want0) and not acc[1:].any()


def test_keyswitch_noiseless_identity(tiny_keys):
    """With sigma = 0 the key switch's output phase under s is exactly
    b + sum_ij z_ij * round16(a_ij)."""
    P, K = tiny_keys
    N = P["N"]
    rng = np.random.default_rng(51)
    lwe = rng.integers(0, 1 << 32, (4, 2 * N + 1), dtype=np.uint64).astype(np.uint32)
    out = o.keyswitch(P, K, lwe)
    for g in range(4):
        want = int(lwe[g, -1])
        for i in range(2):
            for j in range(N):
                a = int(lwe[g, i * N + j])
                want += int(K.z[i, j]) * ((((a + (1 << 15)) >> 16) << 16) & 0xFFFFFFFF)
        assert int(o.phase(P, K, out[g])[0]) == want & 0xFFFFFFFF


@pytest.mark.parametrize("k", [1, 2, 3])
def test_gate_truth_tables_toy(k):
    """All six bootstrapped gates x four input pairs decrypt to their truth
    tables (toy set, sigma 2^-25); k = 1 is single-key TFHE."""
    P = W.toy_params(k)
    K = o.keygen(P, W.CRS_SEED, W.party_seeds(k))
    g, b1, b2 = W.truth_table_inputs()
    c1 = o.encrypt(P, K, 0, b1, W.encryption_seed(1, 0))
    c2 = o.encrypt(P, K, min(1, k - 1), b2, W.encryption_seed(1, 1))
    out = o.gates(P, K, g, c1, c2)
    exp = np.array([TRUTH[int(t)](int(x), int(y)) for t, x, y in zip(g, b1, b2)], np.uint8)
    assert np.array_equal(o.decrypt(P, K, out), exp)
    ph = o.phase(P, K, out)
    assert torus_dist(ph, exp.astype(np.uint32) << 30).max() < 1 << 28  # well inside the 1/8 margin


def test_joint_encryption_all_blocks():
    """Joint-key encryption fills every party block and decrypts."""
    P = W.toy_params(3)
    K = o.keygen(P, W.CRS_SEED, W.party_seeds(3))
    bits = np.array([1, 0, 1, 1], np.uint8)
    c = o.encrypt_joint(P, K, bits, 9)
    assert all(c[:, i * P["n"]:(i + 1) * P["n"]].any() for i in range(3))
    assert np.array_equal(o.decrypt(P, K, c), bits)
