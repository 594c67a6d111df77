"""The exact tensor-core product form (MK_FORM_TC) against plain integer
arithmetic and the CPU oracle.

1. The Toeplitz product kernel alone (mk_tc_negacyclic) on adversarial
   integer inputs: every key byte -128 with every digit -128 (each row of the
   last plane sums to +-2^24, the edge of fp32 exactness), alternating signs,
   the largest positive bytes, and random words.  Reference: the negacyclic
   product written as an exact int64 Toeplitz matrix product, reduced mod 2^32.
2. Stages and whole gates on the toy set, byte-equal to the oracle: mod
   switch, blind rotation after 1, 2, 37 and all steps, extract, key switch.
3. Ragged and multi-wave batches (70 gates: one padded wave; 4096 + 70 gates:
   two waves of the context's workspace).
"""
import numpy as np
import pytest

from conftest import from_dev, oracle_keys, to_dev

pytestmark = pytest.mark.gpu

TRUTH = {0: lambda a, b: a & b, 1: lambda a, b: a | b, 2: lambda a, b: 1 - (a & b),
         3: lambda a, b: 1 - (a | b), 4: lambda a, b: a ^ b, 5: lambda a, b: 1 - (a ^ b)}


def negacyclic_sum_int64(keys, digits):
    """sum_c keys[c] * digits[c][g] in Z[X]/(X^N + 1) mod 2^32, exactly:
    T[m][t] = key[m - t] (m >= t), -key[N + m - t] (m < t); |sums| < 2^50."""
    nch, N = keys.shape
    m = np.arange(N)[:, None]
    t = np.arange(N)[None, :]
    out = np.zeros((digits.shape[1], N), np.int64)
    for c in range(nch):
        k64 = keys[c].astype(np.int64)
        T = np.where(m >= t, k64[(m - t) % N], -k64[(m - t) % N])
        out += (T @ digits[c].astype(np.int64).T).T
    return (out & 0xFFFFFFFF).astype(np.uint32)


def _run_tc(keys, digits, engine=0):
    import torch
    from paper_2205_05825_gb300 import binding as B
    out = torch.zeros((digits.shape[1], keys.shape[1]), dtype=torch.int32, device="cuda")
    B.tc_negacyclic(to_dev(keys), to_dev(digits), out, engine=engine)
    return from_dev(out)


def test_tc05_products_smallest_case(gpu_ready):
    """The tcgen05 engine on its smallest launch (N = 256, 128 gates, one
    key polynomial of random words): word for word."""
    rng = np.random.default_rng(10)
    keys = rng.integers(0, 2 ** 32, size=(1, 256), dtype=np.uint64).astype(np.uint32)
    digits = rng.integers(-128, 128, size=(1, 128, 256)).astype(np.int8)
    assert np.array_equal(_run_tc(keys, digits, engine=1), negacyclic_sum_int64(keys, digits))


@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("N", [256, 1024])
def test_tc_products_adversarial_exact(gpu_ready, N, engine):
    rng = np.random.default_rng(11)
    G = 64 if engine == 0 else 128
    cases = {
        "all -128 x -128": (np.full((1, N), 0x80808080, np.uint32), np.full((1, G, N), -128, np.int8)),
        "alternating": (np.tile(np.array([0x80808080, 0x7F7F7F7F], np.uint32), (3, N // 2)),
                        np.tile(np.array([-128, 127], np.int8), (3, G, N // 2))),
        "max positive": (np.full((2, N), 0x7F7F7F7F, np.uint32), np.full((2, G, N), 127, np.int8)),
        "random": (rng.integers(0, 2 ** 32, size=(3, N), dtype=np.uint64).astype(np.uint32),
                   rng.integers(-128, 128, size=(3, G, N)).astype(np.int8)),
    }
    for name, (keys, digits) in cases.items():
        assert np.array_equal(_run_tc(keys, digits, engine), negacyclic_sum_int64(keys, digits)), name


@pytest.mark.parametrize("engine", [0, 1])
def test_tc_products_several_gate_tiles(gpu_ready, engine):
    """Three CTA gate tiles (192 gates for mma.sync, 384 for tcgen05), two
    chunks, random words."""
    rng = np.random.default_rng(12)
    N, G = 1024, (192 if engine == 0 else 384)
    keys = rng.integers(0, 2 ** 32, size=(2, N), dtype=np.uint64).astype(np.uint32)
    digits = rng.integers(-128, 128, size=(2, G, N)).astype(np.int8)
    assert np.array_equal(_run_tc(keys, digits, engine), negacyclic_sum_int64(keys, digits))


@pytest.mark.parametrize("N,G,nch", [(1024, 5120, 2), (256, 128 * 200, 3)])
def test_tc05_products_several_items_per_cta(gpu_ready, N, G, nch):
    """The persistent tcgen05 kernel with more work items than SMs (320 and
    400 items of 128 coefficients x 128 gates), so every CTA runs passes of
    two or three items back to back: sampled gates (first and last of
    several gate tiles, random others) word for word."""
    rng = np.random.default_rng(13 + N)
    keys = rng.integers(0, 2 ** 32, size=(nch, N), dtype=np.uint64).astype(np.uint32)
    digits = rng.integers(-128, 128, size=(nch, G, N)).astype(np.int8)
    got = _run_tc(keys, digits, engine=1)
    idx = np.unique(np.concatenate([[0, 127, 128, 255, G // 2, G - 129, G - 128, G - 1],
                                    rng.integers(0, G, size=40)]))
    assert np.array_equal(got[idx], negacyclic_sum_int64(keys, digits[:, idx, :]))


def test_tc_products_rejects_bad_shapes(gpu_ready):
    import torch
    from paper_2205_05825_gb300 import binding as B
    keys = torch.zeros((1, 1024), dtype=torch.int32, device="cuda")
    digits = torch.zeros((1, 65, 1024), dtype=torch.int8, device="cuda")
    out = torch.zeros((65, 1024), dtype=torch.int32, device="cuda")
    with pytest.raises(B.MkError):
        B.tc_negacyclic(keys, digits, out)
    d64 = torch.zeros((1, 64, 1024), dtype=torch.int8, device="cuda")
    o64 = torch.zeros((64, 1024), dtype=torch.int32, device="cuda")
    with pytest.raises(B.MkError):  # the tcgen05 engine takes whole 128-gate tiles
        B.tc_negacyclic(keys, d64, o64, engine=1)


@pytest.fixture(scope="module")
def toy_tc(gpu_ready):
    from oracle import oracle as o
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    P = W.toy_params(2)
    keys = oracle_keys(P)
    ctx = B.Context(P, W.CRS_SEED, device=0)
    ctx.import_oracle_keys(keys)
    ctx.set_form("tc")
    g, b1, b2 = W.truth_table_inputs()
    c1 = o.encrypt(P, keys, 0, b1, W.encryption_seed(1, 0))
    c2 = o.encrypt(P, keys, 1, b2, W.encryption_seed(1, 1))
    yield P, keys, ctx, g, b1, b2, c1, c2
    ctx.close()


def test_tc_toy_stages_bit_exact(toy_tc):
    import torch
    from oracle import oracle as o
    from paper_2205_05825_gb300 import binding as B
    P, keys, ctx, g, b1, b2, c1, c2 = toy_tc
    lin_d = to_dev(B.lin_records(g))
    abar = torch.zeros((len(g), ctx.W), dtype=torch.int32, device="cuda")
    ctx.stage_modswitch(lin_d, to_dev(c1), to_dev(c2), abar)
    lins = np.stack([o.gate_linear(P, int(t), x, y) for t, x, y in zip(g, c1, c2)])
    ref_abar = o.modswitch_input(P, lins)
    assert np.array_equal(from_dev(abar), ref_abar)
    for steps in (0, 1, 2, 37, -1):
        acc = torch.zeros((len(g), 3, P["N"]), dtype=torch.int32, device="cuda")
        ctx.stage_blind_rotate(abar, steps, acc)
        assert np.array_equal(from_dev(acc), o.blind_rotate(P, keys, ref_abar, max_steps=steps)), steps
    ext = torch.zeros((len(g), ctx.E), dtype=torch.int32, device="cuda")
    ctx.stage_bootstrap(lin_d, to_dev(c1), to_dev(c2), ext)
    ref_ext = o.bootstrap(P, keys, lins)
    assert np.array_equal(from_dev(ext), ref_ext)
    out = torch.zeros((len(g), ctx.W), dtype=torch.int32, device="cuda")
    ctx.gates(to_dev(g.astype(np.uint8)), to_dev(c1), to_dev(c2), out)
    ctx.sync()  # reports MK_ETIMEOUT if a bounded tcgen05 wait gave up
    assert np.array_equal(from_dev(out), o.gates(P, keys, g, c1, c2))
    exp = np.array([TRUTH[int(t)](int(x), int(y)) for t, x, y in zip(g, b1, b2)], np.uint8)
    assert np.array_equal(ctx.decrypt(out), exp)


def test_tc_toy_ragged_and_two_waves(toy_tc):
    """70 gates (one wave padded to 128) and 4166 gates (waves of 4096 and
    70): all decrypt, sampled rows byte-equal to the oracle, and the first 70
    rows equal in both runs."""
    import torch
    from oracle import oracle as o
    from paper_2205_05825_gb300 import workloads as W
    P, keys, ctx = toy_tc[:3]
    G = 4096 + 70
    types, b1, b2 = W.random_gates(G, config_id=31)
    c1 = o.encrypt(P, keys, 0, b1, W.encryption_seed(31, 0))
    c2 = o.encrypt(P, keys, 1, b2, W.encryption_seed(31, 1))
    d_t, d1, d2 = to_dev(types.astype(np.uint8)), to_dev(c1), to_dev(c2)
    small = torch.zeros((70, ctx.W), dtype=torch.int32, device="cuda")
    ctx.gates(d_t[:70], d1[:70], d2[:70], small)
    out = torch.zeros((G, ctx.W), dtype=torch.int32, device="cuda")
    ctx.gates(d_t, d1, d2, out)
    got = from_dev(out)
    exp = np.array([TRUTH[int(t)](int(x), int(y)) for t, x, y in zip(types, b1, b2)], np.uint8)
    assert np.array_equal(ctx.decrypt(out), exp)
    assert np.array_equal(from_dev(small), got[:70])
    idx = np.array([0, 69, 4095, 4096, 4165])
    assert np.array_equal(got[idx], o.gates(P, keys, types[idx], c1[idx], c2[idx]))


def test_tc_rejects_unsupported_params(gpu_ready):
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    ctx = B.Context(W.paper_params(2), W.CRS_SEED, device=0)  # gadget base 2^9
    with pytest.raises(B.MkError):
        ctx.set_form("tc")
    ctx.close()


def test_autotune_form_keeps_the_fastest_exact_form(gpu_ready):
    """mk_autotune_form over the exact forms: every form is timed, the context
    keeps the fastest, and its gates still equal the oracle's."""
    import torch
    from oracle import oracle as o
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    P = W.toy_params(2)
    keys = oracle_keys(P)
    ctx = B.Context(P, W.CRS_SEED, device=0)
    ctx.import_oracle_keys(keys)
    best, ms = ctx.autotune_form(256, forms=("ntt", "ntt2", "tc"))
    assert set(ms) == {"ntt", "ntt2", "tc"}
    assert best == min(ms, key=ms.get)
    assert ctx.get_form() == B.FORMS[best]
    g, b1, b2 = W.truth_table_inputs()
    c1 = o.encrypt(P, keys, 0, b1, W.encryption_seed(1, 0))
    c2 = o.encrypt(P, keys, 1, b2, W.encryption_seed(1, 1))
    out = torch.zeros((len(g), ctx.W), dtype=torch.int32, device="cuda")
    ctx.gates(to_dev(g.astype(np.uint8)), to_dev(c1), to_dev(c2), out)
    assert np.array_equal(from_dev(out), o.gates(P, keys, g, c1, c2))
    with pytest.raises(B.MkError):
        ctx.autotune_form(256, forms=())
    ctx.close()
