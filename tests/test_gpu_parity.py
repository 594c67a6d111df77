"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

The NTT form is exact, so every ciphertext word must be equal (bit-exact),
stage by stage: mod switch, blind rotation after 1, 2 and all CMux steps,
SampleExtract, key switch, whole gates, NOT (Eq. 8).  Keys and inputs come
from the oracle (seeded); nothing the GPU computes feeds the oracle.
"""
import numpy as np
import pytest

from conftest import from_dev, oracle_keys, to_dev

pytestmark = pytest.mark.gpu

TRUTH = {0: lambda a, b: a & b, 1: lambda a, b: a | b, 2: lambda a, b: 1 - (a & b),
         3: lambda a, b: 1 - (a | b), 4: lambda a, b: a ^ b, 5: lambda a, b: 1 - (a ^ b)}


def _ctx(params, keys):
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    ctx = B.Context(params, W.CRS_SEED, device=0)
    ctx.import_oracle_keys(keys)
    return ctx


def _inputs(params, keys, types, b1, b2, config_id):
    from oracle import oracle as o
    from paper_2205_05825_gb300 import workloads as W
    c1 = o.encrypt(params, keys, 0, b1, W.encryption_seed(config_id, 0))
    c2 = o.encrypt(params, keys, min(1, params["k"] - 1), b2, W.encryption_seed(config_id, 1))
    return c1, c2


@pytest.fixture(scope="module")
def toy(gpu_ready):
    from paper_2205_05825_gb300 import workloads as W
    P = W.toy_params(2)
    keys = oracle_keys(P)
    g, b1, b2 = W.truth_table_inputs()
    c1, c2 = _inputs(P, keys, g, b1, b2, 1)
    return P, keys, _ctx(P, keys), g, b1, b2, c1, c2


def test_toy_truth_tables_bit_exact(toy):
    """Config 1: 6 gates x 4 input pairs, each ciphertext byte-equal to the oracle."""
    import torch
    from oracle import oracle as o
    P, keys, ctx, g, b1, b2, c1, c2 = toy
    ref = o.gates(P, keys, g, c1, c2)
    out = torch.zeros((len(g), ctx.W), dtype=torch.int32, device="cuda")
    ctx.gates(to_dev(g.astype(np.uint8)), to_dev(c1), to_dev(c2), out)
    got = from_dev(out)
    assert np.array_equal(got, ref)
    exp = np.array([TRUTH[int(t)](int(x), int(y)) for t, x, y in zip(g, b1, b2)], np.uint8)
    assert np.array_equal(ctx.decrypt(out), exp)
    assert np.array_equal(o.decrypt(P, keys, got), exp)


def test_toy_uniform_gate_entry(toy):
    """mk_gate (one type for the batch) equals the oracle for every type."""
    import torch
    from oracle import oracle as o
    P, keys, ctx, g, b1, b2, c1, c2 = toy
    for ty in range(6):
        sel = np.nonzero(g == ty)[0]
        out = torch.zeros((len(sel), ctx.W), dtype=torch.int32, device="cuda")
        ctx.gate(ty, to_dev(c1[sel]), to_dev(c2[sel]), out)
        ref = o.gates(P, keys, g[sel], c1[sel], c2[sel])
        assert np.array_equal(from_dev(out), ref), ty


def test_toy_not_exact(toy):
    """MKNOT (Eq. 8): (0, 1/4) - c, word for word, no bootstrapping."""
    import torch
    from oracle import oracle as o
    P, keys, ctx, g, b1, b2, c1, c2 = toy
    src = np.concatenate([c1[:2], c2[:2]])
    out = torch.zeros((4, ctx.W), dtype=torch.int32, device="cuda")
    ctx.mk_not(to_dev(src), out)
    got = from_dev(out)
    for r in range(4):
        assert np.array_equal(got[r], o.mk_not(P, src[r]))
    assert np.array_equal(ctx.decrypt(out), 1 - o.decrypt(P, keys, src))


def test_toy_stages(toy):
    """Mod switch, CMux #1 and #2, full blind rotation, extract, key switch."""
    import torch
    from oracle import oracle as o
    from paper_2205_05825_gb300 import binding as B
    P, keys, ctx, g, b1, b2, c1, c2 = toy
    lin = B.lin_records(g)
    lin_d = to_dev(lin)
    abar = torch.zeros((len(g), ctx.W), dtype=torch.int32, device="cuda")
    ctx.stage_modswitch(lin_d, to_dev(c1), to_dev(c2), abar)
    lins = np.stack([o.gate_linear(P, int(t), x, y) for t, x, y in zip(g, c1, c2)])
    ref_abar = o.modswitch_input(P, lins)
    assert np.array_equal(from_dev(abar), ref_abar)
    sel = slice(0, 8)
    for steps in (1, 2, 37, -1):
        acc = torch.zeros((8, 3, P["N"]), dtype=torch.int32, device="cuda")
        ctx.stage_blind_rotate(abar[sel].contiguous(), steps, acc)
        ref = o.blind_rotate(P, keys, ref_abar[sel], max_steps=steps)
        assert np.array_equal(from_dev(acc), ref), steps
    ext = torch.zeros((len(g), ctx.E), dtype=torch.int32, device="cuda")
    ctx.stage_bootstrap(lin_d, to_dev(c1), to_dev(c2), ext)
    ref_ext = o.bootstrap(P, keys, lins)
    assert np.array_equal(from_dev(ext), ref_ext)
    out = torch.zeros((len(g), ctx.W), dtype=torch.int32, device="cuda")
    ctx.stage_keyswitch(ext, out)
    assert np.array_equal(from_dev(out), o.keyswitch(P, keys, ref_ext))


def test_toy_ragged_batches_and_linear_records(toy):
    """Chunked launches (batch 5 over 28 gates), empty batch, single gate, and
    general linear records with folded NOTs (scalars in [-2, 2])."""
    import torch
    from oracle import oracle as o
    P, keys, ctx, g, b1, b2, c1, c2 = toy
    rng = np.random.default_rng(7)
    cnt = 13
    lin = np.zeros((cnt, 3), np.int32)
    lin[:, 0] = rng.integers(0, 8, cnt).astype(np.uint32).view(np.int32) << 29
    lin[:, 1] = rng.choice([-2, -1, 1, 2], cnt)
    lin[:, 2] = rng.choice([-2, -1, 0, 1, 2], cnt)
    ctx.set_batch(5)
    try:
        out = torch.zeros((cnt, ctx.W), dtype=torch.int32, device="cuda")
        ctx.gates_lin(to_dev(lin), to_dev(c1[:cnt]), to_dev(c2[:cnt]), out)
        ref = np.stack([o.keyswitch(P, keys, o.bootstrap(P, keys, o.lin_comb(
            P, int(lin[r, 0]) & 0xFFFFFFFF, int(lin[r, 1]), c1[r], int(lin[r, 2]), c2[r])))[0]
            for r in range(cnt)])
        assert np.array_equal(from_dev(out), ref)
        empty = torch.zeros((0, ctx.W), dtype=torch.int32, device="cuda")
        ctx.gate(0, empty, empty, empty)
        one = torch.zeros((1, ctx.W), dtype=torch.int32, device="cuda")
        ctx.gate(4, to_dev(c1[:1]), to_dev(c2[:1]), one)
        assert np.array_equal(from_dev(one)[0], o.gates(P, keys, np.array([4]), c1[:1], c2[:1])[0])
    finally:
        ctx.set_batch(4096)


def test_toy_product_keygen_matches_oracle_on_gpu(toy):
    """Keys generated by the library (mk_keygen) give the same gate outputs."""
    import torch
    from oracle import oracle as o
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    P, keys, ctx, g, b1, b2, c1, c2 = toy
    c2x = B.Context(P, W.CRS_SEED, device=0)
    for i, s in enumerate(W.party_seeds(2)):
        c2x.keygen(i, s)
    out = torch.zeros((len(g), ctx.W), dtype=torch.int32, device="cuda")
    c2x.gates(to_dev(g.astype(np.uint8)), to_dev(c1), to_dev(c2), out)
    assert np.array_equal(from_dev(out), o.gates(P, keys, g, c1, c2))


@pytest.fixture(scope="module")
def full2(gpu_ready):
    from paper_2205_05825_gb300 import workloads as W
    P = W.full_params(2)
    keys = oracle_keys(P)
    return P, keys, _ctx(P, keys)


def test_full_k2_sampled_bit_exact_and_all_decrypt(full2):
    """Config 2 shape (n=560, N=1024, k=2), 4096 random gates in the batched
    launch: 12 sampled gates byte-equal to the oracle, all 4096 decrypt to the
    truth table."""
    import torch
    from oracle import oracle as o
    from paper_2205_05825_gb300 import workloads as W
    P, keys, ctx = full2
    G = 4096
    types, b1, b2 = W.random_gates(G)
    c1 = o.encrypt(P, keys, 0, b1, W.encryption_seed(2, 0))
    c2 = o.encrypt(P, keys, 1, b2, W.encryption_seed(2, 1))
    out = torch.zeros((G, ctx.W), dtype=torch.int32, device="cuda")
    ctx.gates(to_dev(types.astype(np.uint8)), to_dev(c1), to_dev(c2), out)
    got = from_dev(out)
    exp = np.array([TRUTH[int(t)](int(x), int(y)) for t, x, y in zip(types, b1, b2)], np.uint8)
    assert np.array_equal(ctx.decrypt(out), exp)
    idx = np.array([0, 1, 2, 3, 511, 1024, 2047, 2048, 3000, 4093, 4094, 4095])
    ref = o.gates(P, keys, types[idx], c1[idx], c2[idx])
    assert np.array_equal(got[idx], ref)


FORM_VARIANTS = [(f, v) for f in ("ntt", "ntt2") for v in range(9)] + [("tc", 0), ("tc", 1)]


@pytest.mark.parametrize("form,variant", FORM_VARIANTS)
def test_toy_every_variant_bit_exact(toy, form, variant):
    """Each exact product form (Goldilocks NTT, two-prime NTT, tensor cores)
    and each kernel variant gives the oracle's ciphertexts."""
    import torch
    from oracle import oracle as o
    P, keys, ctx, g, b1, b2, c1, c2 = toy
    ctx.set_form(form)
    ctx.set_variant(variant)
    ctx.set_cluster("off")  # the batched kernel's variants, not the latency form
    try:
        out = torch.zeros((len(g), ctx.W), dtype=torch.int32, device="cuda")
        ctx.gates(to_dev(g.astype(np.uint8)), to_dev(c1), to_dev(c2), out)
        assert np.array_equal(from_dev(out), o.gates(P, keys, g, c1, c2))
        acc = torch.zeros((4, 3, P["N"]), dtype=torch.int32, device="cuda")
        abar = to_dev(o.modswitch_input(P, np.stack([o.gate_linear(P, int(t), x, y)
                                                     for t, x, y in zip(g[:4], c1[:4], c2[:4])])))
        ctx.stage_blind_rotate(abar, 3, acc)
        ref = o.blind_rotate(P, keys, from_dev(abar), max_steps=3)
        assert np.array_equal(from_dev(acc), ref)
    finally:
        ctx.set_form("ntt2")
        ctx.set_variant(2)
        ctx.set_cluster("auto")


@pytest.mark.parametrize("form,variant", FORM_VARIANTS)
def test_full_k2_every_variant_sampled(full2, form, variant):
    """Full size (n=560, N=1024, k=2): each variant, 96 gates (a ragged last
    wave), 3 sampled gates byte-equal to the oracle, all 96 decrypt."""
    import torch
    from oracle import oracle as o
    from paper_2205_05825_gb300 import workloads as W
    P, keys, ctx = full2
    G = 96
    types, b1, b2 = W.random_gates(G, config_id=7)
    c1 = o.encrypt(P, keys, 0, b1, W.encryption_seed(7, 0))
    c2 = o.encrypt(P, keys, 1, b2, W.encryption_seed(7, 1))
    ctx.set_form(form)
    ctx.set_variant(variant)
    ctx.set_cluster("off")
    try:
        out = torch.zeros((G, ctx.W), dtype=torch.int32, device="cuda")
        ctx.gates(to_dev(types.astype(np.uint8)), to_dev(c1), to_dev(c2), out)
        got = from_dev(out)
    finally:
        ctx.set_form("ntt2")
        ctx.set_variant(2)
        ctx.set_cluster("auto")
    exp = np.array([TRUTH[int(t)](int(x), int(y)) for t, x, y in zip(types, b1, b2)], np.uint8)
    assert np.array_equal(o.decrypt(P, keys, got), exp)
    idx = np.array([0, 50, 95])
    assert np.array_equal(got[idx], o.gates(P, keys, types[idx], c1[idx], c2[idx]))


def test_full_k4_sampled_bit_exact(gpu_ready):
    """Four parties (n=560, N=1024, k=4) with joint-key inputs, so all 4*560
    CMux steps run: 64 gates decrypt, 2 sampled gates byte-equal."""
    import torch
    from oracle import oracle as o
    from paper_2205_05825_gb300 import workloads as W
    P = W.full_params(4)
    keys = oracle_keys(P)
    ctx = _ctx(P, keys)
    G = 64
    types, b1, b2 = W.random_gates(G, config_id=4)
    c1 = o.encrypt_joint(P, keys, b1, W.encryption_seed(4, 0))
    c2 = o.encrypt_joint(P, keys, b2, W.encryption_seed(4, 1))
    out = torch.zeros((G, ctx.W), dtype=torch.int32, device="cuda")
    ctx.gates(to_dev(types.astype(np.uint8)), to_dev(c1), to_dev(c2), out)
    got = from_dev(out)
    exp = np.array([TRUTH[int(t)](int(x), int(y)) for t, x, y in zip(types, b1, b2)], np.uint8)
    assert np.array_equal(ctx.decrypt(out), exp)
    idx = np.array([0, 63])
    assert np.array_equal(got[idx], o.gates(P, keys, types[idx], c1[idx], c2[idx]))
    ctx.close()


@pytest.mark.parametrize("count", [63, 64, 65, 100])
def test_toy_keyswitch_batch_boundaries(toy, count):
    """Key switch through the per-gate kernel (< 64 gates) and the batched
    kernel (>= 64: groups of 32 gates, a ragged last group), word for word."""
    import torch
    from oracle import oracle as o
    P, keys, ctx = toy[:3]
    rng = np.random.default_rng(count)
    ext = rng.integers(0, 2 ** 32, size=(count, ctx.E), dtype=np.uint64).astype(np.uint32)
    out = torch.zeros((count, ctx.W), dtype=torch.int32, device="cuda")
    ctx.stage_keyswitch(to_dev(ext), out)
    assert np.array_equal(from_dev(out), o.keyswitch(P, keys, ext))


@pytest.mark.parametrize("form", ["ntt", "ntt2"])
def test_toy_cluster_form_stages_bit_exact(toy, form):
    """The latency (cluster) form of the blind rotation, forced on: blind
    rotation after 0, 1, 2, 37 and all steps, whole gates, word for word."""
    import torch
    from oracle import oracle as o
    P, keys, ctx, g, b1, b2, c1, c2 = toy
    ctx.set_form(form)
    ctx.set_cluster("on")
    try:
        lins = np.stack([o.gate_linear(P, int(t), x, y) for t, x, y in zip(g, c1, c2)])
        ref_abar = o.modswitch_input(P, lins)
        abar = to_dev(ref_abar)
        for steps in (0, 1, 2, 37, -1):
            acc = torch.zeros((len(g), 3, P["N"]), dtype=torch.int32, device="cuda")
            ctx.stage_blind_rotate(abar, steps, acc)
            assert np.array_equal(from_dev(acc), o.blind_rotate(P, keys, ref_abar, max_steps=steps)), steps
        out = torch.zeros((len(g), ctx.W), dtype=torch.int32, device="cuda")
        ctx.gates(to_dev(g.astype(np.uint8)), to_dev(c1), to_dev(c2), out)
        assert np.array_equal(from_dev(out), o.gates(P, keys, g, c1, c2))
    finally:
        ctx.set_form("ntt2")
        ctx.set_cluster("auto")


@pytest.mark.parametrize("k", [1, 3])
def test_toy_cluster_form_party_counts(gpu_ready, k):
    """The cluster form's digit split at the party counts the other tests do
    not reach: k = 1 (two CTAs, CTA 0 transforms digits 0 and 2 of w) and
    k = 3 (CTA 3 takes no digit).  Joint-key gates forced through the form,
    word for word against the oracle and the batched kernel."""
    import torch
    from oracle import oracle as o
    from paper_2205_05825_gb300 import workloads as W
    P = W.toy_params(k)
    keys = oracle_keys(P)
    ctx = _ctx(P, keys)
    G = 12
    types, b1, b2 = W.random_gates(G, config_id=80 + k)
    c1 = o.encrypt_joint(P, keys, b1, W.encryption_seed(80 + k, 0))
    c2 = o.encrypt_joint(P, keys, b2, W.encryption_seed(80 + k, 1))
    d = (to_dev(types.astype(np.uint8)), to_dev(c1), to_dev(c2))
    outs = {}
    for form in ("ntt2", "ntt"):
        ctx.set_form(form)
        for mode in ("on", "off"):
            ctx.set_cluster(mode)
            out = torch.zeros((G, ctx.W), dtype=torch.int32, device="cuda")
            ctx.gates(*d, out)
            outs[form, mode] = from_dev(out)
    ref = o.gates(P, keys, types, c1, c2)
    for v in outs.values():
        assert np.array_equal(v, ref)
    ctx.close()


@pytest.mark.parametrize("k", [2, 4, 7])
def test_full_cluster_form_sampled(gpu_ready, k):
    """Full size, cluster form forced on, joint-key inputs (all k*n steps):
    every gate decrypts, sampled gates byte-equal to the oracle, and the
    batched kernel gives the same ciphertexts."""
    import torch
    from oracle import oracle as o
    from paper_2205_05825_gb300 import workloads as W
    P = W.full_params(k)
    keys = oracle_keys(P)
    ctx = _ctx(P, keys)
    G = 16
    types, b1, b2 = W.random_gates(G, config_id=60 + k)
    c1 = o.encrypt_joint(P, keys, b1, W.encryption_seed(60 + k, 0))
    c2 = o.encrypt_joint(P, keys, b2, W.encryption_seed(60 + k, 1))
    d = (to_dev(types.astype(np.uint8)), to_dev(c1), to_dev(c2))
    outs = {}
    for mode in ("on", "off"):
        ctx.set_cluster(mode)
        out = torch.zeros((G, ctx.W), dtype=torch.int32, device="cuda")
        ctx.gates(*d, out)
        outs[mode] = from_dev(out)
    assert np.array_equal(outs["on"], outs["off"])
    exp = np.array([TRUTH[int(t)](int(x), int(y)) for t, x, y in zip(types, b1, b2)], np.uint8)
    assert np.array_equal(o.decrypt(P, keys, outs["on"]), exp)
    if k <= 4:  # the schoolbook oracle needs minutes per gate beyond that
        idx = np.array([0])
        assert np.array_equal(outs["on"][idx], o.gates(P, keys, types[idx], c1[idx], c2[idx]))
    ctx.close()
