"""k-bit operators on the GPU (levelised netlists, one batched launch pair per
level) against native two's-complement arithmetic, and word-for-word against
the oracle evaluating its own (identical) netlist."""
import numpy as np
import pytest

from conftest import from_dev, oracle_keys, to_dev
from test_circuits import decode, expected, operands, valid_div

pytestmark = pytest.mark.gpu


def _ctx(P, keys):
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    ctx = B.Context(P, W.CRS_SEED, device=0)
    ctx.import_oracle_keys(keys)
    return ctx


def _run(ctx, op, k, ca, cb):
    import torch
    pairs = ca.shape[0]
    da, db = to_dev(ca), to_dev(cb)
    if op == "div":
        q = torch.zeros((pairs, k, ctx.W), dtype=torch.int32, device="cuda")
        r = torch.zeros_like(q)
        ctx.div_kbit(k, da, db, q, r)
        return np.concatenate([from_dev(q), from_dev(r)], axis=1)
    nout = 2 * k if op == "mul" else k
    out = torch.zeros((pairs, nout, ctx.W), dtype=torch.int32, device="cuda")
    getattr(ctx, op + "_kbit")(k, da, db, out)
    return from_dev(out)


def _encrypt_operands(P, keys, a, b, k, seed):
    from oracle import oracle as o
    from paper_2205_05825_gb300 import workloads as W
    ca = o.encrypt(P, keys, 0, W.int_to_bits(a, k).ravel(), seed).reshape(len(a), k, -1)
    cb = o.encrypt(P, keys, 1, W.int_to_bits(b, k).ravel(), seed + 1).reshape(len(a), k, -1)
    return ca, cb


def _check(P, keys, op, k, a, b, out):
    from oracle import oracle as o
    bits = o.decrypt(P, keys, out.reshape(-1, out.shape[-1])).reshape(len(a), -1)
    got = decode(op, bits, k)
    if op == "div":
        ok = valid_div(a, b, k)
        exp = expected(op, a[ok], b[ok], k)
        assert np.array_equal(got[0][ok], exp[0]) and np.array_equal(got[1][ok], exp[1])
    else:
        assert np.array_equal(got, expected(op, a, b, k))


@pytest.fixture(scope="module")
def toy(gpu_ready):
    from paper_2205_05825_gb300 import workloads as W
    P = W.toy_params(2)
    keys = oracle_keys(P)
    return P, keys, _ctx(P, keys)


STYLES = ["array", "shallow", "paper", "nand"]


@pytest.mark.parametrize("style", STYLES)
@pytest.mark.parametrize("op", ["add", "sub", "mul", "div"])
def test_toy_4bit_exhaustive(toy, op, style):
    """All 256 pairs of 4-bit operands in one levelised batch (toy set), with
    each netlist family."""
    P, keys, ctx = toy
    a, b = operands(4)
    ca, cb = _encrypt_operands(P, keys, a, b, 4, 700)
    ctx.set_circuit_style(style)
    try:
        _check(P, keys, op, 4, a, b, _run(ctx, op, 4, ca, cb))
    finally:
        ctx.set_circuit_style("array")


@pytest.mark.parametrize("style", STYLES)
@pytest.mark.parametrize("op", ["add", "sub", "mul", "div"])
def test_toy_4bit_bit_exact_vs_oracle(toy, op, style):
    """Three pairs, every output ciphertext word equal to the oracle's
    evaluation of its own netlist of the same family (the shallow family has
    gates with constant inputs folded away and pruned, renumbered wires)."""
    from oracle import circuits as C
    P, keys, ctx = toy
    a = np.array([-8, 5, -1], np.int64)
    b = np.array([3, -7, 2], np.int64)
    ca, cb = _encrypt_operands(P, keys, a, b, 4, 710)
    ctx.set_circuit_style(style)
    try:
        got = _run(ctx, op, 4, ca, cb)
    finally:
        ctx.set_circuit_style("array")
    ref = C.eval_encrypted(P, keys, C.build(op, 4, style), ca, cb)
    assert np.array_equal(got, ref)


@pytest.fixture(scope="module")
def full2(gpu_ready):
    from paper_2205_05825_gb300 import workloads as W
    P = W.full_params(2)
    keys = oracle_keys(P)
    return P, keys, _ctx(P, keys)


# Full size (config 3): every operator at 8 and 16 bits for both netlist
# families at two parties, and at four parties with the shallow family (few
# pairs: a call costs its netlist depth in launches whatever its width); the
# paper's 0/1/2-adder multiplier and the NAND-only family.
FULL_CASES = ([("array", 2, op, 8, pr) for op, pr in (("add", 64), ("sub", 64), ("mul", 32), ("div", 16))] +
              [("array", 2, op, 16, pr) for op, pr in (("add", 16), ("sub", 16), ("mul", 8), ("div", 4))] +
              [("shallow", 2, op, kb, 8) for kb in (8, 16) for op in ("add", "sub", "mul", "div")] +
              [("shallow", 4, op, kb, 4) for kb in (8, 16) for op in ("add", "sub", "mul", "div")] +
              [("array", 4, op, 8, 16) for op in ("add", "sub", "mul", "div")] +
              [("paper", 2, "mul", 8, 16), ("paper", 2, "mul", 16, 4), ("paper", 4, "mul", 8, 4),
               ("nand", 2, "add", 8, 8), ("nand", 2, "mul", 8, 4)])


@pytest.fixture(scope="module")
def full4(gpu_ready):
    from paper_2205_05825_gb300 import workloads as W
    P = W.full_params(4)
    keys = oracle_keys(P)
    ctx = _ctx(P, keys)
    yield P, keys, ctx
    ctx.close()


@pytest.mark.parametrize("style,parties,op,k,pairs", FULL_CASES)
def test_full_random_pairs(full2, full4, style, parties, op, k, pairs):
    """Full-size parameters, random signed operands: every output decrypts to
    the native two's-complement result (b = 0 and the one overflowing
    quotient excluded for the divider)."""
    from paper_2205_05825_gb300 import workloads as W
    P, keys, ctx = full2 if parties == 2 else full4
    a, b = W.random_operands(k, pairs, config_id=3)
    if op == "div":
        b = np.where(b == 0, 1, b)
    ca, cb = _encrypt_operands(P, keys, a, b, k, 720 + k)
    ctx.set_circuit_style(style)
    try:
        out = _run(ctx, op, k, ca, cb)
    finally:
        ctx.set_circuit_style("array")
    _check(P, keys, op, k, a, b, out)


def test_full_k2_2bit_add_bit_exact_vs_oracle(full2):
    """Full size, two pairs: every output ciphertext word of the 2-bit adder
    of the shallow family equals the oracle's evaluation of the same netlist
    (the oracle needs about 10 s per full-size gate and core, and an adder's
    levels are one to three gates wide, so wider adders are checked by
    decryption above and word for word at the toy size)."""
    from oracle import circuits as C
    P, keys, ctx = full2
    a = np.array([-2, 1], np.int64)
    b = np.array([1, 1], np.int64)
    ca, cb = _encrypt_operands(P, keys, a, b, 2, 760)
    ctx.set_circuit_style("shallow")
    try:
        got = _run(ctx, "add", 2, ca, cb)
    finally:
        ctx.set_circuit_style("array")
    ref = C.eval_encrypted(P, keys, C.build("add", 2, "shallow"), ca, cb)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("op", ["add", "mul"])
def test_toy_graph_replay_matches_direct_launches(toy, op):
    """The level loop replayed as a captured CUDA graph (twice, so the second
    call replays the cached graph), launched directly, and launched under
    timing (which bypasses graphs) give the same ciphertexts; a form change
    re-captures."""
    P, keys, ctx = toy
    a = np.array([-8, 5, -1, 7, 0], np.int64)
    b = np.array([3, -7, 2, -8, 1], np.int64)
    ca, cb = _encrypt_operands(P, keys, a, b, 4, 720)
    ctx.set_graphs(True)
    g1 = _run(ctx, op, 4, ca, cb)
    g2 = _run(ctx, op, 4, ca, cb)
    ctx.set_graphs(False)
    direct = _run(ctx, op, 4, ca, cb)
    ctx.set_graphs(True)
    ctx.timing_enable(True)
    timed_ = _run(ctx, op, 4, ca, cb)
    ctx.timing_enable(False)
    ctx.set_form("ntt")
    other_form = _run(ctx, op, 4, ca, cb)
    ctx.set_form("ntt2")
    assert np.array_equal(g1, direct) and np.array_equal(g2, direct) and np.array_equal(timed_, direct)
    assert np.array_equal(other_form, direct)
    _check(P, keys, op, 4, a, b, g1)


@pytest.mark.parametrize("style", ["array", "shallow"])
@pytest.mark.parametrize("op", ["add", "sub", "mul", "div"])
def test_toy_persistent_launch_bit_exact(toy, op, style):
    """The whole netlist in one persistent launch (gates waiting for their own
    input wires, no level barrier) gives the level loop's ciphertexts and the
    oracle's, word for word."""
    from oracle import circuits as C
    P, keys, ctx = toy
    a = np.array([-8, 5, -1, 7], np.int64)
    b = np.array([3, -7, 2, -8], np.int64)
    ca, cb = _encrypt_operands(P, keys, a, b, 4, 730)
    ctx.set_circuit_style(style)
    try:
        ctx.set_circuit_exec("persistent")
        got = _run(ctx, op, 4, ca, cb)
        got2 = _run(ctx, op, 4, ca, cb)  # a second call: new epoch, same plan
        ctx.set_circuit_exec("levels")
        lev = _run(ctx, op, 4, ca, cb)
        ctx.sync()
    finally:
        ctx.set_circuit_exec("auto")
        ctx.set_circuit_style("array")
    assert np.array_equal(got, lev) and np.array_equal(got2, lev)
    ref = C.eval_encrypted(P, keys, C.build(op, 4, style), ca[:2], cb[:2])
    assert np.array_equal(got[:2], ref)


@pytest.mark.parametrize("op,pairs", [("add", 64), ("mul", 16)])
def test_full_k2_persistent_launch_equals_levels(full2, op, pairs):
    """Full size: the persistent launch and the level loop give the same
    ciphertexts, which decrypt to the native results."""
    from paper_2205_05825_gb300 import workloads as W
    P, keys, ctx = full2
    a, b = W.random_operands(8, pairs, config_id=34)
    ca, cb = _encrypt_operands(P, keys, a, b, 8, 770)
    try:
        ctx.set_circuit_exec("persistent")
        got = _run(ctx, op, 8, ca, cb)
        ctx.set_circuit_exec("levels")
        lev = _run(ctx, op, 8, ca, cb)
        ctx.sync()
    finally:
        ctx.set_circuit_exec("auto")
    assert np.array_equal(got, lev)
    _check(P, keys, op, 8, a, b, got)


def test_toy_persistent_launch_wait_runs_out(toy):
    """A wire that is never marked ready (test hook): the gates reading it
    give up after the bound, mk_sync reports MK_ETIMEOUT once, and the next
    call on the same context is bit-exact again."""
    from oracle import circuits as C
    from paper_2205_05825_gb300 import binding as B
    P, keys, ctx = toy
    a = np.array([-8, 5], np.int64)
    b = np.array([3, -7], np.int64)
    ca, cb = _encrypt_operands(P, keys, a, b, 4, 740)
    try:
        ctx.set_circuit_exec("persistent")
        ctx.debug_fault("skip_wire_ready", 0, 50_000_000)  # item 0: a first-level gate of the adder
        _run(ctx, "add", 4, ca, cb)
        with pytest.raises(B.MkError, match="MK_ETIMEOUT"):
            ctx.sync()
        ctx.sync()
        ctx.debug_fault("none")
        got = _run(ctx, "add", 4, ca, cb)
        ctx.sync()
    finally:
        ctx.debug_fault("none")
        ctx.set_circuit_exec("auto")
    assert np.array_equal(got, C.eval_encrypted(P, keys, C.build("add", 4), ca, cb))
