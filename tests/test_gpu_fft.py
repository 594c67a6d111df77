"""The FP64 FFT product form (approximate).  Checked against the oracle as
C-12 of the design reading states: (i) after one CMux step every accumulator
coefficient is within 2^12 torus32 units of the oracle's (the per-product
tolerance; a flipped gadget digit is allowed in at most one gate of the
sample), (ii) every gate decrypts to its truth table, (iii) the phase
difference to the oracle's output stays far inside the 1/8 margin."""
import numpy as np
import pytest

from conftest import from_dev, oracle_keys, to_dev
from polyref import signed32

pytestmark = pytest.mark.gpu

TRUTH = {0: lambda a, b: a & b, 1: lambda a, b: a | b, 2: lambda a, b: 1 - (a & b),
         3: lambda a, b: 1 - (a | b), 4: lambda a, b: a ^ b, 5: lambda a, b: 1 - (a ^ b)}


def _ctx(P, keys):
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    ctx = B.Context(P, W.CRS_SEED, device=0)
    ctx.import_oracle_keys(keys)
    ctx.set_form("fft")
    return ctx


@pytest.mark.parametrize("which", ["toy", "full"])
def test_fft_one_cmux_step_within_tolerance(gpu_ready, which):
    import torch
    from oracle import oracle as o
    from paper_2205_05825_gb300 import workloads as W
    P = W.toy_params(2) if which == "toy" else W.full_params(2)
    keys = oracle_keys(P)
    ctx = _ctx(P, keys)
    rng = np.random.default_rng(5)
    G = 16
    abar = rng.integers(1, 2 * P["N"], (G, ctx.W)).astype(np.uint32)
    acc = torch.zeros((G, 3, P["N"]), dtype=torch.int32, device="cuda")
    ctx.stage_blind_rotate(to_dev(abar), 1, acc)
    ref = o.blind_rotate(P, keys, abar, max_steps=1)
    err = np.abs(signed32(from_dev(acc).astype(np.int64) - ref.astype(np.int64))).reshape(G, -1).max(axis=1)
    assert (err <= 1 << 12).sum() >= G - 1, err
    ctx.close()


@pytest.mark.parametrize("which", ["toy", "full"])
def test_fft_gates_decrypt_and_phase_close(gpu_ready, which):
    import torch
    from oracle import oracle as o
    from paper_2205_05825_gb300 import workloads as W
    P = W.toy_params(2) if which == "toy" else W.full_params(2)
    keys = oracle_keys(P)
    ctx = _ctx(P, keys)
    G = 96 if which == "toy" else 256
    types, b1, b2 = W.random_gates(G, config_id=41)
    c1 = o.encrypt(P, keys, 0, b1, W.encryption_seed(41, 0))
    c2 = o.encrypt(P, keys, 1, b2, W.encryption_seed(41, 1))
    out = torch.zeros((G, ctx.W), dtype=torch.int32, device="cuda")
    ctx.gates(to_dev(types.astype(np.uint8)), to_dev(c1), to_dev(c2), out)
    got = from_dev(out)
    exp = np.array([TRUTH[int(t)](int(x), int(y)) for t, x, y in zip(types, b1, b2)], np.uint8)
    assert np.array_equal(o.decrypt(P, keys, got), exp)
    idx = np.arange(0, G, G // 8)
    ref = o.gates(P, keys, types[idx], c1[idx], c2[idx])
    dphi = np.abs(signed32(o.phase(P, keys, got[idx]).astype(np.int64) - o.phase(P, keys, ref).astype(np.int64)))
    assert dphi.max() < 1 << 27  # 1/32 of the torus, a quarter of the decision margin
    ctx.close()
