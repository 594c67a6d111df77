"""mk_gates_noalloc: gates with a fixed, library-owned scratch and no device
allocation, for callers that cannot let the library allocate while they run
(memory reserved up front, or no allocation allowed in a latency-critical
loop).  Collected last on purpose, so that a run stopping at the first
failure has already run every other test.

The checks: the output equals mk_gates (the ordinary entry point) word for
word on two calls in a row with different inputs; oversize batches and a
context whose keys are not yet on the device are refused before any launch.
"""
import numpy as np
import pytest

from conftest import from_dev, to_dev

pytestmark = pytest.mark.gpu


def _setup(params, G, config_id):
    import torch
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    ctx = B.Context(params, W.CRS_SEED, device=0)
    for i, s in enumerate(W.party_seeds(params["k"])):
        ctx.keygen(i, s)
    types, b1, b2 = W.random_gates(G, config_id=config_id)
    c1 = ctx.encrypt(0, b1, W.encryption_seed(config_id, 0))
    c2 = ctx.encrypt(1, b2, W.encryption_seed(config_id, 1))
    return ctx, torch, to_dev(types.astype(np.uint8)), to_dev(c1), to_dev(c2)


@pytest.mark.parametrize("which", ["toy", "full"])
def test_noalloc_matches_mk_gates_twice(gpu_ready, which):
    from paper_2205_05825_gb300 import workloads as W
    P = W.toy_params(2) if which == "toy" else W.full_params(2)
    G = 200
    ctx, torch, t, a, b = _setup(P, 2 * G, 11)
    ref = torch.zeros((2 * G, ctx.W), dtype=torch.int32, device="cuda")
    ctx.gates(t, a, b, ref)  # ordinary entry point; also puts the keys on the device
    for call in range(2):  # two calls in a row on different halves: no stale scratch
        sl = slice(call * G, (call + 1) * G)
        out = torch.full((G, ctx.W), -1, dtype=torch.int32, device="cuda")
        ctx.gates_noalloc(t[sl].contiguous(), a[sl].contiguous(), b[sl].contiguous(), out)
        ctx.sync()
        assert np.array_equal(from_dev(out), from_dev(ref[sl]))
    ctx.close()


def test_noalloc_refuses_oversize_and_missing_keys(gpu_ready):
    import torch
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    P = W.full_params(2)
    ctx, torch, t, a, b = _setup(P, 4, 12)
    out = torch.zeros((4, ctx.W), dtype=torch.int32, device="cuda")
    with pytest.raises(B.MkError, match="MK_ESTATE"):
        ctx.gates_noalloc(t, a, b, out)  # keys not uploaded yet
    ctx.gates(t, a, b, out)
    cap = ((4 << 20) - 256) // (4 * ctx.E + 24)
    assert cap == 510
    big = torch.zeros(cap + 1, dtype=torch.uint8, device="cuda")
    big_ct = torch.zeros((cap + 1, ctx.W), dtype=torch.int32, device="cuda")
    with pytest.raises(B.MkError, match="exceeds the fixed scratch capacity"):
        ctx.gates_noalloc(big, big_ct, big_ct, big_ct)
    ctx.close()
