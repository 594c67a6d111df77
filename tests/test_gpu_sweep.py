"""Precision sweep (config 4 shape): full-size parameters at 2, 4 and 8
parties, joint-key inputs so that all k*n CMux steps run, through every
product form.  Exact forms: sampled outputs byte-equal to the oracle.  FP64
FFT: phase within 1/32 of the oracle's.  Every gate of every form decrypts
to its truth table."""
import numpy as np
import pytest

from conftest import from_dev, oracle_keys, to_dev
from polyref import signed32

pytestmark = pytest.mark.gpu

TRUTH = {0: lambda a, b: a & b, 1: lambda a, b: a | b, 2: lambda a, b: 1 - (a & b),
         3: lambda a, b: 1 - (a | b), 4: lambda a, b: a ^ b, 5: lambda a, b: 1 - (a ^ b)}
SAMPLED = {2: 4, 4: 2, 8: 1}


@pytest.mark.parametrize("k", [2, 4, 8])
def test_sweep_forms_against_oracle(gpu_ready, k):
    import torch
    from oracle import oracle as o
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    P = W.full_params(k)
    keys = oracle_keys(P)
    ctx = B.Context(P, W.CRS_SEED, device=0)
    ctx.import_oracle_keys(keys)
    G = 128
    types, b1, b2 = W.random_gates(G, config_id=40 + k)
    c1 = o.encrypt_joint(P, keys, b1, W.encryption_seed(40 + k, 0))
    c2 = o.encrypt_joint(P, keys, b2, W.encryption_seed(40 + k, 1))
    exp = np.array([TRUTH[int(t)](int(x), int(y)) for t, x, y in zip(types, b1, b2)], np.uint8)
    idx = np.arange(SAMPLED[k])
    ref = o.gates(P, keys, types[idx], c1[idx], c2[idx])
    for form in ("ntt", "ntt2", "fft", "tc"):
        ctx.set_form(form)
        out = torch.zeros((G, ctx.W), dtype=torch.int32, device="cuda")
        ctx.gates(to_dev(types.astype(np.uint8)), to_dev(c1), to_dev(c2), out)
        got = from_dev(out)
        assert np.array_equal(o.decrypt(P, keys, got), exp), form
        if form == "fft":
            d = np.abs(signed32(o.phase(P, keys, got[idx]).astype(np.int64) - o.phase(P, keys, ref).astype(np.int64)))
            assert d.max() < 1 << 27
        else:
            assert np.array_equal(got[idx], ref), form
    ctx.close()
