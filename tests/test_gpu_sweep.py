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
            word_err = np.abs(signed32(got[idx].astype(np.int64) - ref.astype(np.int64)))
            print("\nsweep k=%d fft: output phase error vs oracle max %d torus32 units (2^%.1f), "
                  "%.1f %% of output words bit-identical" % (k, d.max(), np.log2(max(d.max(), 1)),
                                                             100.0 * np.mean(word_err == 0)))
        else:
            assert np.array_equal(got[idx], ref), form
    ctx.close()


def test_full_k8_largest_batch(gpu_ready):
    """Eight parties, 4097 joint-key gates: two launches (4096 + 1) at the
    largest per-launch batch; every gate decrypts, and the gate in the second
    launch equals the same gate bootstrapped on its own."""
    import torch
    from oracle import oracle as o
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    P = W.full_params(8)
    keys = oracle_keys(P)
    ctx = B.Context(P, W.CRS_SEED, device=0)
    ctx.import_oracle_keys(keys)
    G = 4097
    types, b1, b2 = W.random_gates(G, config_id=88)
    c1 = o.encrypt_joint(P, keys, b1, W.encryption_seed(88, 0))
    c2 = o.encrypt_joint(P, keys, b2, W.encryption_seed(88, 1))
    d_t, d1, d2 = to_dev(types.astype(np.uint8)), to_dev(c1), to_dev(c2)
    out = torch.zeros((G, ctx.W), dtype=torch.int32, device="cuda")
    ctx.gates(d_t, d1, d2, out)
    exp = np.array([TRUTH[int(t)](int(x), int(y)) for t, x, y in zip(types, b1, b2)], np.uint8)
    assert np.array_equal(ctx.decrypt(out), exp)
    one = torch.zeros((1, ctx.W), dtype=torch.int32, device="cuda")
    ctx.gates(d_t[4096:], d1[4096:], d2[4096:], one)
    assert np.array_equal(from_dev(one)[0], from_dev(out)[4096])
    ctx.close()
