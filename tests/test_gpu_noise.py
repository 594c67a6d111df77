"""Output noise of bootstrapped gates at the full-size presets, measured on
many gates: the GPU path is bit-exact to the oracle, so its outputs carry
the oracle's noise; their phases are computed on the host by the oracle
(Sec. 3.2's SymDec phase).  The presets' rule (the largest RLWE sigma of the
ladder with an XOR margin of at least six standard deviations: the input
phase of XOR carries 2 (e1 - e2), against the 1/8 half-width of the
decision window) is checked on 1024 joint-key gates per party count, so all
k n CMux steps run."""
import math

import numpy as np
import pytest

from conftest import oracle_keys, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k", [2, 4])
def test_full_preset_output_noise_margin(gpu_ready, k):
    import torch
    from oracle import noise as Nz
    from oracle import oracle as o
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    P = W.full_params(k)
    keys = oracle_keys(P)
    ctx = B.Context(P, W.CRS_SEED, device=0)
    ctx.import_oracle_keys(keys)
    G = 1024
    types, b1, b2 = W.random_gates(G, config_id=91)
    c1 = o.encrypt_joint(P, keys, b1, W.encryption_seed(91, 0))
    c2 = o.encrypt_joint(P, keys, b2, W.encryption_seed(91, 1))
    out = torch.zeros((G, ctx.W), dtype=torch.int32, device="cuda")
    ctx.gates(to_dev(types.astype(np.uint8)), to_dev(c1), to_dev(c2), out)
    got = out.cpu().numpy().view(np.uint32)
    e = Nz.output_errors(P, keys, types, b1, b2, got)
    sd = float(np.sqrt(np.mean(e * e)))
    z = 0.125 / (2.0 * math.sqrt(2.0) * sd)
    assert np.max(np.abs(e)) < 0.125  # every output decrypts
    assert z >= 6.0, (k, sd, z)
    ctx.close()
