"""mk_gates_noalloc: gates with a fixed, library-owned scratch and no device
allocation, for callers that cannot let the library allocate while they run
(memory reserved up front, or no allocation allowed in a latency-critical
loop).  Collected last on purpose, so that a run stopping at the first
failure has already run every other test.

The checks: the output equals mk_gates (the ordinary entry point) word for
word on two calls in a row with different inputs, and the oracle's gates on
the same inputs; every product form and the cluster (latency) kernel;
the device's free memory is the same before and after the calls; oversize
batches and a context whose keys are not yet on the device are refused
before any launch.
"""
import numpy as np
import pytest

from conftest import from_dev, oracle_keys, to_dev

pytestmark = pytest.mark.gpu


def _setup(params, G, config_id, keys=None):
    """A context and 2G random gates; with oracle keys the inputs are the
    oracle's encryptions, otherwise the library's."""
    import torch
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    ctx = B.Context(params, W.CRS_SEED, device=0)
    types, b1, b2 = W.random_gates(G, config_id=config_id)
    if keys is not None:
        from oracle import oracle as o
        ctx.import_oracle_keys(keys)
        c1 = o.encrypt(params, keys, 0, b1, W.encryption_seed(config_id, 0))
        c2 = o.encrypt(params, keys, 1, b2, W.encryption_seed(config_id, 1))
    else:
        for i, s in enumerate(W.party_seeds(params["k"])):
            ctx.keygen(i, s)
        c1 = ctx.encrypt(0, b1, W.encryption_seed(config_id, 0))
        c2 = ctx.encrypt(1, b2, W.encryption_seed(config_id, 1))
    return ctx, torch, types, c1, c2, b1, b2


def _two_calls(ctx, torch, types, c1, c2, G):
    """mk_gates on 2G gates, one set-up call of mk_gates_noalloc, then
    mk_gates_noalloc on each half; returns the reference, the two no-alloc
    outputs and the free device memory before and after those two calls."""
    t, a, b = to_dev(types.astype(np.uint8)), to_dev(c1), to_dev(c2)
    ref = torch.zeros((2 * G, ctx.W), dtype=torch.int32, device="cuda")
    ctx.gates(t, a, b, ref)  # ordinary entry point; also puts the keys on the device
    outs = [torch.full((G, ctx.W), -1, dtype=torch.int32, device="cuda") for _ in range(2)]
    halves = [(t[c * G:(c + 1) * G].contiguous(), a[c * G:(c + 1) * G].contiguous(),
               b[c * G:(c + 1) * G].contiguous()) for c in range(2)]
    # The first call on a device is its set-up: it looks up the fixed array's
    # address, which (with lazy module loading) is when the array's module is
    # loaded and the array reserved.  Free memory is compared after it.
    scratch_out = torch.zeros_like(outs[0])
    ctx.gates_noalloc(*halves[0], scratch_out)
    ctx.sync()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for call in range(2):  # two calls in a row on different halves: no stale scratch
        ctx.gates_noalloc(*halves[call], outs[call])
        ctx.sync()
    free1 = torch.cuda.mem_get_info()[0]
    return from_dev(ref), [from_dev(o) for o in outs], free0, free1


@pytest.mark.parametrize("which", ["toy", "full"])
def test_noalloc_matches_mk_gates_and_oracle_twice(gpu_ready, which):
    from oracle import oracle as o
    from paper_2205_05825_gb300 import workloads as W
    P = W.toy_params(2) if which == "toy" else W.full_params(2)
    keys = oracle_keys(P)
    G = 200
    ctx, torch, types, c1, c2, _, _ = _setup(P, 2 * G, 11, keys)
    ref, outs, free0, free1 = _two_calls(ctx, torch, types, c1, c2, G)
    assert free1 == free0  # the calls allocated no device memory
    for call in range(2):
        assert np.array_equal(outs[call], ref[call * G:(call + 1) * G])
    # against the oracle: every gate at the toy size, two sampled gates per call at full size
    idx = np.arange(G) if which == "toy" else np.array([0, G - 1])
    for call in range(2):
        sel = call * G + idx
        assert np.array_equal(outs[call][idx], o.gates(P, keys, types[sel], c1[sel], c2[sel]))
    ctx.close()


@pytest.mark.parametrize("form", ["ntt", "tc", "fft"])
def test_noalloc_every_form(gpu_ready, form):
    """Toy size: each product form's mk_gates_noalloc equals its mk_gates word
    for word (the FFT form runs the same kernel in both calls) and decrypts
    to the truth table; no device memory is allocated by the calls."""
    from paper_2205_05825_gb300 import workloads as W
    P = W.toy_params(2)
    G = 100
    ctx, torch, types, c1, c2, b1, b2 = _setup(P, 2 * G, 13)
    ctx.set_form(form)
    ref, outs, free0, free1 = _two_calls(ctx, torch, types, c1, c2, G)
    assert free1 == free0
    for call in range(2):
        assert np.array_equal(outs[call], ref[call * G:(call + 1) * G])
    exp = np.array([[x & y, x | y, 1 - (x & y), 1 - (x | y), x ^ y, 1 - (x ^ y)][int(tt)]
                    for tt, x, y in zip(types, b1.astype(int), b2.astype(int))], np.uint8)
    assert np.array_equal(ctx.decrypt(to_dev(np.concatenate(outs))), exp)
    ctx.close()


def test_noalloc_cluster_kernel(gpu_ready):
    """Small batches run the cluster (latency) kernel; mk_gates_noalloc takes
    the same path and gives the oracle's ciphertexts."""
    from oracle import oracle as o
    from paper_2205_05825_gb300 import workloads as W
    P = W.toy_params(2)
    keys = oracle_keys(P)
    G = 6
    ctx, torch, types, c1, c2, _, _ = _setup(P, 2 * G, 14, keys)
    ctx.set_cluster("on")
    ref, outs, free0, free1 = _two_calls(ctx, torch, types, c1, c2, G)
    assert free1 == free0
    for call in range(2):
        sel = slice(call * G, (call + 1) * G)
        assert np.array_equal(outs[call], ref[sel])
        assert np.array_equal(outs[call], o.gates(P, keys, types[sel], c1[sel], c2[sel]))
    ctx.close()


def test_noalloc_refuses_oversize_and_missing_keys(gpu_ready):
    import torch
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    P = W.full_params(2)
    ctx, torch, types, c1, c2, _, _ = _setup(P, 4, 12)
    t, a, b = to_dev(types.astype(np.uint8)), to_dev(c1), to_dev(c2)
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
