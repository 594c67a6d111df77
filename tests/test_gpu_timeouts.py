"""The kernels' bounded waits, run out on purpose without faulting anything.

Three kernels wait on mbarriers for asynchronous copies: the staged blind
rotation (variant 6: each CMux step's key entry, bulk-copied into shared
memory), the cluster latency form (each CTA's key polynomials of the step,
bulk-copied) and the tcgen05 product engine of the tensor form (digit tiles
by TMA).  The test hook mk_debug_fault makes one such copy never be issued, so
the waits for it give up after a short bound; the kernel then lets its own
copies and tensor-core operations finish, records the timeout and returns.
Checked: mk_sync reports MK_ETIMEOUT (once), and the next ordinary gate call
on the same context gives the oracle's ciphertexts word for word.  The
protocols' exits were first checked on the CPU (tests/test_staged_protocol.py,
tests/test_tc05_protocol.py).
"""
import numpy as np
import pytest

from conftest import from_dev, oracle_keys, to_dev

pytestmark = pytest.mark.gpu

WAIT_NS = 50_000_000  # 50 ms


def _toy():
    from oracle import oracle as o
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    P = W.toy_params(2)
    keys = oracle_keys(P)
    ctx = B.Context(P, W.CRS_SEED, device=0)
    ctx.import_oracle_keys(keys)
    g, b1, b2 = W.truth_table_inputs()
    c1 = o.encrypt(P, keys, 0, b1, W.encryption_seed(1, 0))
    c2 = o.encrypt(P, keys, 1, b2, W.encryption_seed(1, 1))
    return P, keys, ctx, g, c1, c2


def _timeout_then_recover(P, keys, ctx, g, c1, c2, kind, arg):
    import torch
    from oracle import oracle as o
    from paper_2205_05825_gb300 import binding as B
    t, a, b = to_dev(g.astype(np.uint8)), to_dev(c1), to_dev(c2)
    out = torch.zeros((len(g), ctx.W), dtype=torch.int32, device="cuda")
    ctx.gates(t, a, b, out)  # keys on the device; a normal call first
    ctx.sync()
    ctx.debug_fault(kind, arg, WAIT_NS)
    ctx.gates(t, a, b, out)
    with pytest.raises(B.MkError, match="MK_ETIMEOUT"):
        ctx.sync()
    ctx.sync()  # the status was cleared: reported once
    ctx.debug_fault("none")
    out.fill_(0)
    ctx.gates(t, a, b, out)
    ctx.sync()
    assert np.array_equal(from_dev(out), o.gates(P, keys, g, c1, c2))


def test_staged_kernel_key_copy_wait_runs_out(gpu_ready):
    P, keys, ctx, g, c1, c2 = _toy()
    ctx.set_form("ntt2")
    ctx.set_variant(6)
    ctx.set_cluster("off")
    _timeout_then_recover(P, keys, ctx, g, c1, c2, "skip_key_step", 5)
    ctx.close()


def test_cluster_kernel_key_copy_wait_runs_out(gpu_ready):
    """The cluster form keeps passing its cluster barriers after a wait runs
    out (no CTA of a cluster may leave early), so only the status tells."""
    P, keys, ctx, g, c1, c2 = _toy()
    ctx.set_form("ntt2")
    ctx.set_cluster("on")
    _timeout_then_recover(P, keys, ctx, g, c1, c2, "skip_key_step", 5)
    ctx.close()


def test_tc05_engine_digit_tile_wait_runs_out(gpu_ready):
    P, keys, ctx, g, c1, c2 = _toy()
    ctx.set_form("tc")
    ctx.set_variant(1)
    _timeout_then_recover(P, keys, ctx, g, c1, c2, "skip_digit_tile", 3)
    ctx.close()
