"""Multi-GPU is replicas only: each rank bootstraps its own independent batch
of gates, and the benchmark takes the max time over ranks.  The host logic
(rank environment, per-rank input shards, max-reduction, barrier) is checked
here with two gloo ranks on the CPU."""
import os
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    from paper_2205_05825_gb300 import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    seed = bench.shard_seed(2, r)
    types, b1, b2 = W.random_gates(64, config_id=seed)
    t = bench.reduce_max(10.0 + rank, w)
    bench.barrier(w)
    q.put((r, w, lr, seed, types.tolist(), t))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, s0, t0, m0), (r1, w1, l1, s1, t1, m1) = res
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert s0 != s1 and t0 != t1  # each rank draws its own independent gates
    assert m0 == m1 == 11.0       # max over ranks


def test_shard_ranges_cover_every_item_once():
    sys.path.insert(0, ROOT)
    from paper_2205_05825_gb300 import replicas as R
    for count in (0, 1, 7, 64, 4096, 4097):
        for world in (1, 2, 3, 8):
            spans = [R.shard_range(count, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == count
            assert all(spans[r][1] == spans[r + 1][0] for r in range(world - 1))
            sizes = [e - s for s, e in spans]
            assert max(sizes) - min(sizes) <= 1


class _FakeCtx:
    """Stands in for a context on the CPU: a 'gate' writes the gate type plus
    the row's first word into every word of its output row."""

    def gates(self, types, a, b, out):
        out[:] = (types.to(out.dtype)[:, None] + a[:, :1]).expand_as(out)


def _shard_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    from paper_2205_05825_gb300 import replicas as R
    dist.init_process_group("gloo", rank=rank, world_size=world)
    count, W = 37, 5
    types = torch.arange(count, dtype=torch.uint8) % 6
    a = torch.arange(count * W, dtype=torch.int32).reshape(count, W)
    out = torch.full((count, W), -1, dtype=torch.int32)
    s, e = R.gates_sharded(_FakeCtx(), types, a, a, out, rank, world)
    untouched = bool((out[:s] == -1).all() and (out[e:] == -1).all())
    R.gather_rows(out, rank, world)
    q.put((rank, s, e, untouched, out.tolist()))
    dist.destroy_process_group()


def test_two_gloo_ranks_evaluate_their_shares_and_gather():
    """Each rank evaluates only its rows; the all-gather puts every row, in
    order, in every rank's output."""
    import torch
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 30500 + os.getpid() % 1000
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, e0, u0, o0), (r1, s1, e1, u1, o1) = res
    assert (s0, e0, s1, e1) == (0, 19, 19, 37) and u0 and u1
    count, W = 37, 5
    types = torch.arange(count, dtype=torch.int32) % 6
    a = torch.arange(count * W, dtype=torch.int32).reshape(count, W)
    expect = (types[:, None] + a[:, :1]).expand(count, W).tolist()
    assert o0 == expect and o1 == expect
