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
