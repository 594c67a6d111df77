"""Replicas across GPUs: one process per GPU, each with its own context and a
copy of the keys, each evaluating its own share of a batch of independent
gates (or of independent operator requests).

Gates of one batch (and of one netlist level) do not depend on each other,
so a batch splits across GPUs with no exchange on the data path; only a
caller that wants every output in one process gathers them afterwards (one
all-gather of the output rows, k n + 1 words each).  Under torchrun every
rank calls the same functions with its RANK / WORLD_SIZE.
"""
import os


def dist_env():
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_range(count, rank, world):
    """[start, end) of rank's share of `count` items: contiguous, in rank
    order, sizes differing by at most one, covering every item once."""
    if world < 1 or not 0 <= rank < world or count < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(count, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def gates_sharded(ctx, types, a, b, out, rank, world):
    """Evaluate this rank's share of a gate batch (device tensors: types
    uint8 [count], a and b [count][k n + 1], out [count][k n + 1]); the other
    rows of `out` are left untouched.  Returns (start, end)."""
    start, end = shard_range(types.shape[0], rank, world)
    if end > start:
        ctx.gates(types[start:end].contiguous(), a[start:end].contiguous(), b[start:end].contiguous(),
                  out[start:end])
    return start, end


def gather_rows(out, rank, world, group=None):
    """All-gather every rank's share of `out` (a tensor of rows whose share
    of rank r is rows shard_range(rows, r, world)) into every rank's `out`,
    with torch.distributed (any backend that supports all_gather)."""
    import torch
    import torch.distributed as dist
    if world == 1:
        return out
    rows = out.shape[0]
    spans = [shard_range(rows, r, world) for r in range(world)]
    width = max(e - s for s, e in spans)
    send = torch.zeros((width,) + tuple(out.shape[1:]), dtype=out.dtype, device=out.device)
    s0, e0 = spans[rank]
    send[:e0 - s0] = out[s0:e0]
    recv = [torch.empty_like(send) for _ in range(world)]
    dist.all_gather(recv, send, group=group)
    for r, (s, e) in enumerate(spans):
        out[s:e] = recv[r][:e - s]
    return out
