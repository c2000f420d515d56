"""Host-side sharding of relabellings across ranks (one process per GPU).

Rows of the permutation testing matrix are independent and exceedance counts
are sums over rows, so a study shards by relabellings with no exchange on the
data path: each rank runs the library on its own contiguous row range and the
per-rank results are merged once at the end (concatenate maxima, sum counts).
RapidPT recovery keys every random draw by the global row index, so a split of
rows gives exactly what one device gives.
"""
import torch
import torch.distributed as dist


def shard_rows(P, world, rank):
    """Contiguous [start, stop) of P rows for ``rank`` of ``world`` (first ranks
    take one more row when P does not divide evenly)."""
    base, extra = divmod(int(P), int(world))
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def merge_maxnull(local, P, group=None):
    """Concatenate every rank's per-relabelling outputs (maxima or argmax; its
    rows of shard_rows) into a P-vector."""
    world = dist.get_world_size(group)
    size = max(shard_rows(P, world, r)[1] - shard_rows(P, world, r)[0] for r in range(world))
    fill = float("-inf") if local.dtype.is_floating_point else -1
    buf = torch.full((size,), fill, dtype=local.dtype, device=local.device)
    buf[:local.numel()] = local
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    out = []
    for r in range(world):
        a, b = shard_rows(P, world, r)
        out.append(parts[r][:b - a])
    return torch.cat(out)


def merge_counts(local, group=None):
    """Sum every rank's per-voxel exceedance counts (int64 on the wire)."""
    tot = local.to(torch.int64).clone()
    dist.all_reduce(tot, op=dist.ReduceOp.SUM, group=group)
    return tot
