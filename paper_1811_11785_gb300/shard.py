"""Frame sharding across GPUs (one process per GPU).

SVD-PHAT localises every frame independently (Algorithm 1's online steps see one frame at
a time), so N GPUs split a batch of T frames into N contiguous ranges, each rank holding a
replica of the offline basis (V, D, the k-d tree: a few MB).  There is no exchange on the
data path; the only collective is the final gather of the per-frame results (index and
scores, 12 bytes per frame) when the caller wants them on every rank.
"""
from __future__ import annotations


def shard_range(T: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [lo, hi) frame range of ``rank``; sizes differ by at most one frame."""
    if world < 1 or not (0 <= rank < world) or T < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(T, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def localize_sharded(localize_fn, frames_host, T: int, group=None):
    """Run ``localize_fn(frames_host[lo:hi]) -> (idx, score, proj)`` (CPU tensors) on this
    rank's shard and all-gather the results into full-length tensors on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    lo, hi = shard_range(T, rank, world)
    idx, score, proj = localize_fn(frames_host[lo:hi])
    if world == 1:
        return idx, score, proj
    sizes = [shard_range(T, r, world) for r in range(world)]
    n_max = max(h - l for l, h in sizes)

    def gather(x, dtype):
        buf = torch.zeros(n_max, dtype=dtype)
        if x is not None:
            buf[: hi - lo] = x
        parts = [torch.empty(n_max, dtype=dtype) for _ in range(world)]
        dist.all_gather(parts, buf, group=group)
        return torch.cat([p[: h - l] for p, (l, h) in zip(parts, sizes)])

    return gather(idx, torch.int32), gather(score, torch.float32), gather(proj, torch.float32)
