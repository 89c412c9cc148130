"""World-size-2 gloo test of the multi-GPU host logic on CPU: each rank localises its own
contiguous shard of frames (here with a stand-in per-frame function, since the CPU has no
GPU) and the results are gathered on every rank, in order, with nothing lost or repeated."""
import os
import socket

import pytest
import torch
import torch.multiprocessing as mp

from paper_1811_11785_gb300.shard import localize_sharded, shard_range


def test_shard_range_partitions():
    for T in [0, 1, 7, 100, 65536]:
        for world in [1, 2, 3, 8]:
            spans = [shard_range(T, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == T
            for (a, b), (c, d) in zip(spans, spans[1:]):
                assert b == c
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _fake_localize(frames):
    # stands in for sp.localize_host: a deterministic function of each frame alone
    v = frames.real.sum(dim=(1, 2))
    return (v * 10).to(torch.int32), v.float(), (2 * v).float()


def _worker(rank, world, port, T, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = torch.Generator().manual_seed(5)
    frames = torch.randn(T, 3, 5, generator=g, dtype=torch.complex64)
    idx, score, proj = localize_sharded(_fake_localize, frames, T)
    ref = _fake_localize(frames)
    ok = torch.equal(idx, ref[0]) and torch.equal(score, ref[1]) and torch.equal(proj, ref[2])
    q.put((rank, ok, int(idx.numel())))
    dist.destroy_process_group()


@pytest.mark.parametrize("T", [101, 8])
def test_gloo_world2_gather(T):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, T, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(r for r, _, _ in res) == [0, 1]
    assert all(ok for _, ok, _ in res)
    assert all(n == T for _, _, n in res)
