"""k-point sharding and result gathering across ranks (world size 2, gloo on
CPU).  The per-k solve here is a stand-in that evaluates the homogeneous-medium
closed form (Section 5.1), so only the host-side partition and gather logic is
under test; the GPU solve itself is covered by the parity tests."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import workloads as wl
from paper_1402_6297_gb300 import sharding


def closed_form(k, n=8, nev=4):
    i = np.arange(n)
    s = [4 * np.sin(np.pi * (i + kk) / n) ** 2 * n ** 2 for kk in k]
    disp = np.sqrt(s[2][:, None, None] + s[1][None, :, None] + s[0][None, None, :]).ravel()
    return np.sort(np.concatenate([disp, disp]))[:nev]


def test_shard_bounds_partition():
    for count in (0, 1, 5, 48, 49):
        for world in (1, 2, 3, 8):
            spans = [sharding.shard_bounds(count, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == count
            for (a, b), (c, d) in zip(spans, spans[1:]):
                assert b == c
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        sharding.shard_bounds(4, 2, 2)


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ks = wl.bz_path_midpoints(9)
    seen = []

    def solve(k):
        seen.append(tuple(k))
        return closed_form(k)
    res = sharding.band_structure(ks, solve, rank, world)
    out.put((rank, [list(map(float, r)) for r in res], seen))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_band_structure_two_ranks_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ks = wl.bz_path_midpoints(9)
    ref = [closed_form(k) for k in ks]
    solved = []
    for rank, res, seen in results:
        assert len(res) == len(ks)
        for a, b in zip(res, ref):
            assert np.allclose(a, b, rtol=0, atol=0)
        solved.extend(seen)
    # every k-point solved exactly once across the two ranks
    assert sorted(solved) == sorted(tuple(k) for k in ks)
