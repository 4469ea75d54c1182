"""Multi-GPU use of the eigensolver: independent Bloch problems per rank.

A band structure (Section 5.3 sweeps k along G-X-M-R-G) is a set of
independent eigenproblems, one per k-point.  The only parallelism that fits
the method is therefore across k-points: each rank solves its own contiguous
share, and the eigenvalues are gathered at the end.  There is no collective
on the data path; the gather moves nev doubles per k-point.
"""

from __future__ import annotations

from typing import Callable, List, Sequence, Tuple


def shard_bounds(count: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous, balanced [start, stop) share of `count` items for `rank`."""
    if world <= 0 or not (0 <= rank < world):
        raise ValueError("bad rank / world size")
    base, extra = divmod(count, world)
    start = rank * base + min(rank, extra)
    stop = start + base + (1 if rank < extra else 0)
    return start, stop


def gather_results(local: List[Tuple[int, Sequence[float]]], world: int):
    """All ranks' (index, eigenvalues) pairs, ordered by index (needs an
    initialised torch.distributed process group when world > 1)."""
    if world == 1:
        merged = list(local)
    else:
        import torch.distributed as dist
        parts = [None] * world
        dist.all_gather_object(parts, list(local))
        merged = [item for part in parts for item in part]
    merged.sort(key=lambda t: t[0])
    return merged


def band_structure(kpoints: Sequence[Sequence[float]], solve: Callable[[Sequence[float]], Sequence[float]],
                   rank: int = 0, world: int = 1):
    """Solve this rank's share of `kpoints` with `solve(k) -> eigenvalues`
    and return every k-point's eigenvalues, in k-point order, on every rank.

    On GPUs `solve` is typically
        lambda k: nfs.Context(grid, k, medium, precision="mixed").eigs(nev, vectors=False)[0]
    with each rank bound to its own device."""
    start, stop = shard_bounds(len(kpoints), rank, world)
    local = [(i, [float(x) for x in solve(kpoints[i])]) for i in range(start, stop)]
    return [vals for _, vals in gather_results(local, world)]
