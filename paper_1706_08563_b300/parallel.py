"""Sharding of the simulation over several processes (one per GPU).

The path shards into independent problems: probes are independent (a
multislice probe, or a PRISM output probe given the S-matrix), and so are
frozen-phonon configurations.  Each rank computes a contiguous block of probes
(or a subset of configurations) and the only exchange is one gather of the
[probe, ring] outputs (or one sum over configurations) at the end.  There is no
collective inside the slice loop.

PRISM splits in two ("PRISM Probe Simulations": every plane wave is propagated
through the sample on its own): each rank builds a contiguous block of the
S-matrix beams into a zeroed buffer, one all-reduce assembles the whole
S-matrix on every rank (the S-matrix keeps beams on its fastest axis, so a
rank's block is not contiguous in memory; the sum adds only zeros to each
value, so it is exact in every storage type and acts as the all-gather of the
blocks), and then each rank computes the output of its block of probes, which
one gather of the rings collects.  Remote data lands in each rank's own memory
before any kernel reads it.

These helpers take the per-rank computation as a callable, so the same code
drives libstem on GPUs (NCCL) and any CPU computation under the gloo backend.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Sequence, Tuple

import torch
import torch.distributed as dist


def shard_range(n: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous block [start, stop) of n items for `rank`; sizes differ by at most 1."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank / world size")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def config_shards(n_configs: int, rank: int, world: int) -> List[int]:
    """Frozen-phonon configurations handled by `rank` (round robin)."""
    return list(range(rank, n_configs, world))


def _rank_world(group=None) -> Tuple[int, int]:
    """(rank, world size); one process without a process group is rank 0 of 1."""
    if not dist.is_available() or not dist.is_initialized():
        return 0, 1
    return dist.get_rank(group), dist.get_world_size(group)


def gather_rows(local: torch.Tensor, n_total: int, group=None) -> torch.Tensor:
    """All-gather per-rank row blocks (from shard_range) into the full [n_total, ...] array."""
    world = _rank_world(group)[1]
    if world == 1:
        return local
    sizes = [shard_range(n_total, r, world) for r in range(world)]
    width = max(b - a for a, b in sizes)
    pad = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[: b - a] for p, (a, b) in zip(parts, sizes)], dim=0)


def sharded_probes(n_probes: int, compute: Callable[[int, int], torch.Tensor], group=None) -> torch.Tensor:
    """Run compute(start, stop) -> [stop - start, n_rings] on this rank's probe block
    and return the full [n_probes, n_rings] output on every rank."""
    rank, world = _rank_world(group)
    a, b = shard_range(n_probes, rank, world)
    return gather_rows(compute(a, b), n_probes, group)


def sharded_configs(n_configs: int, compute: Callable[[int], torch.Tensor], group=None,
                    like: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Mean over frozen-phonon configurations, configurations spread over ranks:
    compute(c) -> rings of configuration c; one all-reduce sum at the end."""
    rank, world = _rank_world(group)
    acc = None if like is None else torch.zeros_like(like)
    for c in config_shards(n_configs, rank, world):
        r = compute(c)
        acc = r.clone() if acc is None else acc + r
    if acc is None:
        raise ValueError("give `like` when a rank may own no configuration")
    if world > 1:
        dist.all_reduce(acc, op=dist.ReduceOp.SUM, group=group)
    return acc / n_configs


def sharded_smatrix(n_beams: int, build: Callable[[int, int], None], parts: Sequence[torch.Tensor],
                    group=None) -> None:
    """Zero the S-matrix (`parts`: typed views that cover its buffer, e.g. the
    float32 scales and the 16-bit values, so that each sum runs in its own
    type), build this rank's block of beams with build(b0, b1), which writes
    only beams [b0, b1), then sum every part over the ranks in place: every rank
    ends with the whole S-matrix."""
    rank, world = _rank_world(group)
    b0, b1 = shard_range(n_beams, rank, world)
    for t in parts:
        t.zero_()
    build(b0, b1)
    if world > 1:
        for t in parts:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)


def sharded_prism(n_beams: int, n_probes: int, build: Callable[[int, int], None], parts: Sequence[torch.Tensor],
                  output: Callable[[int, int], torch.Tensor], group=None) -> torch.Tensor:
    """The PRISM split: beams sharded for the S-matrix (one all-reduce per part
    assembles it), then probes sharded for the output step (one gather):
    output(start, stop) -> [stop - start, n_rings] rings from the whole S-matrix."""
    sharded_smatrix(n_beams, build, parts, group)
    return sharded_probes(n_probes, output, group)
