"""Data-parallel sharding of SF batches over ranks (one process per GPU).

The samples of a batch are independent (every sample is its own fixed-point
problem, Appendix), and so are scenes: a batch is split into contiguous
ranges of its concatenated samples, one range per rank, with no collective on
the data path. A scene cut by a range boundary appears on both ranks with
its own robots' start / goal rows and the samples each rank owns. What
crosses ranks is only the timing (the slowest rank) and, when one consumer
needs every result, an all-gather of the outputs.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch


def sample_ranges(n_samples, rank: int, world: int):
    """Per scene, the [lo, hi) sample range owned by `rank` when the
    concatenated samples are split into `world` contiguous, balanced ranges."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    total = int(sum(int(s) for s in n_samples))
    g_lo, g_hi = total * rank // world, total * (rank + 1) // world
    out, off = [], 0
    for s in n_samples:
        s = int(s)
        out.append((min(max(g_lo - off, 0), s), min(max(g_hi - off, 0), s)))
        off += s
    return out


@dataclass
class Shard:
    xi_bar: torch.Tensor      # flat coefficients of the owned samples, scene by scene
    start: torch.Tensor       # [sum N over kept scenes][dim]
    goal: torch.Tensor
    n_robots: list
    n_samples: list
    scenes: list              # (scene index, lo, hi) per kept scene, hi > lo
    sample_offset: list       # global index of the first owned sample of each kept scene


def shard_batch(xi_bar, start, goal, n_robots, n_samples, dim: int, rank: int, world: int,
                nvar: int = 11) -> Shard:
    """The part of a batch that `rank` of `world` projects: the scenes with
    at least one owned sample, their start / goal rows, and the owned
    samples' coefficients (layout as in the full batch)."""
    xi_flat = xi_bar.reshape(-1)
    ranges = sample_ranges(n_samples, rank, world)
    xs, st, gl, nr, ns, kept, soff = [], [], [], [], [], [], []
    c_off = r_off = s_off = 0
    for q, ((lo, hi), N, S) in enumerate(zip(ranges, n_robots, n_samples)):
        N, S = int(N), int(S)
        per = dim * N * nvar
        if hi > lo:
            xs.append(xi_flat[c_off + lo * per: c_off + hi * per])
            st.append(start[r_off: r_off + N])
            gl.append(goal[r_off: r_off + N])
            nr.append(N)
            ns.append(hi - lo)
            kept.append((q, lo, hi))
            soff.append(s_off + lo)
        c_off += S * per
        r_off += N
        s_off += S
    empty = xi_flat[:0]
    return Shard(xi_bar=torch.cat(xs) if xs else empty,
                 start=torch.cat(st) if st else start[:0], goal=torch.cat(gl) if gl else goal[:0],
                 n_robots=nr, n_samples=ns, scenes=kept, sample_offset=soff)


def max_over_ranks(value: float, device="cpu") -> float:
    """The maximum of `value` over the ranks of the default process group
    (the value itself without one): the timed region of a data-parallel step
    ends when the slowest rank does."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
