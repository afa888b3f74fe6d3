"""Multi-GPU host logic: independent instances over ranks, timing over ranks.

The Schwarz iteration couples the subdomains of one instance at every step
(global normalisation in imaginary time) and at every window (Robin data);
independent instances do not couple at all (Sec. 5.4 applies per instance).
So a batch is sharded by instance, each rank solves its share with its own
context on its own GPU, and no collective runs on the data path: only the
timing and the solve counts are combined at the end (max of the times, sum of
the counts).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

from . import problems as P


def instance_cost(inst: P.Instance) -> float:
    """Bytes of step matrices one time step streams (sum of K^2 over the stepped
    subdomains; an antisymmetric 2-electron instance steps only the subdomains
    (i1, i2) with i1 <= i2, sid = i1 + L i2, the others being mirror images)."""
    kds = inst.K_d if isinstance(inst.K_d, (list, tuple)) else [inst.K_d] * inst.n_sub
    anti = getattr(inst, "symmetry", "none") == "antisymmetric" and inst.n_elec == 2
    return float(sum((kd ** inst.n_elec) ** 2 for sid, kd in enumerate(kds)
                     if not (anti and sid % inst.L > sid // inst.L)))


def shard(instances: Sequence[P.Instance], rank: int, world: int) -> List[int]:
    """Indices of the instances rank `rank` of `world` solves: contiguous runs
    in input order, cut where the running cost crosses multiples of
    total/world, so every rank gets about the same step-matrix traffic.  The
    shards are disjoint and cover the batch; a rank may get none when there
    are fewer instances than ranks."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    costs = [instance_cost(i) for i in instances]
    total = sum(costs)
    out, cum = [], 0.0
    for idx, c in enumerate(costs):
        mid = cum + 0.5 * c
        r = min(world - 1, int(mid * world / total)) if total > 0 else idx % world
        if r == rank:
            out.append(idx)
        cum += c
    return out


def combine(seconds: float, solves: int, group=None) -> Tuple[float, int]:
    """(max over ranks of the timed seconds, sum over ranks of the subdomain
    solves) for the whole-job throughput; identity without torch.distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return seconds, solves
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    n = torch.tensor([float(solves)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(n, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), int(n.item())
