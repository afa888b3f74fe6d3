"""Multi-GPU host logic: instances over ranks, one instance's subdomains over
ranks, timing over ranks.

Independent instances do not couple at all (Sec. 5.4 applies per instance):
a batch is sharded by instance, each rank solves its share with its own
context on its own GPU, and no collective runs on the data path; only the
timing and the solve counts are combined at the end (max of the times, sum of
the counts).

The subdomains of ONE instance are independent within a Schwarz iteration
(the local problems of Sec. 5.4 step 2 are solved in parallel; the paper's
complexity remarks count one message exchange per iteration), so one
instance can also be partitioned: contiguous blocks of its L^N subdomain grid
per rank (`partition_subdomains`).  The ranks then exchange

* once per Schwarz iteration, the whole time window of each subdomain's
  contribution to its neighbours' averaged Robin data (Sec. 5.1, Eq. RTC with
  the multi-subdomain average) -- point to point, only between ranks whose
  blocks touch (`exchange_plan`, `exchange_windows`);
* once per imaginary-time step, the per-subdomain partials of the global
  normalisation and of the stop test (system SIT, Sec. 5.2), and once per
  iteration the per-subdomain partials of Res(k) (Eq. residueIT) --
  all-gathered and summed in global subdomain order (`gather_ordered`), so
  that the partitioned run reproduces the single-rank sums bit for bit.

Every run of this build has one GPU, so these routines are exercised on CPU
ranks (gloo) with the CPU oracle's local arithmetic; the CUDA window kernels
have no cross-rank path.
"""
from __future__ import annotations

from typing import Callable, Dict, List, Sequence, Tuple

import numpy as np

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


# ------------------------------------------------- one instance over ranks

def _split(n: int, parts: int) -> List[Tuple[int, int]]:
    """[lo, hi) ranges of n items in `parts` contiguous, near-equal pieces."""
    return [(n * r // parts, n * (r + 1) // parts) for r in range(parts)]


def process_grid(world: int, n_elec: int) -> Tuple[int, ...]:
    """Ranks per coordinate: all along the one coordinate for N = 1, the most
    square factorisation px x py = world for N = 2 (px >= py)."""
    if n_elec == 1:
        return (world,)
    py = int(np.floor(np.sqrt(world)))
    while world % py:
        py -= 1
    return (world // py, py)


def partition_subdomains(L: int, n_elec: int, world: int) -> List[List[int]]:
    """Subdomain ids (sid = i1 + L i2) owned by each rank: the L^N grid cut into
    contiguous blocks, rank r = r1 + px r2 owning i1 in block r1 and i2 in
    block r2.  Blocks are disjoint and cover the grid; with more ranks than
    subdomains along a coordinate some ranks own none."""
    grid = process_grid(world, n_elec)
    ranges = [_split(L, g) for g in grid]
    out: List[List[int]] = [[] for _ in range(world)]
    if n_elec == 1:
        for r, (lo, hi) in enumerate(ranges[0]):
            out[r] = list(range(lo, hi))
        return out
    px, py = grid
    for r2, (b0, b1) in enumerate(ranges[1]):
        for r1, (a0, a1) in enumerate(ranges[0]):
            out[r1 + px * r2] = [i1 + L * i2 for i2 in range(b0, b1) for i1 in range(a0, a1)]
    return out


def owner_map(L: int, n_elec: int, world: int) -> List[int]:
    """Rank owning each subdomain id."""
    own = [-1] * (L ** n_elec)
    for r, sids in enumerate(partition_subdomains(L, n_elec, world)):
        for sid in sids:
            own[sid] = r
    return own


def neighbours(L: int, n_elec: int, sid: int) -> List[int]:
    """Subdomains other than sid in its 3^N block (the only ones whose closure
    can hold interface nodes of sid: overlap bands are narrower than a core)."""
    idx = [sid % L] if n_elec == 1 else [sid % L, sid // L]
    out = []
    if n_elec == 1:
        for d in (-1, 1):
            j = idx[0] + d
            if 0 <= j < L:
                out.append(j)
        return out
    for d2 in (-1, 0, 1):
        for d1 in (-1, 0, 1):
            if d1 == 0 and d2 == 0:
                continue
            j1, j2 = idx[0] + d1, idx[1] + d2
            if 0 <= j1 < L and 0 <= j2 < L:
                out.append(j1 + L * j2)
    return sorted(out)


def exchange_plan(L: int, n_elec: int, world: int) -> Dict[Tuple[int, int], List[Tuple[int, int]]]:
    """Point-to-point messages of one Schwarz iteration: for each ordered rank
    pair (src, dst), src != dst, the (j, i) pairs whose data travel -- j owned
    by src contributes to the Robin data of its neighbour i owned by dst --
    sorted by (i, j), the order both sides use."""
    own = owner_map(L, n_elec, world)
    plan: Dict[Tuple[int, int], List[Tuple[int, int]]] = {}
    for i in range(L ** n_elec):
        for j in neighbours(L, n_elec, i):
            a, b = own[j], own[i]
            if a != b:
                plan.setdefault((a, b), []).append((j, i))
    for k in plan:
        plan[k].sort(key=lambda ji: (ji[1], ji[0]))
    return plan


def exchange_windows(plan: Dict[Tuple[int, int], List[Tuple[int, int]]], rank: int,
                     produce: Callable[[int, int], np.ndarray], group=None) -> Dict[Tuple[int, int], np.ndarray]:
    """One Schwarz iteration's exchange: for every message this rank sends,
    produce(j, i) gives the whole time window of j's contribution at i's
    interface nodes (any float64/complex128 array); the arrays of one message
    travel as one flat buffer after a header of shapes.  Returns the received
    arrays keyed by (j, i).  Deadlock-free: all sends and receives are posted
    non-blocking, then waited for."""
    import torch
    import torch.distributed as dist
    reqs, keep = [], []
    for (a, b), pairs in sorted(plan.items()):
        if a != rank:
            continue
        arrs = [np.ascontiguousarray(produce(j, i)) for j, i in pairs]
        cplx = any(np.iscomplexobj(x) for x in arrs)
        flat = np.concatenate([(x.astype(np.complex128) if cplx else x.astype(np.float64)).ravel() for x in arrs])
        if cplx:
            flat = flat.view(np.float64)
        head = np.array([1.0 if cplx else 0.0] + [float(d) for x in arrs for d in (x.ndim,) + x.shape])
        for buf in (np.array([float(head.size), float(flat.size)]), head, flat):
            t = torch.from_numpy(buf.copy())
            keep.append(t)
            reqs.append(dist.isend(t, dst=b, group=group))
    recv: Dict[Tuple[int, int], np.ndarray] = {}
    incoming = [(a, pairs) for (a, b), pairs in sorted(plan.items()) if b == rank]
    for a, pairs in incoming:
        sizes = torch.zeros(2, dtype=torch.float64)
        dist.recv(sizes, src=a, group=group)
        head = torch.zeros(int(sizes[0].item()), dtype=torch.float64)
        dist.recv(head, src=a, group=group)
        flat = torch.zeros(int(sizes[1].item()), dtype=torch.float64)
        dist.recv(flat, src=a, group=group)
        h = head.numpy()
        cplx = h[0] > 0.5
        data = flat.numpy().view(np.complex128) if cplx else flat.numpy()
        pos, off = 1, 0
        for j, i in pairs:
            nd = int(h[pos])
            shape = tuple(int(x) for x in h[pos + 1:pos + 1 + nd])
            pos += 1 + nd
            n = int(np.prod(shape)) if shape else 1
            recv[(j, i)] = data[off:off + n].reshape(shape).copy()
            off += n
    for r in reqs:
        r.wait()
    return recv


def gather_ordered(values: Dict[int, object], n_items: int, group=None) -> List[object]:
    """All-gather of per-subdomain values (any picklable object: scalars,
    arrays), returned as a list indexed by global subdomain id, so that every
    rank can reduce them in the single-rank order."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        out = [None] * n_items
        for k, v in values.items():
            out[k] = v
        return out
    parts: List[Dict[int, object]] = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, values, group=group)
    out = [None] * n_items
    for part in parts:
        for k, v in part.items():
            out[k] = v
    return out
