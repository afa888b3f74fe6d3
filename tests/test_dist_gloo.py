"""Multi-rank host logic on CPU ranks (gloo, world size 2): instance sharding
and the max/sum combination of timings that bench.py uses under torchrun."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_1710_02401_gb300 import dist as D, problems as P
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    insts = P.batched_uneven(40, seed=5)
    mine = D.shard(insts, rank, world)
    cost = sum(D.instance_cost(insts[i]) for i in mine)
    t, n = D.combine(1.0 + rank, 100 * (rank + 1))
    dist.destroy_process_group()
    q.put((rank, mine, cost, t, n))


def test_shard_and_combine_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, c0, t0, n0), (r1, m1, c1, t1, n1) = out
    assert sorted(m0 + m1) == list(range(40)) and not set(m0) & set(m1)
    assert m0 == sorted(m0) and m1 == sorted(m1) and (not m0 or not m1 or max(m0) < min(m1))
    assert 0.5 < c0 / c1 < 2.0  # balanced step-matrix traffic
    assert t0 == t1 == 2.0 and n0 == n1 == 300  # max of the times, sum of the solves


def test_shard_edge_cases():
    from paper_1710_02401_gb300 import dist as D, problems as P
    insts = P.batched_uneven(3, seed=1)
    parts = [D.shard(insts, r, 8) for r in range(8)]
    assert sorted(sum(parts, [])) == [0, 1, 2]
    assert D.shard([], 0, 2) == []
    with pytest.raises(ValueError):
        D.shard(insts, 2, 2)


def test_cost_of_antisymmetric_instances_counts_the_stepped_subdomains():
    from paper_1710_02401_gb300 import dist as D
    from paper_1710_02401_gb300 import problems as P
    inst = P.small_tise_2d(L=3).replace(K_d=[6, 7, 8, 7, 6, 9, 8, 9, 5])  # mirror pairs (1,3), (2,6), (5,7) equal
    sym = D.instance_cost(inst)
    anti = D.instance_cost(inst.replace(symmetry="antisymmetric"))
    K2 = [(kd * kd) ** 2 for kd in inst.K_d]
    assert sym == sum(K2)
    assert anti == K2[0] + K2[4] + K2[8] + K2[3] + K2[6] + K2[7]  # diagonal and upper (i1 <= i2) subdomains
