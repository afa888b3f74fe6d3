"""One instance partitioned over CPU ranks (gloo, world size 2).

The host logic of paper_1710_02401_gb300/dist.py -- contiguous blocks of the
subdomain grid per rank, one point-to-point exchange per Schwarz iteration of
whole-window Robin contributions between ranks whose blocks touch, per-step
all-gathers of the normalisation and stop-test partials, and the residual's
partials summed in global order -- composed with the CPU oracle's local
arithmetic (each rank assembles and steps only its own subdomains).  The
partitioned run must reproduce the single-rank oracle bit for bit: window
lengths, Res(k) and energies compare with ==.
"""
import math
import os
import socket
import types

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _light_local(O, inst, sid):
    """What the exchange needs of a subdomain this rank does not own: its basis
    (with the same per-coordinate reduction), its interface nodes and their
    contributors -- no Galerkin matrices."""
    raw = O.Basis(inst, sid)
    basis = O.Basis(inst, sid, [O.orth_coordinate(O.overlap_1d(inst, raw, d), inst.orth_tau) for d in range(raw.N)])
    gam = O.gamma_nodes(inst, sid)
    contrib = [[j for j in range(inst.n_sub) if j != sid and O.contains_closed(inst, j, x)] for x in gam.X]
    return types.SimpleNamespace(basis=basis, gamma=gam, contrib=contrib)


def partitioned_swr(inst, rank, world, kmax):
    """Imaginary-time SWR (Sec. 5.4 steps 1-5) with this rank's subdomains."""
    import scipy.linalg as sla
    from oracle import swr_oracle as O
    from paper_1710_02401_gb300 import dist as D
    S = inst.n_sub
    mine = D.partition_subdomains(inst.L, inst.n_elec, world)[rank]
    plan = D.exchange_plan(inst.L, inst.n_elec, world)
    locs = [O.build_local(inst, s) if s in mine else _light_local(O, inst, s) for s in range(S)]
    ops = O.TraceOps(inst, locs)
    kappa, dt, mu = inst.kinetic, inst.dt, inst.mu

    def norm2(vecs, mats):  # sum_i c_i^T M_i c_i over all subdomains, in subdomain order
        parts = D.gather_ordered({i: np.vdot(vecs[i], mats[i] @ vecs[i]) for i in mine}, S)
        return float(np.real(sum(parts)))

    achi = {i: locs[i].Achi for i in mine}
    c0 = {i: locs[i].c0.astype(float) for i in mine}
    s0 = math.sqrt(norm2(c0, achi))
    c0 = {i: c / s0 for i, c in c0.items()}
    lu = {i: sla.lu_factor(locs[i].A + dt * locs[i].Ht) for i in mine}
    g_prev, n_prev, u_prev = None, 0, None
    records = []
    for k in range(1, kmax + 1):
        def g_at(i, n):
            if g_prev is None:
                return np.zeros(locs[i].gamma.w.size)
            return g_prev[i][min(n, n_prev)]

        coeffs = dict(c0)
        hist, hist_raw = [coeffs], [coeffs]
        n_done = 0
        for n in range(inst.max_steps):
            new = {}
            for i in mine:
                l = locs[i]
                b = l.own_vals.T @ (l.gamma.w * g_at(i, n + 1))
                new[i] = sla.lu_solve(lu[i], l.A @ coeffs[i] + kappa * dt * b)
            raw = new
            s = math.sqrt(norm2(new, achi))
            new = {i: c / s for i, c in new.items()}
            n_done = n + 1
            hist_raw.append(raw)
            diff = {i: new[i] - coeffs[i] for i in mine}
            coeffs = new
            hist.append(coeffs)
            if math.sqrt(max(0.0, norm2(diff, achi))) <= inst.ngf_tol:
                break
        # whole-window Robin contributions of j at i's interface nodes (Eq. RTC)
        def contribution(j, i):
            rows, vals, ders = ops.ops[i][0][j]
            return np.array([(ders @ h[j]) + mu * (vals @ h[j]) for h in hist_raw])

        recv = D.exchange_windows(plan, rank, contribution)
        g_new, u_hist = {}, {}
        for i in mine:
            per_j, cnt = ops.ops[i]
            G = cnt.size
            steps = []
            for n in range(n_done + 1):
                g = np.zeros(G)
                for j, (rows, _v, _d) in per_j.items():
                    x = recv[(j, i)] if (j, i) in recv else contribution(j, i)
                    g[rows] += x[n]
                with np.errstate(invalid="ignore", divide="ignore"):
                    g = np.where(cnt > 0, g / np.maximum(cnt, 1), 0.0)
                steps.append(g)
            g_new[i] = np.array(steps)
            u_hist[i] = np.array([locs[i].own_vals @ h[i] for h in hist])
        # Res(k): per-subdomain terms, accumulated in the single-rank order
        n_cmp = max(n_done, 0 if u_prev is None else n_prev)
        terms = {}
        for i in mine:
            w = locs[i].gamma.w
            t = []
            for n in range(1, n_cmp + 1):
                a = u_hist[i][min(n, n_done)]
                b = np.zeros_like(a) if u_prev is None else u_prev[i][min(n, n_prev)]
                t.append(dt * float(np.sum(w * np.abs(a - b) ** 2)))
            terms[i] = t
        r2 = 0.0
        for t in D.gather_ordered(terms, S):
            for x in t:
                r2 += x
        num = D.gather_ordered({i: np.vdot(coeffs[i], locs[i].Hchi @ coeffs[i]) for i in mine}, S)
        energy = float(np.real(sum(num))) / norm2(coeffs, achi)
        records.append((n_done, math.sqrt(r2), energy))
        g_prev, n_prev, u_prev = g_new, n_done, u_hist
    return records


def _worker(rank, world, port, case, q):
    import torch.distributed as dist
    from paper_1710_02401_gb300 import problems as P
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    inst = _case(P, case)
    try:
        q.put((rank, partitioned_swr(inst, rank, world, 3)))
    finally:
        dist.destroy_process_group()


def _case(P, case):
    if case == "2e":
        return P.small_tise_2d(L=3, K_d=6, q_p=6, n_mid=2, max_steps=400)
    return P.tise_1d_two_subdomains(q_p=8).replace(L=4, K_d=16, delta=1.5, max_steps=400)


@pytest.mark.parametrize("case", ["2e", "1e"])
def test_partitioned_instance_matches_single_rank_bit_for_bit(case):
    import torch.multiprocessing as mp
    from oracle import swr_oracle as O
    from paper_1710_02401_gb300 import dist as D, problems as P
    inst = _case(P, case)
    parts = D.partition_subdomains(inst.L, inst.n_elec, 2)
    assert all(parts) and sorted(sum(parts, [])) == list(range(inst.n_sub))
    assert D.exchange_plan(inst.L, inst.n_elec, 2)  # the blocks touch: data cross ranks
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, case, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=600) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = O.run_swr(inst, kmax=3, tol=0.0)
    want = [(r.n_win, r.res, r.energy) for r in ref.records]
    assert out[0] == out[1] == want, (out, want)


def test_partition_blocks_and_exchange_plan():
    from paper_1710_02401_gb300 import dist as D
    for L, N, world in [(4, 2, 4), (8, 2, 8), (5, 2, 3), (7, 1, 3), (2, 2, 4)]:
        parts = D.partition_subdomains(L, N, world)
        assert sorted(sum(parts, [])) == list(range(L ** N))  # disjoint cover
        own = D.owner_map(L, N, world)
        plan = D.exchange_plan(L, N, world)
        for (a, b), pairs in plan.items():
            assert a != b
            for j, i in pairs:
                assert own[j] == a and own[i] == b and j in D.neighbours(L, N, i)
        # every cross-rank neighbour pair travels exactly once
        cross = {(j, i) for i in range(L ** N) for j in D.neighbours(L, N, i) if own[i] != own[j]}
        sent = [ji for pairs in plan.values() for ji in pairs]
        assert sorted(sent) == sorted(cross)
    # 4 x 4 grid on 2 x 2 ranks: each rank a 2 x 2 block
    assert D.partition_subdomains(4, 2, 4)[0] == [0, 1, 4, 5]
    assert D.neighbours(4, 2, 5) == [0, 1, 2, 4, 6, 8, 9, 10]
