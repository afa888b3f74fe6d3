"""GPU parity of the window plans and of the batched uneven workload.

The imaginary-time window (Sec. 5.2, system SIT) runs as one persistent
launch over all subdomains of all instances.  Its plan (kernel variant,
row-task size, task state in shared or global memory) changes only the order
of the FP64 sums, so every plan must meet the oracle at the FP64 tolerance of
the other parity tests.  The batched sample draws instances from the uneven
family (1- and 2-electron problems, random nuclei, softening and per-subdomain
basis sizes) small enough for the oracle, with 8-row tasks so that CTAs hold
more tasks than shared memory does.
"""
import math

import numpy as np
import pytest

from oracle import swr_oracle as O
from paper_1710_02401_gb300 import problems as P

pytestmark = pytest.mark.gpu

REL = 1e-10


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_02401_gb300 import build as B
    B.build()
    from paper_1710_02401_gb300 import swr
    return swr


def _steps(s, n):
    res, wins, en, cv = [], [], [], []
    for _ in range(n):
        s.step()
        res.append(s.residual().copy())
        wins.append(s.window().copy())
        en.append(s.energy().copy())
        cv.append(s.cvtot().copy())
    _steps.cvtot = np.array(cv)
    return np.array(res), np.array(wins), np.array(en)


def _check(res, wins, en, refs, cv=None):
    cv = _steps.cvtot if cv is None else cv
    for i, ref in enumerate(refs):
        rmax = max(r.res for r in ref.records)
        cmax = max(r.cvtot for r in ref.records)
        for k, r in enumerate(ref.records):
            assert wins[k][i] == r.n_win, (i, k)
            assert abs(res[k][i] - r.res) <= REL * rmax, (i, k, res[k][i], r.res)
            assert abs(en[k][i] - r.energy) <= REL * abs(r.energy), (i, k, en[k][i], r.energy)
            assert abs(cv[k][i] - r.cvtot) <= REL * cmax, (i, k, cv[k][i], r.cvtot)


PLAN_INST = P.small_tise_2d(K_d=16, q_p=8, n_mid=3)  # 9 subdomains, K = 256


@pytest.fixture(scope="module")
def plan_ref():
    return [O.run_swr(PLAN_INST, kmax=3, tol=0.0)]


@pytest.mark.parametrize("precision,variant,rows,many", [
    (0, 1, 8, 0),     # FP64 two-phase, 8-row tasks
    (0, 1, 256, 1),   # FP64, one 256-row task per subdomain: task state in global memory
    (1, 1, 32, 0),    # double-single two-phase
    (1, 1, 256, 1),   # double-single two-phase, task state in global memory
    (1, 2, 16, 0),    # fused (W) single-barrier
    (1, 3, 16, 1),    # split single-barrier (u = G y, w = G b' in one pass)
    (1, 3, 256, 1),
    (1, 4, 16, 0),    # resident: split recursion, static tasks, several tasks per CTA (G_hi from L2)
    (1, 4, 64, 0),    # resident: one task per CTA, its G_hi rows in shared memory
    (2, 4, 32, 0),    # resident with the FP32-rounded matrices (hi plane only): Res/energy not compared
])
def test_window_plans_match_oracle(S, plan_ref, precision, variant, rows, many):
    s = S.SWR(PLAN_INST, precision=precision, window_variant=variant, rows_per_task=rows)
    plan = s.window_plan()
    assert plan["variant"] == variant and plan["task_state_global"] == many
    assert plan["tasks"] == 9 * math.ceil(256 / rows)
    s.assemble()
    if precision == 2:  # FP32-rounded matrices: a different problem; it must run and stay finite
        res, wins, en = _steps(s, 3)
        assert np.all(np.isfinite(res)) and np.all(np.isfinite(en)) and np.all(wins > 0)
        assert abs(en[-1][0] - plan_ref[0].records[-1].energy) <= 1e-6 * abs(plan_ref[0].records[-1].energy)
        return
    _check(*_steps(s, 3), plan_ref)


@pytest.fixture(scope="module")
def batch():
    insts = [i.replace(max_steps=300) for i in P.batched_uneven(6, seed=7, k_lo=36, k_hi=100)]
    refs = [O.run_swr(i, kmax=2, tol=0.0) for i in insts]
    return insts, refs


@pytest.mark.parametrize("precision,variant", [(0, 0), (1, 0), (1, 3)])
def test_batched_uneven_many_tasks_per_cta(S, batch, precision, variant):
    # the two-phase and split kernels with their task state in global memory
    # (automatic plans: two-phase in FP64, split in mixed precision)
    insts, refs = batch
    s = S.SWR(insts, precision=precision, rows_per_task=8, window_variant=variant)
    plan = s.window_plan()
    Ks = [kd ** i.n_elec for i in insts for kd in i.K_d]
    expect = 3 if (variant == 3 or (variant == 0 and precision == 1)) else 1  # automatic: split in mixed precision
    if expect == 3:
        # split window: 8-row tasks for the widest subdomain, the same bytes for the others
        n_tasks = sum(math.ceil(K / min(256, (8 * max(Ks) + K // 2) // K)) for K in Ks)
    else:
        n_tasks = sum(math.ceil(K / 8) for K in Ks)
        assert plan["tasks"] > 4 * plan["ctas"]
    assert plan["tasks"] == n_tasks
    assert plan["task_state_global"] == 1 and plan["variant"] == expect
    s.assemble()
    _check(*_steps(s, 2), refs)


def test_autotune_then_solve_matches_oracle(S, plan_ref):
    s = S.SWR(PLAN_INST, precision=1)
    s.assemble()
    rep = s.autotune(steps=16)
    assert rep["candidates"] >= 4
    assert 0 < rep["seconds_per_step"] <= rep["seconds_default"]
    plan = s.window_plan()
    assert plan["variant"] == rep["variant"] and plan["rows_per_task"] == rep["rows_per_task"]
    _check(*_steps(s, 3), plan_ref)
    with pytest.raises(S.SWRError) as e:
        s.autotune(steps=16)  # only before the first Schwarz iteration
    assert e.value.status == S.SWR_ESTATE


@pytest.mark.parametrize("which", ["tise", "tdse"])
def test_graph_replay_is_bit_identical_to_direct_launches(S, which):
    inst = P.small_tise_2d(L=2, K_d=6, q_p=6, n_mid=2) if which == "tise" else P.small_tdse_2d(L=2, K_d=6, q_p=6, n_mid=2)
    out = []
    for mode in (S.LAUNCH_GRAPH, S.LAUNCH_DIRECT):
        s = S.SWR(inst, launch_mode=mode)
        s.assemble()
        assert s.window_plan()["graph"] == (1 if mode == S.LAUNCH_GRAPH else 0)
        res = [s.step().res for _ in range(4)]  # both parities, first and later iterations
        c = s.counters()
        assert c["window_ms"] > 0 and c["step_ms"] >= c["window_ms"]
        out.append((res, s.own_traces(), s.robin_data(), s.psi_nodes()))
        assert s.window_plan()["graph"] == (1 if mode == S.LAUNCH_GRAPH else 0)  # the capture succeeded
    (ra, ua, ga, pa), (rb, ub, gb, pb) = out
    assert ra == rb
    for x, y in zip(ua + ga + pa, ub + gb + pb):
        np.testing.assert_array_equal(x, y)


EDGE_INSTS = [
    P.small_tise_2d(L=2, K_d=8, q_p=6, n_mid=2).replace(max_steps=40),             # stops at its cap
    P.small_tise_2d(L=2, K_d=9, q_p=6, n_mid=2).replace(nuclei=((0.3, 2.0),)),    # NGF stop, ~1080 steps
    P.tise_1d_two_subdomains().replace(L=1, K_d=30, delta=2.0, q_p=12, n_mid=6),  # one subdomain, no interface
    P.tise_1d_two_subdomains().replace(K_d=96, delta=16.0, q_p=24, n_mid=8, max_steps=400),  # K_d = 96
]


@pytest.fixture(scope="module")
def edge_refs():
    return [O.run_swr(i, kmax=2, tol=0.0) for i in EDGE_INSTS]


@pytest.mark.parametrize("precision,variant", [(1, 3), (0, 0)])
def test_window_edge_cases_in_one_launch(S, edge_refs, precision, variant):
    # instances that stop at the cap beside ones that stop on the NGF tolerance,
    # a single-subdomain instance and a 1-electron basis of 96 Gaussians (its
    # Kronecker factors leave one CTA per SM), in one persistent launch
    s = S.SWR(EDGE_INSTS, precision=precision, window_variant=variant)
    assert s.window_plan()["variant"] == (3 if precision == 1 else 1)
    s.assemble()
    _check(*_steps(s, 2), edge_refs)
