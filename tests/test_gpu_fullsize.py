"""GPU parity at the sizes the product runs, against stored oracle values.

The expected values in tests/golden/*.npz were written by
tests/golden/make_golden.py, which calls only the FP64 CPU oracle:

* tise_2e_16sd_k3: the 2-electron ground-state workload at full size (4 x 4
  subdomains, K = 576), first three Schwarz iterations; compared through the
  plans the benchmark runs: the fused double-single window (G_hi rows resident
  in shared memory), the split double-single window (rows streamed by bulk
  copies) and the FP64 two-phase window;
* tdse_2e_k1024_4sd: the real-time workload's subdomain shape (K = 1024
  complex) on 2 x 2 subdomains, 20 Crank-Nicolson steps, two iterations;
  FP64 complex matvec and the four-plane double-single one;
* batched_k1024: three instances of the uneven batch in one launch, two of
  them with K = 1024 two-electron subdomains (split window stages of 66 KB),
  two iterations.

Compared per Schwarz iteration: window lengths (exact), Res(k) and CVTOT(k)
(absolute against 1e-10 of their largest value), energies or norm and dipole
(1e-10 relative); for the last iteration the own traces and Robin data at
every interface node of the stored steps plus seeded samples over the whole
window, and psi at every 7th volume node, against 1e-10 of the largest
magnitude (Robin data included).  The largest measured differences are
printed.
"""
import os

import numpy as np
import pytest

from paper_1710_02401_gb300 import problems as P

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden")
REL = 1e-10
REL_ROBIN = 1e-10
# The NGF stop quantity ||c^n - c^(n-1)|| (Sec. 5.2) is a difference of
# unit-norm iterates near delta = 1e-12, so FP64 rounding (~1e-16 absolute)
# moves it by ~1e-4 relative: where the oracle's own value sits within this
# band of delta, the GPU may stop one step earlier or later.
STOP_BAND = 1e-3
# Res(k) and CVTOT(k) integrate over the window in time: a window one step off
# at the threshold changes them by about one step's share of the integral
# (1/W of the squared sum), so from that iteration on they are compared at
# this bound; every other result keeps 1e-10.
REL_ONE_STEP = 1e-3


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_02401_gb300 import build as B
    B.build()
    from paper_1710_02401_gb300 import swr as S_
    return S_


def _case(name):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLD, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    insts, kmax = mg.case_instances(name)
    path = os.path.join(GOLD, name + ".npz")
    if not os.path.exists(path):
        pytest.fail(f"missing stored values {path}: run tests/golden/make_golden.py {name}")
    return insts, kmax, dict(np.load(path))


def _check(S, name, precision, variant=0, expect_variant=None, contraction_path=None):
    insts, kmax, G = _case(name)
    if contraction_path is None:
        contraction_path = S.CONTRACT_FP64
    s = S.SWR(insts, precision=precision, window_variant=variant, contraction_path=contraction_path)
    s.assemble()
    plan = s.window_plan()
    assert plan["tensor_contractions"] == (1 if contraction_path == S.CONTRACT_TENSOR else 0), plan
    if expect_variant is not None:
        assert plan["variant"] == expect_variant, plan
    ni = len(insts)
    hist = {k: [] for k in ("win", "res", "cvtot", "energy", "norm2", "dipole")}
    for _ in range(kmax):
        s.step()
        hist["win"].append(s.window().astype(np.int64))
        hist["res"].append(s.residual())
        hist["cvtot"].append(s.cvtot())
        if insts[0].mode == P.TDSE:
            hist["norm2"].append(s.norm2())
            hist["dipole"].append(s.dipole())
        else:
            hist["energy"].append(s.energy())
    u_all, g_all, psi_all = s.own_traces(), s.robin_data(), s.psi_nodes()
    worst = {}

    def note(key, val):
        worst[key] = max(worst.get(key, 0.0), float(val))

    sub0 = 0
    for ii, inst in enumerate(insts):
        p = f"i{ii}_"
        win = np.array([h[ii] for h in hist["win"]])
        first_off = None
        for k, (w, wg) in enumerate(zip(win.tolist(), G[p + "win"].tolist())):
            if w == wg:
                continue
            first_off = k if first_off is None else first_off
            # one step off, only where the oracle's stop quantity is within the band of delta
            tol = inst.ngf_tol
            assert p + "stop_prev" in G, (name, ii, k, w, wg)
            if w == wg - 1:
                assert G[p + "stop_prev"][k] <= tol * (1 + STOP_BAND), (name, ii, k, w, wg, G[p + "stop_prev"][k])
            else:
                assert w == wg + 1 and G[p + "stop_last"][k] >= tol * (1 - STOP_BAND), (name, ii, k, w, wg)
            note("window_steps_off_at_threshold", 1)
        for key in ("res", "cvtot"):
            got = np.array([h[ii] for h in hist[key]])
            ref = G[p + key]
            errs = np.abs(got - ref) / ref.max()
            bound = np.full(len(errs), REL)
            if first_off is not None:
                bound[first_off:] = REL_ONE_STEP
            note(key, errs.max())
            assert np.all(errs <= bound), (name, ii, key, got, ref)
        if inst.mode == P.TDSE:
            for key in ("norm2", "dipole"):
                got = np.array([h[ii] for h in hist[key]])
                ref = G[p + key]
                err = (np.abs(got - ref) / np.maximum(np.abs(ref), 1.0 if key == "dipole" else 0.0)).max()
                note(key, err)
                assert err <= REL, (name, ii, key, got, ref)
        else:
            got = np.array([h[ii] for h in hist["energy"]])
            ref = G[p + "energy"]
            err = (np.abs(got - ref) / np.abs(ref)).max()
            note("energy", err)
            assert err <= REL, (name, ii, got, ref)
        # steps of the last iteration, held at the GPU's last step when its window
        # ended one step earlier at the threshold (the iterates then differ by ~1e-12)
        st = np.minimum(G[p + "steps"], int(win[-1]))
        umax = max(np.abs(G[p + f"u{i}"]).max() for i in range(inst.n_sub) if G[p + f"u{i}"].size)
        gmax = max(np.abs(G[p + f"g{i}"]).max() for i in range(inst.n_sub) if G[p + f"g{i}"].size)
        pmax = max(np.abs(G[p + f"psi{i}"]).max() for i in range(inst.n_sub))
        for i in range(inst.n_sub):
            u, g, psi = u_all[sub0 + i], g_all[sub0 + i], psi_all[sub0 + i]
            if G[p + f"u{i}"].size:
                eu = np.abs(u[st] - G[p + f"u{i}"]).max() / umax
                eg = np.abs(g[st] - G[p + f"g{i}"]).max() / gmax
                note("own_traces", eu)
                note("robin", eg)
                assert eu <= REL, (name, ii, i, eu)
                assert eg <= REL_ROBIN, (name, ii, i, eg)
            ep = np.abs(psi[::int(G["psi_stride"])] - G[p + f"psi{i}"]).max() / pmax
            note("psi", ep)
            assert ep <= REL, (name, ii, i, ep)
        idx = G[p + "smp_idx"]
        su = np.array([u_all[sub0 + i][min(n, int(win[-1])), k] for i, n, k in idx])
        sg = np.array([g_all[sub0 + i][min(n, int(win[-1])), k] for i, n, k in idx])
        eu = np.abs(su - G[p + "smp_u"]).max() / umax
        eg = np.abs(sg - G[p + "smp_g"]).max() / gmax
        note("own_traces", eu)
        note("robin", eg)
        assert eu <= REL and eg <= REL_ROBIN, (name, ii, eu, eg)
        sub0 += inst.n_sub
    print(f"\n{name} precision={precision} inverse={contraction_path} plan={plan}: largest relative differences "
          + ", ".join(f"{k} {v:.2e}" for k, v in sorted(worst.items())))


def test_fullsize_ground_state_fused_double_single(S):
    _check(S, "tise_2e_16sd_k3", S.PREC_MIXED, S.WINDOW_FUSED, expect_variant=S.WINDOW_FUSED)


def test_fullsize_ground_state_automatic_plan_is_the_cluster_window(S):
    insts, _, _ = _case("tise_2e_16sd_k3")
    s = S.SWR(insts, precision=S.PREC_MIXED)
    assert s.window_plan()["variant"] == S.WINDOW_CLUSTER


def test_fullsize_ground_state_split_double_single(S):
    _check(S, "tise_2e_16sd_k3", S.PREC_MIXED, S.WINDOW_SPLIT, expect_variant=S.WINDOW_SPLIT)


def test_fullsize_ground_state_resident_double_single(S):
    _check(S, "tise_2e_16sd_k3", S.PREC_MIXED, S.WINDOW_RESIDENT, expect_variant=S.WINDOW_RESIDENT)


def test_fullsize_ground_state_cluster(S):
    # one cluster per subdomain, K = 576 rows on chip (G_hi in shared memory,
    # G_lo in tensor memory)
    _check(S, "tise_2e_16sd_k3", S.PREC_MIXED, S.WINDOW_CLUSTER, expect_variant=S.WINDOW_CLUSTER)


def test_fullsize_ground_state_fp64(S):
    _check(S, "tise_2e_16sd_k3", S.PREC_FP64, 0, expect_variant=S.WINDOW_TWO_PHASE)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_fullsize_real_time_k1024(S, precision):
    _check(S, "tdse_2e_k1024_4sd", precision)


@pytest.mark.parametrize("precision,variant", [(1, 3), (1, 0), (0, 0)], ids=["split", "mixed-auto", "fp64"])
def test_fullsize_batched_k1024(S, precision, variant):
    _check(S, "batched_k1024", precision, variant)


# the step-matrix inverses with the Gauss-Jordan trailing updates on the tensor
# cores (FP64 emulated by BF16 slices): the same stored values, the same bar
@pytest.mark.parametrize("name,precision", [("tise_2e_16sd_k3", 1), ("tise_2e_16sd_k3", 0),
                                            ("tdse_2e_k1024_4sd", 0), ("tdse_2e_k1024_4sd", 1),
                                            ("batched_k1024", 1)],
                         ids=["k576-mixed", "k576-fp64", "k1024-complex-fp64", "k1024-complex-mixed", "batched"])
def test_fullsize_tensor_core_inverse(S, name, precision):
    _check(S, name, precision, contraction_path=S.CONTRACT_TENSOR)


def test_automatic_contraction_path_follows_subdomain_size(S):
    # automatic choice: tensor cores when every subdomain has K >= 768
    for name, want in (("tdse_2e_k1024_4sd", 1), ("tise_2e_16sd_k3", 0), ("batched_k1024", 0)):
        insts, _, _ = _case(name)
        s = S.SWR(insts, contraction_path=S.CONTRACT_AUTO)
        s.assemble()
        assert s.window_plan()["tensor_contractions"] == want, name
