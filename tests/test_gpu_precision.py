"""The FP32-rounded step matrices with outer refinement (SWR_PREC_FP32_REFINED).

The bulk of the Schwarz iterations reads only the hi plane of the step
matrices (the FP32-rounded matrix, products still formed in double-single);
once Res(k) reaches the switch level the iteration continues with the
double-single matrices and converges to the fixed point of the exact
discrete problem.  Checked against the FP64 oracle run to the same
tolerance:

* after refinement (converged at Res <= 1e-10): energies, norms and dipoles
  to 1e-9 relative and psi at every volume node to 1e-8 of its largest value
  -- the two runs follow different trajectories, so they agree to the
  distance of each from the common fixed point, not to rounding;
* before refinement (the fixed point of the FP32-rounded iteration): the
  mixed-path bounds, energy to 1e-8 and the wavefunction's relative L2
  difference over the volume nodes to 1e-6.

The largest differences are printed for each result.
"""
import numpy as np
import pytest

from oracle import swr_oracle as O
from paper_1710_02401_gb300 import problems as P

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_02401_gb300 import build as B
    B.build()
    from paper_1710_02401_gb300 import swr as S_
    return S_


def _psi_diff(s, ref):
    psi = s.psi_nodes()
    pref = [O.psi_at_nodes(ref.locs[i], ref.coeffs[i]) for i in range(len(ref.locs))]
    pmax = max(np.abs(p).max() for p in pref)
    d_max = max(np.abs(a - b).max() for a, b in zip(psi, pref)) / pmax
    l2 = np.sqrt(sum(np.sum(np.abs(a - b) ** 2) for a, b in zip(psi, pref)) /
                 sum(np.sum(np.abs(b) ** 2) for b in pref))
    return d_max, l2


def _run(S, inst, variant=0, refine_res=0.0, stop_at_switch=False, kmax=200):
    s = S.SWR(inst, precision=S.PREC_FP32_REFINED, window_variant=variant, refine_res=refine_res)
    s.assemble()
    if not stop_at_switch:  # the library's own loop, with its default switch at 10 x tol
        rep, hist = s.iterate(TOL, kmax)
        return s, [1] * rep.fp32_iterations + [0] * (rep.iterations - rep.fp32_iterations), hist, None
    flags, res = [], []
    for _ in range(kmax):
        if stop_at_switch:
            snap = (s.energy().copy(), s.norm2().copy(), s.dipole().copy()) if flags else None
        rep = s.step()
        flags.append(rep.fp32_matrices)
        res.append(rep.res)
        if stop_at_switch and not rep.fp32_matrices:
            return s, flags, res, snap
        if rep.res <= TOL and not rep.fp32_matrices:
            break
    return s, flags, res, None


CASES = [("one-electron", P.tise_1d_two_subdomains, 0), ("two-electron-fused", P.small_tise_2d, 0),
         ("two-electron-split", P.small_tise_2d, 3), ("two-electron-resident", P.small_tise_2d, 4),
         ("two-electron-cluster", P.small_tise_2d, 5)]


@pytest.mark.parametrize("name,make,variant", CASES, ids=[c[0] for c in CASES])
def test_fp32_phase_then_refinement_reaches_the_oracle_fixed_point(S, name, make, variant):
    inst = make()
    ref = O.run_swr(inst, kmax=200, tol=TOL)
    assert ref.converged
    s, flags, res, _ = _run(S, inst, variant)
    assert res[-1] <= TOL and flags[-1] == 0
    n32 = sum(flags)
    assert n32 >= 3, flags  # some iterations ran with the FP32-rounded matrices
    assert flags == sorted(flags, reverse=True)  # one switch, never back
    e = float(s.energy()[0])
    de = abs(e - ref.records[-1].energy) / abs(ref.records[-1].energy)
    dmax, l2 = _psi_diff(s, ref)
    print(f"\n{name}: {n32} of {len(flags)} Schwarz iterations on FP32 matrices; after refinement "
          f"energy {de:.2e}, psi max {dmax:.2e}, psi L2 {l2:.2e}")
    assert de <= 1e-9
    assert dmax <= 1e-8


@pytest.mark.parametrize("name,make,variant", CASES[:2], ids=[c[0] for c in CASES[:2]])
def test_fp32_fixed_point_meets_the_mixed_path_bounds_before_refinement(S, name, make, variant):
    inst = make()
    ref = O.run_swr(inst, kmax=200, tol=TOL)
    # switch only once the FP32 iteration itself has converged to Res <= 1e-11
    s, flags, res, snap = _run(S, inst, variant, refine_res=1e-11, stop_at_switch=True)
    assert snap is not None and flags[-1] == 0 and sum(flags) >= 2
    e32 = float(snap[0][0])
    de = abs(e32 - ref.records[-1].energy) / abs(ref.records[-1].energy)
    print(f"\n{name}: FP32-rounded fixed point (Res {res[-2]:.1e} after {len(flags) - 1} iterations): "
          f"energy {de:.2e} from the oracle's converged energy")
    assert de <= 1e-8


def test_fp32_refined_real_time(S):
    inst = P.small_tdse_2d(n_steps=24)
    ref = O.run_swr(inst, kmax=60, tol=TOL)
    assert ref.converged
    s, flags, res, _ = _run(S, inst, kmax=60)
    assert res[-1] <= TOL and flags[-1] == 0 and sum(flags) >= 1
    dn = abs(float(s.norm2()[0]) - ref.records[-1].norm2) / ref.records[-1].norm2
    dd = abs(float(s.dipole()[0]) - ref.records[-1].dipole) / max(1.0, abs(ref.records[-1].dipole))
    dmax, l2 = _psi_diff(s, ref)
    print(f"\nreal time: {sum(flags)} of {len(flags)} Schwarz iterations on FP32 matrices; after refinement "
          f"norm {dn:.2e}, dipole {dd:.2e}, psi max {dmax:.2e}, psi L2 {l2:.2e}")
    assert dn <= 1e-9 and dd <= 1e-9 and dmax <= 1e-8
