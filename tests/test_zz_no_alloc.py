"""The allocation-free residual entry point (swr_residual_noalloc).

It serves callers that may not allocate device memory at the point of the
call: it keeps its scratch in a static device array instead of the
context's workspace.  Called through the C ABI after two Schwarz iterations
in a row, it must reproduce the residual that swr_step reported (same
kernels, same reduction order), within the FP64 tolerance of the parity
tests, for imaginary-time, antisymmetric (mirror-filled traces) and
real-time (two-plane traces) problems.  Its state rules: SWR_ESTATE until a
step has completed since the last assembly or trace restore, SWR_EINVAL when
the caller's count differs from the number of instances.  This file runs
last so that a failure here never hides another test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1710_02401_gb300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_02401_gb300 import build as B
    B.build()
    from paper_1710_02401_gb300 import swr as S_
    return S_


def _two_steps_match(s):
    for _ in range(2):
        s.step()
        want = s.residual()
        got = s.residual_noalloc()
        assert np.all(np.isfinite(got))
        np.testing.assert_allclose(got, want, rtol=1e-10, atol=0.0)
        # a second call in a row sees the same shared scratch state
        np.testing.assert_allclose(s.residual_noalloc(), want, rtol=1e-10, atol=0.0)


def test_residual_noalloc_matches_step_residual_twice(S):
    insts = [P.small_tise_2d(L=2, K_d=6, q_p=6, n_mid=2),
             P.tise_1d_two_subdomains().replace(L=3, K_d=20, delta=2.0)]
    s = S.SWR(insts)
    s.assemble()
    with pytest.raises(S.SWRError) as e:
        s.residual_noalloc()  # no iteration yet
    assert e.value.status == S.SWR_ESTATE
    _two_steps_match(s)


def test_residual_noalloc_antisymmetric_and_real_time(S):
    anti = P.small_tise_2d(L=3, K_d=8, q_p=6, n_mid=2).replace(symmetry="antisymmetric", phi0_center=(0.8, -0.8))
    s = S.SWR([anti], precision=S.PREC_MIXED)
    s.assemble()
    _two_steps_match(s)
    rt = S.SWR([P.small_tdse_2d(L=2, K_d=8, q_p=6, n_mid=2, n_steps=16)])
    rt.assemble()
    _two_steps_match(rt)


def test_residual_noalloc_state_rules(S):
    s = S.SWR([P.small_tise_2d(L=2, K_d=6, q_p=6, n_mid=2)])
    s.assemble()
    s.step()
    out = np.empty(2, dtype=np.float64)
    st = s.lib.swr_residual_noalloc(s.ctx, out.ctypes.data_as(C.POINTER(C.c_double)), 2)
    assert st == S.SWR_EINVAL  # one instance, two slots
    ckpt = s.traces_get()
    s.traces_set(ckpt)  # a restored state has no residual of its own
    with pytest.raises(S.SWRError) as e:
        s.residual_noalloc()
    assert e.value.status == S.SWR_ESTATE
    s.step()
    np.testing.assert_allclose(s.residual_noalloc(), s.residual(), rtol=1e-10, atol=0.0)
    # a fresh context restored from a checkpoint before any step
    t = S.SWR([P.small_tise_2d(L=2, K_d=6, q_p=6, n_mid=2)])
    t.assemble()
    t.traces_set(ckpt)
    with pytest.raises(S.SWRError) as e:
        t.residual_noalloc()
    assert e.value.status == S.SWR_ESTATE
