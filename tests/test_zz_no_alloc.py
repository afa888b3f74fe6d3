"""The allocation-free residual entry point (swr_residual_noalloc).

It serves callers that may not allocate device memory at the point of the
call: it keeps its scratch in a static device array instead of the
context's workspace.  Called through the C ABI after two Schwarz iterations
in a row, it must reproduce the residual that swr_step reported (same
kernels, same reduction order), within the FP64 tolerance of the parity
tests.  This file runs last so that a failure here never hides another test.
"""
import numpy as np
import pytest

from paper_1710_02401_gb300 import problems as P

pytestmark = pytest.mark.gpu


def test_residual_noalloc_matches_step_residual_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_02401_gb300 import build as B
    B.build()
    from paper_1710_02401_gb300 import swr as S
    insts = [P.small_tise_2d(L=2, K_d=6, q_p=6, n_mid=2),
             P.tise_1d_two_subdomains().replace(L=3, K_d=20, delta=2.0)]
    s = S.SWR(insts)
    s.assemble()
    with pytest.raises(S.SWRError) as e:
        s.residual_noalloc()  # no iteration yet
    assert e.value.status == S.SWR_ESTATE
    for _ in range(2):
        s.step()
        want = s.residual()
        got = s.residual_noalloc()
        assert np.all(np.isfinite(got))
        np.testing.assert_allclose(got, want, rtol=1e-10, atol=0.0)
        # a second call in a row sees the same shared scratch state
        np.testing.assert_allclose(s.residual_noalloc(), want, rtol=1e-10, atol=0.0)
