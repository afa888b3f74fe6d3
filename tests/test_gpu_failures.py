"""Failure detection through the C ABI, made to fire without faulting the GPU.

* SWR_ETIMEOUT: the device-side waits of the window kernels are bounded by a
  per-problem poll limit; a limit of one poll makes the grid barriers of a
  normal window give up (the cluster window on a problem whose subdomains
  differ in size, where some CTAs wait at every step).  Every CTA returns (the limit bounds each wait, and
  a CTA that finds the error flag set stops waiting), the host reads the
  status, and the context stays usable: with the default limit restored and
  the checkpoint of the previous iteration put back, the next step
  reproduces an undisturbed run bit for bit.
* SWR_ENUMERIC: a NaN placed in the Robin source of a restored trace window
  (swr_traces SET) reaches the normalisation of the next window.
* SWR_ENOTCONV: swr_iterate stops at kmax above tol and still fills its
  report.
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


def _bvec_offset(s, inst, sub):
    """Byte offset of the Robin source b' of subdomain `sub`, step 0, in the
    swr_traces buffer: [window per instance, int64] then per subdomain
    u[(cap+1) x max(n_gamma, 1) x nch] and b'[(cap+1) x K x nch] (doubles)."""
    counts = s.node_counts()
    nch = 2 if inst.mode == P.TDSE else 1
    total = s.trace_bytes()
    ni = len(s.instances)
    per_sub = [(max(int(ng), 1) + int(K)) * nch for (_q, ng, K) in counts]
    cap1 = (total - 8 * ni) // (8 * sum(per_sub))
    off = 8 * ni
    for j in range(sub):
        off += 8 * cap1 * per_sub[j]
    return off + 8 * cap1 * max(int(counts[sub][1]), 1) * nch


def _uneven_cluster_instance():
    """Four subdomains, one of them with a 4 x 4 basis against 16 x 16 for
    the others.  The cluster window forms G y^n before it waits for the
    partials of s_n, so with even subdomains every partial is usually there
    at the first poll; here the small subdomain's CTAs reach the poll far
    ahead of the others' partials at every step."""
    base = P.small_tise_2d(L=2, q_p=8, n_mid=3)
    kds = [16, 16, 16, 4]
    return base.replace(K_d=kds, delta=[P.spacing_rule_delta(base.box, 2, base.overlap, k) for k in kds])


@pytest.mark.parametrize("precision,variant", [(0, 1), (1, 2), (1, 5)], ids=["fp64-two-phase", "mixed-fused",
                                                                            "mixed-cluster"])
def test_barrier_timeout_is_reported_and_the_context_recovers(S, precision, variant):
    inst = _uneven_cluster_instance() if variant == 5 else P.small_tise_2d()
    ref = S.SWR(inst, precision=precision, window_variant=variant)
    ref.assemble()
    ref.step()
    ref.step()
    want_res, want_e = ref.residual().copy(), ref.energy().copy()

    s = S.SWR(inst, precision=precision, window_variant=variant)
    s.assemble()
    s.step()
    ckpt = s.traces_get()
    assert s.window_plan()["ctas"] > 1  # a single CTA would never wait
    s.set_spin_limit(1)
    with pytest.raises(S.SWRError) as e:
        s.step()
    assert e.value.status == S.SWR_ETIMEOUT
    with pytest.raises(S.SWRError) as e:  # the failed step left no residual to recompute
        s.residual_noalloc()
    assert e.value.status == S.SWR_ESTATE
    s.set_spin_limit(0)
    s.traces_set(ckpt)
    s.step()
    np.testing.assert_array_equal(s.residual(), want_res)
    np.testing.assert_array_equal(s.energy(), want_e)


def test_timeout_limit_is_validated(S):
    with pytest.raises(S.SWRError) as e:
        S.SWR(P.small_tise_2d(), spin_limit=-1)
    assert e.value.status == S.SWR_EINVAL


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_nan_in_restored_traces_is_reported(S, precision):
    inst = P.small_tise_2d()
    s = S.SWR(inst, precision=precision)
    s.assemble()
    s.step()
    good = s.traces_get()
    bad = good.copy()
    K = int(s.node_counts()[4][2])
    off = _bvec_offset(s, inst, 4) + 8 * (K + 8)  # b' of the centre subdomain, step 1, element 8
    bad[off:off + 8] = np.frombuffer(np.array([np.nan]).tobytes(), dtype=np.uint8)
    s.traces_set(bad)
    with pytest.raises(S.SWRError) as e:
        s.step()
    assert e.value.status == S.SWR_ENUMERIC
    s.traces_set(good)  # the restored checkpoint steps normally
    s.step()
    assert np.all(np.isfinite(s.residual()))


def test_nan_in_real_time_traces_is_reported(S):
    inst = P.small_tdse_2d(n_steps=12)
    s = S.SWR(inst)
    s.assemble()
    s.step()
    bad = s.traces_get().copy()
    K = int(s.node_counts()[4][2])
    off = _bvec_offset(s, inst, 4) + 8 * (2 * K + 3)  # step 1 (two planes per step), element 3
    bad[off:off + 8] = np.frombuffer(np.array([np.inf]).tobytes(), dtype=np.uint8)
    s.traces_set(bad)
    with pytest.raises(S.SWRError) as e:
        s.step()
    assert e.value.status == S.SWR_ENUMERIC


def test_not_converged_fills_the_report(S):
    s = S.SWR(P.small_tise_2d())
    s.assemble()
    rep = S.swr_report()
    hist = (C.c_double * 3)()
    st = s.lib.swr_iterate(s.ctx, 1e-30, 3, C.byref(rep), hist)
    assert st == S.SWR_ENOTCONV
    assert rep.iterations == 3 and rep.converged == 0
    assert rep.res_last == hist[2] > 1e-30
    assert rep.subdomain_solves > 0 and rep.seconds > 0
    assert b"after 3 iterations" in s.lib.swr_last_error(s.ctx)
