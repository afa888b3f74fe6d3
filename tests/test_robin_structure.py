"""The Robin source b' of every subdomain and step has the edge structure the
GPU path's precomputed Robin response relies on (swr_robin.cu).

b' is the Galerkin load of the Robin data on the interior edges (Sec. 5.1,
Eq. RTC).  In a tensor-product basis, as a K_d x K_d matrix B[a][b] (index
a + K_d b), an edge of coordinate 0 at x1 = e contributes phi_a(e) h[b] and
an edge of coordinate 1 contributes h[a] phi_b(e), so B = U X^T + Y V^T with
U (V) the edge-value vectors of the present edges of coordinate 0 (1).  The
GPU path recovers (X, Y) from the stored b' by the gauge-fixed decomposition
Y = B V (V^T V)^{-1}, X^T = (U^T U)^{-1} U^T (B - Y V^T) and forms
G b' = (G E) h; this holds only if the reconstruction is exact, which these
tests check on the oracle's own Robin sources (no GPU code involved).
"""
import numpy as np
import pytest

from oracle import swr_oracle as O
from paper_1710_02401_gb300 import problems as P


def _edge_vectors(loc, d):
    """Edge-value vectors (basis factor of coordinate d at its interior edges)."""
    gam = loc.gamma
    out = []
    for sgn in (-1, 1):
        sel = (gam.dim == d) & (gam.sign == sgn)
        if np.any(sel):
            e = float(gam.X[sel][0, d])
            out.append(loc.basis._factor(np.array([e]), d, O.phi)[0])
    return np.array(out).T if out else np.zeros((loc.basis.r[d], 0))


def _decompose(Bm, U, V):
    p, q = U.shape[1], V.shape[1]
    Y = Bm @ V @ np.linalg.inv(V.T @ V) if q else np.zeros((Bm.shape[0], 0))
    R = Bm - Y @ V.T if q else Bm
    Xt = np.linalg.inv(U.T @ U) @ U.T @ R if p else np.zeros((0, Bm.shape[1]))
    return Xt, Y


@pytest.mark.parametrize("make", [lambda: P.small_tise_2d(L=3, K_d=6, q_p=6, n_mid=2),
                                  lambda: P.small_tdse_2d(L=3, K_d=6, q_p=6, n_mid=2, n_steps=8)],
                         ids=["imaginary-time", "real-time"])
def test_robin_sources_have_the_edge_rank_structure(make):
    inst = make()
    res = O.run_swr(inst, kmax=2, tol=0.0)
    checked = 0
    for i, loc in enumerate(res.locs):
        r1, r2 = loc.basis.r
        U, V = _edge_vectors(loc, 0), _edge_vectors(loc, 1)
        g = res.robin[i]
        for n in range(0, g.shape[0], max(1, g.shape[0] // 6)):
            b = loc.own_vals.T @ (loc.gamma.w * g[n])
            Bm = b.reshape(r2, r1).T  # Bm[a, b] = b'[a + r1 b]
            scale = np.linalg.norm(Bm)
            if scale == 0.0:
                continue
            Xt, Y = _decompose(Bm, U, V)
            rec = (U @ Xt if U.shape[1] else 0.0) + (Y @ V.T if V.shape[1] else 0.0)
            assert np.linalg.norm(rec - Bm) <= 1e-11 * scale, (i, n)
            if U.shape[1] and V.shape[1]:
                assert np.linalg.norm(Xt @ V) <= 1e-11 * scale  # the gauge X^T V = 0
            checked += 1
    assert checked > 20


def test_a_generic_vector_is_not_of_that_form():
    # the decomposition is a projection: a vector outside the edge subspace
    # is not reproduced (the structure above is a property of b', not of the
    # formula)
    inst = P.small_tise_2d(L=3, K_d=6, q_p=6, n_mid=2)
    res = O.run_swr(inst, kmax=1, tol=0.0)
    loc = res.locs[4]  # the centre subdomain: four interior edges
    r1, r2 = loc.basis.r
    U, V = _edge_vectors(loc, 0), _edge_vectors(loc, 1)
    assert U.shape[1] == 2 and V.shape[1] == 2
    Bm = np.random.default_rng(3).standard_normal((r1, r2))
    Xt, Y = _decompose(Bm, U, V)
    assert np.linalg.norm(U @ Xt + Y @ V.T - Bm) > 0.1 * np.linalg.norm(Bm)
