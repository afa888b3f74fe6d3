"""Pins of the FP64 CPU oracle against what the mathematics fixes.

Each test checks an oracle function against something other than itself:
closed forms (erf integrals, harmonic-oscillator spectrum, heat kernel, free
Gaussian packet, Ehrenfest motion under a uniform field), an independent
adaptive quadrature, invariants (Crank-Nicolson norm, NGF energy decrease,
exchange symmetry) and brute-force geometric counts.  The cases are chosen
so that a dropped term, a wrong sign, a wrong index order or a transposed
operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.special import erf

from oracle import swr_oracle as O
from paper_1710_02401_gb300 import problems as P


# ----------------------------------------------------------- closed forms

def _moments(al, be, d, l, r):
    """int_l^r u^k exp(-2 d u^2) du (k = 0,1,2) with u = x - m, m = (al+be)/2,
    times the prefactor exp(-d (al-be)^2 / 2)."""
    m = 0.5 * (al + be)
    D = al - be
    c = 2.0 * d
    a, b = l - m, r - m
    pref = np.exp(-d * D * D / 2.0)
    I0 = 0.5 * np.sqrt(np.pi / c) * (erf(np.sqrt(c) * b) - erf(np.sqrt(c) * a))
    I1 = (np.exp(-c * a * a) - np.exp(-c * b * b)) / (2.0 * c)
    I2 = (a * np.exp(-c * a * a) - b * np.exp(-c * b * b)) / (2.0 * c) + I0 / (2.0 * c)
    return pref, m, D, I0, I1, I2


def closed_S(al, be, d, l, r):
    pref, m, D, I0, I1, I2 = _moments(al, be, d, l, r)
    return pref * I0


def closed_X(al, be, d, l, r):
    pref, m, D, I0, I1, I2 = _moments(al, be, d, l, r)
    return pref * (m * I0 + I1)


def closed_Kf(al, be, d, l, r):
    """int phi_a' phi_b' = 4 d^2 int (x-al)(x-be) phi_a phi_b."""
    pref, m, D, I0, I1, I2 = _moments(al, be, d, l, r)
    return 4.0 * d * d * pref * (I2 - 0.25 * D * D * I0)


def _grid(c):
    return c[:, None], c[None, :]


def test_gauss_legendre_exact_on_polynomials():
    inst = P.tise_1d_two_subdomains(q_p=6).replace(n_mid=3)
    for k in range(inst.L):
        x, w = O.nodes_1d(inst, k)
        lo, hi = O.sub_interval(inst, k)
        assert abs(w.sum() - (hi - lo)) < 1e-13
        # exact for degree <= 2 q_p - 1 on every panel -> on the whole interval
        for deg in range(0, 2 * inst.q_p):
            exact = (hi ** (deg + 1) - lo ** (deg + 1)) / (deg + 1)
            got = np.sum(w * x ** deg)
            assert abs(got - exact) <= 1e-12 * max(1.0, abs(exact)), deg


def test_geometry_breakpoints_and_overlap():
    inst = P.tise_2e_16_subdomains()
    for k in range(inst.L - 1):
        lo1, hi1 = O.sub_interval(inst, k)
        lo2, hi2 = O.sub_interval(inst, k + 1)
        assert abs((hi1 - lo2) - inst.overlap) < 1e-13
    lo0, _ = O.sub_interval(inst, 0)
    _, hiL = O.sub_interval(inst, inst.L - 1)
    assert abs(lo0 - (inst.box[0] - inst.overlap / 2)) < 1e-14
    assert abs(hiL - (inst.box[1] + inst.overlap / 2)) < 1e-14


def test_1d_matrices_against_erf_closed_forms():
    inst = P.tise_1d_two_subdomains(q_p=20).replace(nuclei=(), ee_coef=0.0)
    for sid in range(inst.n_sub):
        loc = O.build_local(inst, sid)
        c = loc.basis.centres[0]
        d = loc.basis.delta
        lo, hi = O.sub_interval(inst, sid)
        A, B = _grid(c)
        S = closed_S(A, B, d, lo, hi)
        X = closed_X(A, B, d, lo, hi)
        Kf = closed_Kf(A, B, d, lo, hi)
        assert np.abs(loc.A - S).max() <= 1e-13 * np.abs(S).max()
        assert np.abs(loc.Qx - X).max() <= 1e-13 * np.abs(X).max()
        assert np.abs(loc.Kf - Kf).max() <= 1e-12 * np.abs(Kf).max()
        assert np.abs(loc.V).max() == 0.0


def test_2d_tensor_index_convention_and_dipole():
    inst = P.small_tise_2d(K_d=5, q_p=16).replace(nuclei=(), ee_coef=0.0)
    sid = 1 + inst.L * 2          # i1 = 1, i2 = 2: not symmetric in the two coordinates
    loc = O.build_local(inst, sid)
    k1, k2 = O.sub_multi_index(inst, sid)
    assert (k1, k2) == (1, 2)
    c1, c2 = loc.basis.centres
    d = loc.basis.delta
    l1, h1 = O.sub_interval(inst, k1)
    l2, h2 = O.sub_interval(inst, k2)
    S1 = closed_S(*_grid(c1), d, l1, h1)
    S2 = closed_S(*_grid(c2), d, l2, h2)
    X1 = closed_X(*_grid(c1), d, l1, h1)
    X2 = closed_X(*_grid(c2), d, l2, h2)
    K1 = closed_Kf(*_grid(c1), d, l1, h1)
    K2 = closed_Kf(*_grid(c2), d, l2, h2)
    # m = a + K_d * b  (a: first coordinate)  ->  kron(second, first)
    assert np.allclose(loc.A, np.kron(S2, S1), rtol=0, atol=1e-13 * np.abs(S1).max() ** 2)
    Q = np.kron(S2, X1) + np.kron(X2, S1)
    assert np.allclose(loc.Qx, Q, rtol=0, atol=1e-12 * np.abs(Q).max())
    Kf = np.kron(S2, K1) + np.kron(K2, S1)
    assert np.allclose(loc.Kf, Kf, rtol=0, atol=1e-12 * np.abs(Kf).max())


def test_robin_mass_is_edge_values_times_tangential_overlap():
    inst = P.small_tise_2d(K_d=5, q_p=16).replace(nuclei=(), ee_coef=0.0)
    sid = 0 + inst.L * 1          # i1 = 0 (right edge only), i2 = 1 (bottom and top edges)
    loc = O.build_local(inst, sid)
    k1, k2 = O.sub_multi_index(inst, sid)
    c1, c2 = loc.basis.centres
    d = loc.basis.delta
    l1, h1 = O.sub_interval(inst, k1)
    l2, h2 = O.sub_interval(inst, k2)
    S1 = closed_S(*_grid(c1), d, l1, h1)
    S2 = closed_S(*_grid(c2), d, l2, h2)
    e_h1 = O.phi(h1, c1, d)
    e_l2 = O.phi(l2, c2, d)
    e_h2 = O.phi(h2, c2, d)
    R1 = np.outer(e_h1, e_h1)                       # x1 = hi1 edge
    R2 = np.outer(e_l2, e_l2) + np.outer(e_h2, e_h2)  # x2 = lo2 and hi2 edges
    R = np.kron(S2, R1) + np.kron(R2, S1)
    assert np.abs(loc.R - R).max() <= 1e-13 * np.abs(R).max()
    assert loc.gamma.w.size == 3 * (inst.n_mid + 2) * inst.q_p


def test_soft_coulomb_against_adaptive_quadrature():
    inst = P.tise_1d_two_subdomains(q_p=24).replace(K_d=12, delta=1.0,
                                                    nuclei=((0.3, 2.0), (-1.1, 1.0)), eta_en=0.6)
    loc = O.build_local(inst, 0)
    c = loc.basis.centres[0]
    d = loc.basis.delta
    lo, hi = O.sub_interval(inst, 0)

    def v(x):
        return sum(-z / math.sqrt((x - xa) ** 2 + inst.eta_en ** 2) for xa, z in inst.nuclei)
    for (a, b) in ((11, 11), (9, 11), (5, 7), (0, 11)):
        f = lambda x: math.exp(-d * (x - c[a]) ** 2 - d * (x - c[b]) ** 2) * v(x)
        ref, _ = integrate.quad(f, lo, hi, points=[0.3, -1.1], epsabs=1e-15, epsrel=1e-13, limit=400)
        assert abs(loc.V[a, b] - ref) <= 1e-11 * max(1.0, abs(ref)), (a, b)


def test_electron_repulsion_against_adaptive_quadrature():
    inst = P.small_tise_2d(L=2, K_d=4, q_p=24, n_mid=6).replace(nuclei=())
    loc = O.build_local(inst, 3)
    c1, c2 = loc.basis.centres
    d = loc.basis.delta
    l1, h1 = O.sub_interval(inst, 1)
    l2, h2 = O.sub_interval(inst, 1)
    K = inst.K_d
    for (a, b, cc, dd) in ((0, 0, 0, 0), (1, 2, 3, 1)):
        m, mp = a + K * b, cc + K * dd
        f = lambda y, x: (math.exp(-d * ((x - c1[a]) ** 2 + (x - c1[cc]) ** 2 + (y - c2[b]) ** 2 + (y - c2[dd]) ** 2))
                          / math.sqrt((x - y) ** 2 + inst.eta_ee ** 2))
        ref, _ = integrate.dblquad(f, l1, h1, l2, h2, epsabs=1e-13, epsrel=1e-11)
        assert abs(loc.V[m, mp] - ref) <= 1e-9 * abs(ref), (a, b, cc, dd)


# ------------------------------------------------------------ spectrum

def _ho(L, kd, delta, q_p=20, **kw):
    return P.harmonic_1d_two_subdomains(q_p=q_p).replace(L=L, K_d=kd, delta=delta, **kw)


def test_harmonic_oscillator_generalized_eigenvalues():
    inst = _ho(1, 40, 0.4)
    loc = O.build_local(inst, 0)
    ev = O.generalized_eigs(loc)
    assert np.allclose(ev[:3], [0.5, 1.5, 2.5], atol=1e-9)


def test_canonical_orthogonalisation_of_an_overcomplete_basis():
    # 60 Gaussians of width ~1.3 at spacing 0.36: the overlap Cholesky meets a
    # pivot below 1e-12 of the diagonal, so the basis is reduced to the
    # eigenvectors of S above 1e-12 lambda_max (X^T S X = I on them); the
    # oscillator spectrum n + 1/2 is still reproduced to the accuracy the
    # retained subspace can carry
    inst = _ho(1, 60, 0.3)
    loc = O.build_local(inst, 0)
    S = O.overlap_1d(inst, loc.basis, 0)
    X = O.orth_coordinate(S, inst.orth_tau)
    assert X is not None and 0 < X.shape[1] < 60
    # orthonormal to the rounding of the smallest kept eigenpairs (eps lambda_max / lambda ~ 1e-4)
    np.testing.assert_allclose(X.T @ S @ X, np.eye(X.shape[1]), atol=1e-4)
    lam = np.linalg.eigvalsh(S)
    assert X.shape[1] == int(np.sum(lam > inst.orth_tau * lam.max()))
    ev = O.generalized_eigs(loc)
    assert abs(ev[0] - 0.5) < 1e-6 and abs(ev[1] - 1.5) < 1e-5
    assert np.allclose(ev[:4], [0.5, 1.5, 2.5, 3.5], atol=1e-3)
    # a well-conditioned basis keeps every function (Cholesky path)
    assert O.orth_coordinate(O.overlap_1d(_ho(1, 20, 2.0), O.Basis(_ho(1, 20, 2.0), 0), 0), 1e-12) is None


def test_swr_on_reduced_bases_converges_to_ground_state():
    r = O.run_swr(_ho(2, 60, 0.3, ngf_tol=1e-10), kmax=40, tol=1e-8)
    assert all(l.basis.K < 60 for l in r.locs)
    assert r.converged and abs(r.records[-1].energy - 0.5) < 1e-4


def test_two_electron_harmonic_ground_state():
    # K_d odd and delta = 1/2: the exact ground state exp(-(x1^2+x2^2)/2) is the
    # centre basis function, so E0 = 1 up to rounding; E1 = 2 (twice degenerate)
    inst = P.small_tise_2d(L=1, K_d=15, q_p=16, n_mid=4).replace(
        box=(-6.0, 6.0), overlap=0.5, delta=0.5, nuclei=(), ee_coef=0.0, harmonic=1.0)
    loc = O.build_local(inst, 0)
    ev = O.generalized_eigs(loc)
    assert abs(ev[0] - 1.0) < 1e-10
    assert abs(ev[1] - 2.0) < 1e-3 and abs(ev[2] - ev[1]) < 1e-9


def test_ngf_energy_decreases_to_lowest_eigenvalue():
    inst = _ho(1, 40, 1.0).replace(nuclei=((0.5, 1.0),), eta_en=0.7, phi0_gamma=0.3)
    r = O.run_swr(inst, kmax=1, step_energies=True)
    E = np.array(r.step_energy)
    assert np.all(np.diff(E) <= 1e-13)
    ev = O.generalized_eigs(r.locs[0])
    assert abs(E[-1] - ev[0]) < 1e-10


def test_swr_harmonic_matches_ground_state_and_converges():
    # accurate bases are ill-conditioned (kappa(A) ~ 1e12): the inner stop uses
    # a tolerance above the rounding floor of the Gram quadratic form
    r = O.run_swr(_ho(2, 40, 2.0, ngf_tol=1e-10), kmax=40, tol=1e-8)
    assert r.converged
    res = r.res
    assert res[-1] <= 1e-8 and res[-1] < res[2] * 1e-4
    # the overlapping Galerkin-Robin fixed point is a different discretisation
    # from the single-domain one: agreement to its discretisation error (a
    # wrong transmission sign or scaling moves E by ~1e-2)
    assert abs(r.records[-1].energy - 0.5) < 1e-4
    r2 = O.run_swr(_ho(2, 60, 5.0, ngf_tol=1e-10), kmax=40, tol=1e-8)
    assert r2.converged and abs(r2.records[-1].energy - 0.5) < 1e-4


def test_contributor_sets_match_brute_force_counts():
    inst = P.small_tise_2d(L=3, K_d=4, q_p=4, n_mid=2)
    mid = 1 + 3 * 1
    g = O.gamma_nodes(inst, mid)
    loc = O.build_local(inst, mid)
    counts = np.array([len(c) for c in loc.contrib])
    assert set(counts.tolist()) == {1, 3}
    # nodes in an overlap band of the tangential coordinate see 3 neighbours
    for x, n, d in zip(g.X, counts, g.dim):
        o = 1 - d
        lo, hi = O.sub_interval(inst, 1)
        in_band = (x[o] < lo + inst.overlap) or (x[o] > hi - inst.overlap)
        assert n == (3 if in_band else 1)
        assert O.cover_count(inst, x) == n + 1
    assert g.w.size == 4 * (inst.n_mid + 2) * inst.q_p


# --------------------------------------------------------------- heat

def _heat(dt, n_steps):
    return P.Instance(n_elec=1, box=(-15.0, 15.0), L=3, overlap=1.0, K_d=60, delta=6.0,
                      q_p=16, n_mid=9, nuclei=(), ee_coef=0.0, kinetic=1.0, mu=1.0,
                      mode=P.TISE, normalize=False, dt=dt, n_steps=n_steps, ngf_tol=0.0,
                      phi0_gamma=0.2)


@pytest.mark.slow
def test_heat_equation_first_order_in_time():
    T = 1.0
    X = np.linspace(-8, 8, 33)[:, None]
    exact = (1 + 0.8 * T) ** -0.5 * np.exp(-0.2 * X[:, 0] ** 2 / (1 + 0.8 * T))
    errs = []
    for dt in (0.1, 0.05):
        inst = _heat(dt, int(round(T / dt)))
        r = O.run_swr(inst, kmax=60, tol=1e-11)
        assert r.converged
        got = O.reconstruct_at(inst, r.locs, r.coeffs, X)
        errs.append(np.abs(got - exact).max())
    assert errs[1] < 5e-3
    assert 1.7 < errs[0] / errs[1] < 2.3


# ------------------------------------------------------------ real time

def _free(dt, n_steps, field=(0.0, 1.0, 0.0, 0.0), V=False):
    return P.Instance(n_elec=1, box=(-10.0, 10.0), L=1, overlap=1.0, K_d=90, delta=3.6,
                      q_p=16, n_mid=12, nuclei=((0.4, 1.0),) if V else (), eta_en=0.8,
                      ee_coef=0.0, mu=-10j, mode=P.TDSE, dt=dt, n_steps=n_steps,
                      field=field, phi0_gamma=1.0)


def test_crank_nicolson_conserves_norm_without_boundary():
    inst = _free(0.01, 300, V=True)
    r = O.run_swr(inst, kmax=1)
    loc = r.locs[0]
    n0 = np.real(np.vdot(loc.c0, loc.A @ loc.c0))
    n1 = np.real(np.vdot(r.coeffs[0], loc.A @ r.coeffs[0]))
    assert abs(n1 - n0) <= 1e-12 * n0


def test_free_packet_spreading_second_order():
    errs = []
    for dt in (0.04, 0.02):
        inst = _free(dt, int(round(1.0 / dt)))
        r = O.run_swr(inst, kmax=1)
        loc = r.locs[0]
        psi = O.psi_at_nodes(loc, r.coeffs[0])
        p2 = loc.w * np.abs(psi) ** 2
        x2 = np.sum(p2 * loc.X[:, 0] ** 2) / np.sum(p2)
        errs.append(abs(x2 - (0.25 + 1.0 * 1.0 ** 2)))
    assert errs[1] < 1e-3
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_uniform_field_moves_packet_by_ehrenfest():
    field = (0.5, 1.0, 8.0, 0.3)
    dt, T = 0.01, 1.0
    inst = _free(dt, int(round(T / dt)), field=field)
    r = O.run_swr(inst, kmax=1)
    e = lambda s: O.field_e(inst, s)
    exact, _ = integrate.quad(lambda s: -(T - s) * e(s), 0.0, T, epsabs=1e-14, limit=200)
    assert abs(r.records[-1].dipole - exact) < 2e-5
    assert abs(exact) > 1e-3


def test_absorbing_robin_condition_does_not_increase_norm():
    inst = P.small_tdse_2d(L=2, K_d=6, q_p=6, n_mid=2, n_steps=10)
    norms = []
    for n in (5, 10, 20):
        r = O.run_swr(inst.replace(n_steps=n, field=(0.0, 1.0, 0.0, 0.0)), kmax=1)
        norms.append(r.records[-1].norm2)
    assert norms[0] >= norms[1] >= norms[2]


# ------------------------------------------------------------ symmetry

def test_singlet_ground_state_is_exchange_symmetric():
    inst = P.small_tise_2d(L=2, K_d=6, q_p=6, n_mid=2)
    r = O.run_swr(inst, kmax=6, tol=1e-8)
    q = (inst.n_mid + 2) * inst.q_p
    for sid in range(inst.n_sub):
        i1, i2 = O.sub_multi_index(inst, sid)
        mir = i2 + inst.L * i1
        a = O.psi_at_nodes(r.locs[sid], r.coeffs[sid]).reshape(q, q)      # [q2, q1]
        b = O.psi_at_nodes(r.locs[mir], r.coeffs[mir]).reshape(q, q)
        assert np.abs(a - b.T).max() <= 1e-11 * np.abs(a).max()


def test_classical_swr_by_penalty_is_consistent_to_order_one_over_mu():
    # Classical SWR (Dirichlet condition psi_i = psi_j on the interfaces, Sec. 4)
    # imposed through the same boundary term with data g = mu psi_j: the fixed
    # point satisfies d_n psi_i + mu psi_i = mu psi_j, so psi_i - psi_j = O(1/mu)
    # and the converged energy of the harmonic oscillator (exact 1/2) is off by
    # C/mu; the Robin data (d_n + mu) psi_j is consistent for any mu.  Keeping
    # the normal derivative in the classical data, or dropping the 1/|J|
    # average, breaks one of the two.
    err = {}
    for mu in (10.0, 100.0, 1000.0):
        r = O.run_swr(_ho(2, 24, 1.0, q_p=12, ngf_tol=1e-10, mu=mu, tc="dirichlet"), kmax=100, tol=1e-8)
        assert r.converged
        err[mu] = r.records[-1].energy - 0.5
    c = [err[mu] * mu for mu in err]
    assert all(abs(x) > 0.05 for x in c)
    assert max(c) - min(c) < 0.2 * max(abs(x) for x in c)  # error * mu constant: first order in 1/mu
    rr = O.run_swr(_ho(2, 24, 1.0, q_p=12, ngf_tol=1e-10, mu=10.0), kmax=100, tol=1e-8)
    assert rr.converged and abs(rr.records[-1].energy - 0.5) < 1e-4


def test_antisymmetric_states_by_mirror_projection():
    # two non-interacting electrons in a harmonic well: the lowest state is
    # symmetric (1/2 + 1/2 = 1), the lowest antisymmetric one has one electron
    # in each of the two lowest levels (1/2 + 3/2 = 2).  Each step acts on the
    # antisymmetric part of its input over mirror subdomains (Appendix A), so
    # the imaginary-time iteration reaches 2 instead of 1.
    base = P.small_tise_2d(L=1, K_d=14, q_p=10, n_mid=3).replace(
        nuclei=(), ee_coef=0.0, harmonic=1.0, phi0_center=(0.8, -0.8), ngf_tol=1e-10)
    ra = O.run_swr(base.replace(symmetry="antisymmetric"), kmax=5, tol=1e-8)
    rs = O.run_swr(base, kmax=5, tol=1e-8)
    assert abs(ra.records[-1].energy - 2.0) < 2e-4 and abs(rs.records[-1].energy - 1.0) < 2e-4
    # 2 x 2 subdomains: two diagonal subdomains and one mirror pair
    b2 = P.small_tise_2d(L=2, K_d=12, q_p=10, n_mid=3)
    inst = b2.replace(nuclei=(), ee_coef=0.0, harmonic=1.0, overlap=1.0, phi0_center=(0.8, -0.8), ngf_tol=1e-10,
                      delta=P.spacing_rule_delta(b2.box, 2, 1.0, 12), symmetry="antisymmetric")
    r = O.run_swr(inst, kmax=40, tol=1e-8)
    assert r.converged and abs(r.records[-1].energy - 2.0) < 5e-3  # discretisation error of this basis
    # the iterate itself is antisymmetric: psi_sigma(i)(x2, x1) = -psi_i(x1, x2)
    for i in range(inst.n_sub):
        j = (i // inst.L) + inst.L * (i % inst.L)
        X = r.locs[i].X
        a = r.locs[i].basis.values(X) @ r.coeffs[i]
        b = r.locs[j].basis.values(X[:, ::-1]) @ r.coeffs[j]
        assert np.abs(a + b).max() <= 1e-9 * np.abs(a).max()


def test_real_time_keeps_antisymmetric_states_antisymmetric():
    # the Hamiltonian, the dipole field term x1 + x2 and the decomposition are
    # exchange-symmetric, so Crank-Nicolson steps of antisymmetric data stay
    # antisymmetric (no projection in real time; measured 2.5e-10 relative)
    inst = P.small_tdse_2d().replace(symmetry="antisymmetric", phi0_center=(0.8, -0.8))
    r = O.run_swr(inst, kmax=2, tol=0.0)
    for i in range(inst.n_sub):
        j = (i // inst.L) + inst.L * (i % inst.L)
        X = r.locs[i].X
        a = r.locs[i].basis.values(X) @ r.coeffs[i]
        b = r.locs[j].basis.values(X[:, ::-1]) @ r.coeffs[j]
        assert np.abs(a + b).max() <= 1e-8 * np.abs(a).max()
    assert r.records[-1].norm2 > 0.1


# ------------------------------------------------ Res(k) and CVTOT (Sec. 4, 6)
#
# A 2 x 2 decomposition of [-4, 4]^2 (overlap 1, 11 Gaussians of exponent 2
# per coordinate, centres 0.5 apart) where the Gaussian exp(-2 |x|^2) is a
# basis function of every subdomain: it is projected exactly, and with no
# kinetic term, no potential and no Robin source the implicit Euler step is
# the identity, so every iterate of every Schwarz iteration is that Gaussian.
# Interface integrals of it are erf closed forms.

_PIN_DELTA = 2.0


def _pin_instance(**kw):
    base = P.Instance(n_elec=2, box=(-4.0, 4.0), L=2, overlap=1.0, K_d=11, delta=_PIN_DELTA, q_p=12, n_mid=3,
                      nuclei=(), ee_coef=0.0, harmonic=0.0, kinetic=0.0, mu=10.0, mode=P.TISE,
                      normalize=False, dt=0.37, n_steps=5, ngf_tol=0.0, phi0_gamma=_PIN_DELTA,
                      phi0_center=(0.0, 0.0))
    return base.replace(**kw) if kw else base


def _edge_integral(p, lo, hi, d=_PIN_DELTA):
    """int_lo^hi exp(-2 d (p^2 + x^2)) dx: |exp(-d |x|^2)|^2 along the line x_e = p."""
    c = 2.0 * d
    return math.exp(-c * p * p) * 0.5 * math.sqrt(math.pi / c) * (erf(math.sqrt(c) * hi) - erf(math.sqrt(c) * lo))


def _pin_locs(inst):
    locs = O.assemble(inst)
    for l in locs:  # the raw Gaussians are kept (Cholesky accepted): basis functions are exact Gaussians
        assert all(t is None for t in l.basis.T)
    return locs


def test_residual_closed_form_through_the_schwarz_loop():
    inst = _pin_instance()
    r = O.run_swr(inst, kmax=2, tol=0.0)
    # every subdomain has two interior edges of length 5 at distance 0.5 from the origin
    edge = _edge_integral(0.5, -4.5, 0.5)
    want = math.sqrt(inst.n_steps * inst.dt * 8.0 * edge)
    assert abs(r.records[0].res - want) <= 1e-12 * want, (r.records[0].res, want)
    assert r.records[1].res <= 1e-12 * want  # the same iterates again
    # every local solution is the same function; CVTOT sums per-pair norms of the
    # rounding of c0 = A^-1 c~ (kappa(A) eps ~ 1e-13 per coefficient)
    assert r.records[0].cvtot <= 1e-10 * want


def test_residual_holds_the_shorter_window_at_its_last_value():
    inst = _pin_instance()
    locs = _pin_locs(inst)
    u0 = [l.own_vals @ l.c0 for l in locs]  # exp(-2|x|^2) at each subdomain's interface nodes
    edge8 = 8.0 * _edge_integral(0.5, -4.5, 0.5)
    rng = np.random.default_rng(7)
    dt = 0.23
    for W, Wp in ((4, 7), (7, 3), (5, 5)):
        f = rng.normal(size=W + 1)
        g = rng.normal(size=Wp + 1)
        u_k = [np.outer(f, u) for u in u0]
        u_km1 = [np.outer(g, u) for u in u0]
        want2 = edge8 * sum(dt * (f[min(n, W)] - g[min(n, Wp)]) ** 2 for n in range(1, max(W, Wp) + 1))
        got = O.schwarz_residual(locs, dt, u_k, u_km1)
        assert abs(got - math.sqrt(want2)) <= 1e-12 * math.sqrt(want2), (W, Wp, got, math.sqrt(want2))
    # first iteration: u^(0) = 0
    f = rng.normal(size=6)
    got = O.schwarz_residual(locs, dt, [np.outer(f, u) for u in u0], None)
    want = math.sqrt(edge8 * dt * float(np.sum(f[1:] ** 2)))
    assert abs(got - want) <= 1e-12 * want


def test_interface_mismatch_closed_form_of_pairwise_norms():
    # psi_0 = f_n exp(-2|x|^2) on the lower-left subdomain, psi = 0 on the others:
    # the mismatch on Gamma_{i;j} is psi_0 wherever 0 is one of the pair, so the
    # pair norms are square roots of sums of edge integrals:
    #   (0,(1,0)), (0,(0,1)), ((1,0),0), ((0,1),0): a full edge + a corner band
    #   (0,(1,1)), ((1,1),0): two corner bands
    inst = _pin_instance()
    locs = _pin_locs(inst)
    ops = O.TraceOps(inst, locs)
    e0 = np.zeros(locs[0].basis.K)
    e0[9 + 11 * 9] = 1.0  # centre (0, 0) of subdomain 0 (centres -4.5 .. 0.5)
    rng = np.random.default_rng(11)
    f = rng.normal(size=7)
    hist = [[f[n] * e0] + [np.zeros(l.basis.K) for l in locs[1:]] for n in range(7)]
    A = _edge_integral(0.5, -4.5, 0.5)
    B = _edge_integral(0.5, -0.5, 0.5)
    C = 4.0 * math.sqrt(A + B) + 2.0 * math.sqrt(2.0 * B)
    dt = 0.41
    want = C * math.sqrt(dt * float(np.sum(f[1:] ** 2)))
    got = O.interface_mismatch(locs, ops, hist, dt)
    assert abs(got - want) <= 1e-11 * want, (got, want)


def test_interface_mismatch_stays_at_the_discretisation_error_when_res_vanishes():
    # Eq. CVTOT2 measures psi_i - psi_j on the interfaces; at the converged
    # Schwarz iterate those still differ by the discretisation error, while
    # Res(k) (successive iterates) goes to 0
    r = O.run_swr(P.harmonic_1d_two_subdomains(), kmax=50, tol=1e-10)
    assert r.converged
    c = [rec.cvtot for rec in r.records]
    assert c[-1] > 1e3 * r.records[-1].res
    assert abs(c[-1] - c[-2]) <= 1e-6 * c[-1]


def test_recorded_ngf_stop_values_bracket_the_tolerance():
    # Sec. 5.2: the window ends at the first step whose ||c^n - c^(n-1)|| is at
    # most delta; the recorded values of its last two steps straddle delta
    inst = P.small_tise_2d(L=2, K_d=6, q_p=6, n_mid=2)
    r = O.run_swr(inst, kmax=2, tol=0.0)
    for rec in r.records:
        W = rec.n_win
        assert set(rec.stop_values) == {W - 1, W}
        assert rec.stop_values[W] <= inst.ngf_tol < rec.stop_values[W - 1]
