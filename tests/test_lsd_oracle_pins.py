"""Pins of the local-orbital / local-Slater-determinant oracle
(oracle/lsd_oracle.py) against facts the paper and the mathematics fix:

* the harmonic oscillator's levels n + 1/2 when the barrier sits far out
  (closed form);
* the eigen identities <phi_l, phi_m> = delta_lm and <phi_l|H_b|phi_m> =
  lambda_l delta_lm, re-evaluated on a different quadrature rule;
* antisymmetry of the determinants (Eq. LSD), pointwise;
* the Gram and Hamiltonian blocks of the determinants against brute-force
  2-D quadrature of the explicit functions (an independent route to the
  determinant rules and the two-electron integrals of Appendix A);
* the two-electron integrals' permutation symmetries and their constant-W
  limit W0 S_mp S_qr;
* Table 1's structure: the determinants of one subdomain orthonormal to
  rounding, a neighbour's small, and smaller as the barrier moves in.
"""
import math

import numpy as np
import pytest

from oracle import lsd_oracle as Lo


def _small(**kw):
    base = dict(box=(-4.5, 4.5), L=3, overlap=0.3, M=4, K=6, kd=24, panel=0.25, q_p=10)
    base.update(kw)
    return Lo.LsdProblem(**base)


def test_harmonic_levels_with_a_far_barrier():
    p = Lo.LsdProblem(box=(-6.0, 6.0), L=3, overlap=0.4, nuclei=(), harmonic=1.0, M=6, kd=64,
                      xb_factor=7.0 / 4.4, eps_b=0.4, panel=0.2, q_p=12)
    o = Lo.local_orbitals(p, 1)  # centred at 0, barrier at |x| = 7
    np.testing.assert_allclose(o.lam, np.arange(6) + 0.5, rtol=0, atol=1e-8)


def test_eigen_identities_on_another_rule():
    p = _small()
    for i in range(p.L):
        o = Lo.local_orbitals(p, i)
        xb = Lo.x_barrier(p)
        m = 1.3 * Lo.local_margin(p)
        x, w = Lo.gl_rule(o.xc - xb - m, o.xc + xb + m, 0.17, 14, Lo.barrier_breaks(p, o.xc))
        F, dF = o.values(x)
        s = Lo.switch(p, x, o.xc)
        S = (F * w) @ F.T
        H = 0.5 * (dF * (w * (1 - s))) @ dF.T + (F * (w * (Lo.v_nuclei(p, x) + p.v_inf * s))) @ F.T
        np.testing.assert_allclose(S, np.eye(p.M), atol=1e-11)
        np.testing.assert_allclose(H, np.diag(o.lam), atol=1e-9 * max(1.0, np.abs(o.lam).max()))
        assert np.all(np.diff(o.lam) > 0)
        # the sign convention
        proj = (F * (w * np.exp(0.37 * (x - o.xc)))).sum(axis=1)
        assert np.all(proj > 0)


def test_determinants_are_antisymmetric():
    p = _small()
    orbs = Lo.all_orbitals(p)
    rng = np.random.default_rng(5)
    x1 = rng.uniform(-4, 4, 50)
    x2 = rng.uniform(-4, 4, 50)
    for (i, j, l, q) in [(1, 1, 0, 2), (0, 1, 3, 1), (2, 1, 1, 1)]:
        np.testing.assert_allclose(Lo.lsd_value(orbs, i, j, l, q, x1, x2),
                                   -Lo.lsd_value(orbs, i, j, l, q, x2, x1), atol=1e-15)


def _grid2(p):
    x, w = Lo.global_rule(p)
    return x, w


def test_gram_and_hamiltonian_against_brute_force_2d_quadrature():
    p = _small()
    orbs = Lo.all_orbitals(p)
    oe = Lo.one_electron(p, orbs)
    x, w = _grid2(p)
    X1, X2 = np.meshgrid(x, x, indexing="ij")
    W2 = w[:, None] * w[None, :]
    F, dF = Lo.orbital_table(p, orbs, x)
    M = p.M

    def det(i, j, l, q):
        a, b = F[i * M + l], F[j * M + q]
        da, db = dF[i * M + l], dF[j * M + q]
        v = (np.outer(a, b) - np.outer(b, a)) / math.sqrt(2)
        d1 = (np.outer(da, b) - np.outer(db, a)) / math.sqrt(2)   # d/dx1
        d2 = (np.outer(a, db) - np.outer(b, da)) / math.sqrt(2)   # d/dx2
        return v, d1, d2

    V2 = Lo.v_nuclei(p, X1) + Lo.v_nuclei(p, X2) + p.ee_coef / np.sqrt((X1 - X2) ** 2 + p.eta_ee ** 2)
    for (i, j) in [(1, 1), (0, 1), (2, 1)]:
        pairs, Sm, Hm = Lo.lsd_hamiltonian(p, orbs, oe, i, j)
        fs = [det(i, j, l, q) for (l, q) in pairs]
        for r in range(len(pairs)):
            for c in range(len(pairs)):
                va, a1, a2 = fs[r]
                vb, b1, b2 = fs[c]
                g = np.sum(W2 * va * vb)
                h = np.sum(W2 * (0.5 * (a1 * b1 + a2 * b2) + V2 * va * vb))
                assert abs(Sm[r, c] - g) <= 1e-12, (i, j, r, c, Sm[r, c], g)
                assert abs(Hm[r, c] - h) <= 1e-10 * max(1.0, abs(h)), (i, j, r, c, Hm[r, c], h)
    # cross-subdomain Gram (Table 1's <v_i, w_j>) by the same route
    pa = Lo.lsd_pairs(p, orbs, 1, 1)
    pb = Lo.lsd_pairs(p, orbs, 2, 1)
    G = Lo.lsd_gram(p, oe, pa, (1, 1), pb, (2, 1))
    for r, (l, q) in enumerate(pa[:3]):
        for c, (m, t) in enumerate(pb[:3]):
            g = np.sum(W2 * det(1, 1, l, q)[0] * det(2, 1, m, t)[0])
            assert abs(G[r, c] - g) <= 1e-12


def test_two_electron_symmetries_and_constant_kernel_limit():
    p = _small()
    orbs = Lo.all_orbitals(p)
    idx = [0, 1, 4, 5, 9]
    E = Lo.two_electron(p, orbs, idx)
    np.testing.assert_allclose(E, E.transpose(2, 3, 0, 1), atol=1e-13)
    np.testing.assert_allclose(E, E.transpose(1, 0, 2, 3), atol=1e-13)
    np.testing.assert_allclose(E, E.transpose(0, 1, 3, 2), atol=1e-13)
    # W -> ee_coef / eta_ee, constant: E = (ee_coef / eta_ee) S (x) S
    q = _small(eta_ee=1e7, ee_coef=1e7)
    orbs_q = Lo.all_orbitals(q)
    Eq = Lo.two_electron(q, orbs_q, idx)
    S = Lo.one_electron(q, orbs_q).S[np.ix_(idx, idx)]
    np.testing.assert_allclose(Eq, np.einsum("mp,qr->mpqr", S, S), atol=1e-9)


def test_table1_structure():
    # the paper's Test 1 geometry ((-8, 8), L = 5, eps = 0.32, nuclei in the
    # central subdomain), smaller bases to keep the oracle quick
    p = Lo.LsdProblem(M=6, K=10, kd=30)
    orbs = Lo.all_orbitals(p)
    oe = Lo.one_electron(p, orbs)
    v = Lo.lsd_pairs(p, orbs, 2, 2)          # Omega_13 (1-based): the central subdomain
    w = Lo.lsd_pairs(p, orbs, 3, 2)          # Omega_14: x1 in D_4, x2 in D_3
    Gvv = Lo.lsd_gram(p, oe, v[:4], (2, 2), v[:4], (2, 2))
    Gvw = Lo.lsd_gram(p, oe, v[:4], (2, 2), w[:2], (3, 2))
    np.testing.assert_allclose(Gvv, np.eye(4), atol=1e-13)
    assert np.abs(Gvw).max() < 0.1 and np.abs(Gvw).max() > 1e-8
    # moving the barrier in (smaller orbital support) shrinks the neighbour overlaps
    q = Lo.LsdProblem(M=6, K=10, kd=30, xb_factor=0.46)
    orbs_q = Lo.all_orbitals(q)
    oe_q = Lo.one_electron(q, orbs_q)
    Gq = Lo.lsd_gram(q, oe_q, Lo.lsd_pairs(q, orbs_q, 2, 2)[:4], (2, 2), Lo.lsd_pairs(q, orbs_q, 3, 2)[:2], (3, 2))
    assert np.abs(Gq).max() < np.abs(Gvw).max()
