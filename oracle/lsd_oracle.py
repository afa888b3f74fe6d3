"""Plain FP64 CPU oracle of the local orbitals (LOs) and local Slater
determinants (LSDs) of the paper's second basis family.

TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the benchmark's
CPU-baseline / reference arm may import or run this module.  The product path
(the CUDA library and its Python binding) never calls it and shares no code
with it.

What it restates (E. Lorin, "Domain Decomposition Method for the N-body
Time-Independent and Time-Dependent Schroedinger Equation"):

  local orbitals ...... Sec. 3.2 "Local orbital construction": in each 1-D
                         subdomain D_i the one-electron eigenproblem
                         (-1/2 d/dx(a d/dx) + V_en + V_b(x - x_ci)) phi = lambda phi
                         with the barrier potential of Eq. BARPOT and
                         a = 1 - s (the kinetic coefficient switched off
                         where the barrier is on); the M lowest eigenpairs
  LSDs ................ Eq. LSD: v_{l,p}^{i,j}(x1, x2) =
                         (phi_l^i(x1) phi_p^j(x2) - phi_l^i(x2) phi_p^j(x1)) / sqrt(2)
  LSD Hamiltonian ..... Appendix A "Discrete local Hamiltonian construction
                         with local Slater's determinants": the one-electron
                         integrals I_lm^ij (kinetic and nuclear attraction) and
                         J_lm^ij (position), the two-electron integrals
                         I_mpqr^ijkl = int int phi_m^i phi_p^j (x) W(x - s)
                         phi_q^k phi_r^l (s), combined into the matrix of
                         H0 = h(1) + h(2) + W(x1 - x2) between determinants
  orthogonality ....... Sec. 7 Test 1, Table 1: L2 inner products of the
                         LSDs of one subdomain and of a neighbour's

Readings where the paper is silent, garbled or not usable in 1-D:
  * Coulomb interactions are the soft-Coulomb forms of the Gaussian path
    (-Z / sqrt((x - x_A)^2 + eta_en^2), 1 / sqrt((x1 - x2)^2 + eta_ee^2)): the
    mollified G_eps of Eq. GEPS diverges in 1-D (1/|x| is not locally
    integrable), so it is not built;
  * the smooth step s of Eq. BARPOT rises from 0 to 1 over
    [x_b - eps_b/2, x_b + eps_b/2] (the text gives the lower edge twice), as the
    C^2 quintic 6u^5 - 15u^4 + 10u^3; the barrier and the kinetic switch act
    on |x - x_ci| (an orbital support (x_ci - x_b, x_ci + x_b), as the text
    states);
  * the eigenproblem is discretised by Galerkin on Gaussians
    exp(-delta (x - alpha_k)^2), alpha_k equally spaced on
    [x_ci - x_b, x_ci + x_b], with composite Gauss-Legendre quadrature on
    [x_ci - x_b - m, x_ci + x_b + m], m = max(eps_b, 8 Gaussian standard
    deviations), whose panels break where the step starts and ends (the paper
    uses a grid of N
    points; the Gaussian form makes every later integral a quadrature of
    smooth functions);
  * an eigenvector's sign is fixed by int phi(x) exp(0.37 (x - x_ci)) dx > 0
    (a positive weight without symmetry, nonzero for even and odd orbitals);
  * the LSDs of Omega_{i,j} (x1 in D_i, x2 in D_j, index i + L j): pairs
    (l, p) of orbital indices, l < p when i = j (a determinant of one orbital
    with itself vanishes), every pair otherwise, ordered by
    lambda_l^i + lambda_p^j (sums within 1e-9 relative count as ties, broken by
    l, then p), the first K kept (the paper selects K LSDs among the
    candidate determinants without giving the rule);
  * Test 1's K = N_phi (N_phi + 1) / 2 = 45 determinants per subdomain with
    N_phi = 9: a diagonal subdomain needs l < p, and 45 = C(10, 2), so the
    default takes M = 10 orbitals per 1-D subdomain and K = 45;
  * x_b, eps_b and V_inf are not given for the tests: x_b = |D_i|/2 (the
    barrier at half height on the edge of D_i, the orbitals not null there),
    eps_b = 0.4, V_inf = 100; with these the neighbour inner products of
    Table 1 come out at 1e-2 rather than the paper's 1e-5 to 3e-3 (they fall
    as the barrier moves in);
  * integrals between orbitals run over the whole line (the orbitals' common
    support, Appendix A), by one composite Gauss-Legendre rule on [a, b]
    widened by the orbital supports and the same margin m.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Sequence, Tuple

import numpy as np
from numpy.polynomial.legendre import leggauss
from scipy.linalg import eigh


@dataclass(frozen=True)
class LsdProblem:
    box: Tuple[float, float] = (-8.0, 8.0)
    L: int = 5                      # 1-D subdomains
    overlap: float = 0.32           # width of the overlap of neighbouring D_i
    nuclei: Tuple[Tuple[float, float], ...] = ((-0.5, 1.0), (0.5, 1.0))  # (x_A, Z_A)
    eta_en: float = 0.5
    eta_ee: float = 0.5
    ee_coef: float = 1.0
    harmonic: float = 0.0           # + harmonic x^2 / 2 in the one-electron potential
    M: int = 10                     # local orbitals per 1-D subdomain
    K: int = 45                     # LSDs per 2-D subdomain
    kd: int = 40                    # Gaussians of one orbital basis
    delta: float = 0.0              # Gaussian exponent (0: spacing rule)
    xb_factor: float = 0.5          # x_b = xb_factor |D_i|
    eps_b: float = 0.4              # width of the barrier's rise
    v_inf: float = 100.0            # barrier height
    q_p: int = 12                   # GL nodes per panel
    panel: float = 0.2              # panel width of the quadrature rules


def subdomain(p: LsdProblem, i: int) -> Tuple[float, float, float]:
    """D_i = [a + i H - eps/2, a + (i+1) H + eps/2] (the opening of Sec. 6),
    returned with its centre x_ci."""
    a, b = p.box
    H = (b - a) / p.L
    lo = a + i * H - 0.5 * p.overlap
    hi = a + (i + 1) * H + 0.5 * p.overlap
    return lo, hi, 0.5 * (lo + hi)


def x_barrier(p: LsdProblem) -> float:
    lo, hi, _ = subdomain(p, 0)
    return p.xb_factor * (hi - lo)


def gaussian_exponent(p: LsdProblem) -> float:
    """delta from the spacing h of the centres: delta = 1 / (2 h^2) (standard
    deviation one spacing), unless given."""
    if p.delta > 0.0:
        return p.delta
    h = 2.0 * x_barrier(p) / (p.kd - 1)
    return 0.5 / (h * h)


def smooth_step(u):
    """0 for u <= 0, 1 for u >= 1, 6u^5 - 15u^4 + 10u^3 between (C^2)."""
    u = np.clip(u, 0.0, 1.0)
    return u * u * u * (u * (6.0 * u - 15.0) + 10.0)


def switch(p: LsdProblem, x, xc: float):
    """s_{eps_b}(|x - x_c| - x_b): the rise over [x_b - eps_b/2, x_b + eps_b/2]."""
    t = np.abs(x - xc) - x_barrier(p)
    return smooth_step((t + 0.5 * p.eps_b) / p.eps_b)


def v_nuclei(p: LsdProblem, x):
    """One-electron potential: soft-Coulomb nuclei (reading above) and an
    optional harmonic term."""
    x = np.asarray(x, dtype=float)
    v = 0.5 * p.harmonic * x * x
    for (xa, za) in p.nuclei:
        v = v - za / np.sqrt((x - xa) ** 2 + p.eta_en ** 2)
    return v


def gl_rule(lo: float, hi: float, panel: float, q: int, breaks=()):
    """Composite Gauss-Legendre rule on [lo, hi] with panel edges at the given
    breakpoints (where the integrand is only piecewise smooth) and panels of
    width <= panel between them."""
    pts = sorted(set([lo, hi] + [b for b in breaks if lo < b < hi]))
    t, wt = leggauss(q)
    xs, ws = [], []
    for s0, s1 in zip(pts[:-1], pts[1:]):
        n = max(1, int(math.ceil((s1 - s0) / panel - 1e-12)))
        edges = np.linspace(s0, s1, n + 1)
        for e0, e1 in zip(edges[:-1], edges[1:]):
            xs.append(0.5 * (e1 - e0) * t + 0.5 * (e1 + e0))
            ws.append(0.5 * (e1 - e0) * wt)
    return np.concatenate(xs), np.concatenate(ws)


def barrier_breaks(p: "LsdProblem", xc: float):
    """Where the C^2 step of the barrier starts and ends around x_c."""
    xb, e = x_barrier(p), 0.5 * p.eps_b
    return (xc - xb - e, xc - xb + e, xc + xb - e, xc + xb + e)


def local_margin(p: "LsdProblem") -> float:
    """How far past the outermost centres the integrals run: past the barrier's
    rise and 8 standard deviations of a Gaussian (its value below e^-32)."""
    return max(p.eps_b, 8.0 / math.sqrt(2.0 * gaussian_exponent(p)))


def gaussian_table(centres: np.ndarray, delta: float, x: np.ndarray):
    """B[k, n] = exp(-delta (x_n - alpha_k)^2) and its x-derivative."""
    d = x[None, :] - centres[:, None]
    g = np.exp(-delta * d * d)
    return g, -2.0 * delta * d * g


@dataclass
class Orbitals:
    lam: np.ndarray        # [M] eigenvalues lambda_l^i
    coef: np.ndarray       # [kd, M] Gaussian coefficients
    centres: np.ndarray    # [kd]
    delta: float
    xc: float

    def values(self, x: np.ndarray):
        g, dg = gaussian_table(self.centres, self.delta, x)
        return self.coef.T @ g, self.coef.T @ dg


def local_orbitals(p: LsdProblem, i: int) -> Orbitals:
    """Sec. 3.2: the M lowest eigenpairs of
    1/2 int a phi' psi' + int (V_en + V_b) phi psi = lambda int phi psi
    (weak form of Eq. BARPOT's eigenproblem) in the Gaussian basis of D_i."""
    _, _, xc = subdomain(p, i)
    xb = x_barrier(p)
    delta = gaussian_exponent(p)
    centres = np.linspace(xc - xb, xc + xb, p.kd)
    m = local_margin(p)
    x, w = gl_rule(xc - xb - m, xc + xb + m, p.panel, p.q_p, barrier_breaks(p, xc))
    g, dg = gaussian_table(centres, delta, x)
    s = switch(p, x, xc)
    a = 1.0 - s
    V = v_nuclei(p, x) + p.v_inf * s
    S = (g * w) @ g.T
    H = 0.5 * (dg * (w * a)) @ dg.T + (g * (w * V)) @ g.T
    lam, X = eigh(H, S)
    lam, X = lam[: p.M], X[:, : p.M].copy()
    # sign: int phi exp(0.37 (x - xc)) dx > 0
    proj = (g * (w * np.exp(0.37 * (x - xc)))).sum(axis=1) @ X
    X *= np.where(proj < 0.0, -1.0, 1.0)[None, :]
    return Orbitals(lam=lam, coef=X, centres=centres, delta=delta, xc=xc)


def all_orbitals(p: LsdProblem) -> List[Orbitals]:
    return [local_orbitals(p, i) for i in range(p.L)]


def global_rule(p: LsdProblem):
    """The rule of every integral between orbitals: [a, b] widened by the
    orbital supports and the local margin."""
    a, b = p.box
    lo0, hi0, _ = subdomain(p, 0)
    m = x_barrier(p) - 0.5 * (hi0 - lo0) + local_margin(p)
    return gl_rule(a - p.overlap / 2 - m, b + p.overlap / 2 + m, p.panel, p.q_p)


@dataclass
class OneElectron:
    S: np.ndarray   # [L M, L M] overlaps <phi_l^i, phi_m^j>
    h: np.ndarray   # [L M, L M] int 1/2 phi' psi' + V_en phi psi (Appendix A's I_lm^ij)
    J: np.ndarray   # [L M, L M] int x phi psi (Appendix A's J_lm^ij)


def orbital_table(p: LsdProblem, orbs: Sequence[Orbitals], x: np.ndarray):
    """Values and derivatives of every orbital (index i M + l) at x."""
    vals, ders = zip(*(o.values(x) for o in orbs))
    return np.concatenate(vals, axis=0), np.concatenate(ders, axis=0)


def one_electron(p: LsdProblem, orbs: Sequence[Orbitals]) -> OneElectron:
    """Appendix A, I_lm^ij and J_lm^ij, and the overlaps, over the whole line:
    the kinetic term in its symmetric weak form 1/2 int phi' psi' (= -1/2 int
    phi psi'' for orbitals that vanish at infinity)."""
    x, w = global_rule(p)
    F, dF = orbital_table(p, orbs, x)
    S = (F * w) @ F.T
    h = 0.5 * (dF * w) @ dF.T + (F * (w * v_nuclei(p, x))) @ F.T
    J = (F * (w * x)) @ F.T
    return OneElectron(S=S, h=h, J=J)


def two_electron(p: LsdProblem, orbs: Sequence[Orbitals], idx: Sequence[int]) -> np.ndarray:
    """Appendix A, I_mpqr = int int phi_m phi_p (x) W(x - s) phi_q phi_r (s) for
    the orbitals idx (global indices i M + l), W the soft-Coulomb e-e
    interaction: E[m, p, q, r] with the pair densities phi_m phi_p at the
    nodes of the global rule."""
    x, w = global_rule(p)
    F, _ = orbital_table(p, orbs, x)
    F = F[list(idx)]
    n = len(idx)
    W = p.ee_coef / np.sqrt((x[:, None] - x[None, :]) ** 2 + p.eta_ee ** 2)
    P = (F[:, None, :] * F[None, :, :]).reshape(n * n, -1) * w[None, :]
    E = P @ W @ P.T
    return E.reshape(n, n, n, n)


TIE = 1e-9  # orbital-energy sums this close (relative) count as equal


def lsd_pairs(p: LsdProblem, orbs: Sequence[Orbitals], i: int, j: int) -> List[Tuple[int, int]]:
    """The K determinants of Omega_{i,j} (reading above): (l, p) with the
    orbital phi_l^i in the first slot and phi_p^j in the second, ranked by
    lambda_l^i + lambda_p^j; sums within TIE (relative) are ties, broken by
    (l, p) (mirror-image subdomains have equal spectra, so exact ties occur
    and rounding must not order them)."""
    cand = [(l, q) for l in range(p.M) for q in range(p.M) if (i != j or l < q)]
    if len(cand) < p.K:
        raise ValueError(f"Omega_({i},{j}) has {len(cand)} candidate determinants, fewer than K = {p.K}")
    e = [orbs[i].lam[l] + orbs[j].lam[q] for (l, q) in cand]

    def before(u, v):
        d = e[u] - e[v]
        if abs(d) <= TIE * (1.0 + abs(e[u]) + abs(e[v])):
            return cand[u] < cand[v]
        return d < 0.0

    rank = [sum(1 for v in range(len(cand)) if v != u and before(v, u)) for u in range(len(cand))]
    if sorted(rank) != list(range(len(cand))):
        raise ValueError(f"Omega_({i},{j}): the tie rule does not order the candidates")
    out = [None] * len(cand)
    for u, r in enumerate(rank):
        out[r] = cand[u]
    return out[: p.K]


def lsd_gram(p: LsdProblem, oe: OneElectron, pa, ia: Tuple[int, int], pb, ib: Tuple[int, int]) -> np.ndarray:
    """<v_a, v_b> for the determinants pa of Omega_ia and pb of Omega_ib:
    <det(a,b), det(c,d)>/2 expands to <a,c><b,d> - <a,d><b,c> (Eq. LSD)."""
    S = oe.S
    G = np.zeros((len(pa), len(pb)))
    for r, (l, q) in enumerate(pa):
        a, b = ia[0] * p.M + l, ia[1] * p.M + q
        for c_, (m, t) in enumerate(pb):
            c, d = ib[0] * p.M + m, ib[1] * p.M + t
            G[r, c_] = S[a, c] * S[b, d] - S[a, d] * S[b, c]
    return G


def lsd_hamiltonian(p: LsdProblem, orbs: Sequence[Orbitals], oe: OneElectron, i: int, j: int):
    """Matrix of H0 = h(1) + h(2) + W(x1 - x2) between the K determinants of
    Omega_{i,j} (Appendix A): <det(a,b)|h(1)+h(2)|det(c,d)> =
    h_ac S_bd + S_ac h_bd - h_ad S_bc - S_ad h_bc and <det(a,b)|W|det(c,d)> =
    I_acbd - I_adbc, with the determinants normalised by 1/sqrt(2)."""
    pairs = lsd_pairs(p, orbs, i, j)
    idx = sorted(set([i * p.M + l for l in range(p.M)] + [j * p.M + q for q in range(p.M)]))
    pos = {g: k for k, g in enumerate(idx)}
    E = two_electron(p, orbs, idx)
    S, h = oe.S, oe.h
    K = len(pairs)
    Hm = np.zeros((K, K))
    for r, (l, q) in enumerate(pairs):
        a, b = i * p.M + l, j * p.M + q
        for c_, (m, t) in enumerate(pairs):
            c, d = i * p.M + m, j * p.M + t
            one = h[a, c] * S[b, d] + S[a, c] * h[b, d] - h[a, d] * S[b, c] - S[a, d] * h[b, c]
            two = E[pos[a], pos[c], pos[b], pos[d]] - E[pos[a], pos[d], pos[b], pos[c]]
            Hm[r, c_] = one + two
    Sm = lsd_gram(p, oe, pairs, (i, j), pairs, (i, j))
    return pairs, Sm, Hm


def lsd_value(orbs: Sequence[Orbitals], i: int, j: int, l: int, q: int, x1, x2):
    """v_{l,q}^{i,j}(x1, x2) pointwise (Eq. LSD)."""
    a1, _ = orbs[i].values(np.atleast_1d(x1))
    a2, _ = orbs[i].values(np.atleast_1d(x2))
    b1, _ = orbs[j].values(np.atleast_1d(x1))
    b2, _ = orbs[j].values(np.atleast_1d(x2))
    return (a1[l] * b2[q] - a2[l] * b1[q]) / math.sqrt(2.0)
