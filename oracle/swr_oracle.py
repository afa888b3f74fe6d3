"""Plain FP64 CPU oracle of the Schwarz Waveform Relaxation (SWR) Galerkin sweep.

TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the benchmark's
CPU-baseline / reference arm may import or run this module.  The product path
(the CUDA library and its Python binding) never calls it and shares no code
with it: different algorithms (dense 2-D quadrature and direct generalized
solves here, Kronecker/sum-factorised assembly and explicit inverses there),
different geometry logic (float containment tests here, panel indices there).

Every function restates one passage of the paper (E. Lorin, "Domain
Decomposition Method for the N-body Time-Independent and Time-Dependent
Schroedinger Equation"), in plain, slow numpy:

  geometry ............ opening of Sec. 6 (overlapping hypercubes Omega_{i+jL})
  basis ............... Sec. 2, Eq. gauss1d and the tensor products v_{l,p}
  local systems ....... Sec. 5.1 "Construction of the local approximate
                         solutions": A_i, H~_i (incl. Robin R_i), Q_i
  Robin TC ............ Sec. 5.1, Eq. RTC; averaging over several overlapping
                         subdomains (Sec. 5.1, multi-subdomain zones)
  basis reduction ..... Sec. 2's Gaussian overlaps are ill-conditioned: per
                         coordinate Cholesky when every pivot >= tau * max
                         diagonal, else canonical orthogonalisation (eigen-
                         vectors with lambda > tau lambda_max), the local
                         basis being the tensor product of the kept
                         per-coordinate functions
  initial data ........ Sec. 6.1 (Test 1.a): c~ = <phi0, v>, A c = c~
  time stepping ....... Sec. 5.4 step 2: Crank-Nicolson (real time), implicit
                         Euler (imaginary time), step 4 normalisation
  inner NGF stop ...... Sec. 5.2 (||phi^{n+1} - phi^n|| <= delta)
  reconstruction ...... Sec. 5.3 (average over the covering subdomains)
  residual ............ Sec. 6.2, Eq. residueRT and Sec. 6.3, Eq. residueIT
  interface mismatch .. Sec. 4.1, Eq. CVTOT and Sec. 4.2, Eq. CVTOT2

Readings where the paper is silent or garbled:
  * weak form of -kappa*Lap with the Robin condition (d_n + mu) psi = g gives
    H~ = kappa (K + mu R) + V and a source +kappa*b (imaginary time) or
    -kappa*b (real time), kappa = 1/2 from H0 (Sec. 1.1);
  * edges on the outer boundary carry the natural condition (no term);
  * normalisation by the partition-of-unity norm sum_i int chi_i |phi_i|^2,
    chi_i = 1 / #(subdomains whose closure contains x);
  * Robin data at a node = average over all other subdomains whose closure
    contains the node (closed-set reading of the averaged condition);
  * g^(0) = 0; a shorter previous window is held at its last value;
  * in imaginary time the Robin data at t_{n+1} is taken from the neighbour's
    iterate before the normalisation of t_{n+1} (the transmission condition of
    system SIT acts on (t_n, t_{n+1}), the normalisation at t_{n+1}^+); with
    this reading the local Robin eigenproblem is a fixed point of the scheme;
  * Res(k)^2 = sum_n dt sum_i sum_{Gamma-nodes} w |u_i^(k) - u_i^(k-1)|^2,
    with u^(0) = 0, over the interior interfaces only;
  * CVTOT(k)^2 = sum_n dt (sum_{(i,j)} ||psi_i^(k) - psi_j^(k)||_{Gamma_{i;j}})^2
    over n = 1..W, Gamma_{i;j} = interface nodes of Omega_i in closure(Omega_j);
  * field e(t) = E0 sin^2(pi t/T) sin(omega t + phase) on [0, T], 0 after.

Parity pins: see tests/test_oracle_pins.py (closed forms, invariants, brute
force).  No function of this module is left without a pin.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np
import scipy.linalg as sla
from numpy.polynomial.legendre import leggauss

TISE = "tise"
TDSE = "tdse"


# ------------------------------------------------------------------ geometry

def sub_interval(inst, k: int):
    """1-D subdomain k (0-based): [a_k - eps/2, b_k + eps/2], a_k = a + k(b-a)/L,
    b_k = a + (k+1)(b-a)/L (opening of Sec. 6, with the index shift the text
    uses for a_i read also for c_i)."""
    a, b = inst.box
    H = (b - a) / inst.L
    return a + k * H - 0.5 * inst.overlap, a + (k + 1) * H + 0.5 * inst.overlap


def sub_multi_index(inst, sid: int):
    """Omega_{i1 + L*i2} (0-based), Sec. 4.1 notation."""
    idx = []
    for _ in range(inst.n_elec):
        idx.append(sid % inst.L)
        sid //= inst.L
    return idx


def contains_closed(inst, sid: int, x) -> bool:
    """x in closure(Omega_sid), by direct comparison."""
    for d, k in enumerate(sub_multi_index(inst, sid)):
        lo, hi = sub_interval(inst, k)
        if not (lo <= x[d] <= hi):
            return False
    return True


def cover_count(inst, x) -> int:
    return sum(1 for j in range(inst.n_sub) if contains_closed(inst, j, x))


# ------------------------------------------------------------- quadrature

def nodes_1d(inst, k: int):
    """Composite Gauss-Legendre rule on subdomain interval k: the overlap bands
    [lo, lo+eps] and [hi-eps, hi] are one panel each, the middle zone is cut
    into n_mid equal panels; q_p nodes per panel."""
    lo, hi = sub_interval(inst, k)
    eps = inst.overlap
    t, wt = leggauss(inst.q_p)
    xs, ws = [], []
    m = inst.n_mid
    brk = [lo, lo + eps] + [lo + eps + (hi - lo - 2 * eps) * j / m for j in range(1, m)] + [hi - eps, hi]
    for (p0, p1) in zip(brk[:-1], brk[1:]):
        xs.append(0.5 * (p1 - p0) * t + 0.5 * (p1 + p0))
        ws.append(0.5 * (p1 - p0) * wt)
    return np.concatenate(xs), np.concatenate(ws)


# ------------------------------------------------------------------ basis

def centres_1d(inst, sid: int, k: int):
    lo, hi = sub_interval(inst, k)
    kd = inst.k_d_of(sid)
    return np.linspace(lo, hi, kd)


def phi(x, alpha, delta):
    """phi_j(x) = exp(-delta (x - alpha_j)^2), Eq. gauss1d."""
    return np.exp(-delta * (x - alpha) ** 2)


def dphi(x, alpha, delta):
    return -2.0 * delta * (x - alpha) * np.exp(-delta * (x - alpha) ** 2)


class Basis:
    """Tensor-product Gaussian basis of one subdomain: v_m = prod_d phi_{a_d}(x_d),
    m = a_1 + K_d a_2 (Sec. 2, v_{l,p}(x1,x2) = phi_l(x1) phi_p(x2)).

    With per-coordinate transforms T_d (K_d x r_d, canonical orthogonalisation)
    the functions of coordinate d are phi'_i = sum_a T_d[a, i] phi_a and the
    basis is their tensor product (index i_1 + r_1 i_2): each factor is
    evaluated per coordinate, so the products stay O(1) functions."""

    def __init__(self, inst, sid: int, transforms=None):
        self.inst = inst
        self.sid = sid
        self.N = inst.n_elec
        self.kd = inst.k_d_of(sid)
        self.delta = inst.delta_of(sid)
        self.midx = sub_multi_index(inst, sid)
        self.centres = [centres_1d(inst, sid, k) for k in self.midx]
        self.T = list(transforms) if transforms is not None else [None] * self.N
        self.r = [self.kd if t is None else t.shape[1] for t in self.T]
        self.K = int(np.prod(self.r))

    def _factor(self, x, d, fn):
        f = fn(x[:, None], self.centres[d][None, :], self.delta)
        return f if self.T[d] is None else f @ self.T[d]

    def _tensor(self, f, npts):
        if self.N == 1:
            return f[0]
        # m = a + r_1 * b  ->  column index b*r_1 + a
        return (f[1][:, :, None] * f[0][:, None, :]).reshape(npts, -1)

    def values(self, X):
        """X: (P, N) points -> (P, K) basis values."""
        X = np.atleast_2d(X)
        return self._tensor([self._factor(X[:, d], d, phi) for d in range(self.N)], X.shape[0])

    def grad(self, X, dim: int):
        """d/dx_dim of every basis function at the points X."""
        X = np.atleast_2d(X)
        return self._tensor([self._factor(X[:, d], d, dphi if d == dim else phi) for d in range(self.N)],
                            X.shape[0])


# --------------------------------------------------------------- potential

def potential(inst, X):
    """V(x) = sum_e [sum_A -Z_A/sqrt((x_e-x_A)^2+eta_en^2) + harmonic x_e^2/2]
              + ee_coef / sqrt((x_1-x_2)^2 + eta_ee^2)   (Sec. 1.1 H0 with the
    regularisation of Eq. pseudo)."""
    X = np.atleast_2d(X)
    V = np.zeros(X.shape[0])
    for e in range(inst.n_elec):
        xe = X[:, e]
        for (xa, za) in inst.nuclei:
            V -= za / np.sqrt((xe - xa) ** 2 + inst.eta_en ** 2)
        V += 0.5 * inst.harmonic * xe ** 2
    if inst.n_elec == 2 and inst.ee_coef != 0.0:
        V += inst.ee_coef / np.sqrt((X[:, 0] - X[:, 1]) ** 2 + inst.eta_ee ** 2)
    return V


def field_e(inst, t: float) -> float:
    """Dipole field amplitude e(t) along every coordinate (Sec. 1.2)."""
    E0, T, om, ph = inst.field
    if E0 == 0.0 or t < 0.0 or t > T:
        return 0.0
    return E0 * math.sin(math.pi * t / T) ** 2 * math.sin(om * t + ph)


# -------------------------------------------------------- local subdomain

@dataclass
class GammaSet:
    """Interior interface nodes of one subdomain (parts of its boundary that lie
    inside the global domain), with quadrature weights and outward normals."""
    X: np.ndarray            # (G, N) node coordinates
    w: np.ndarray            # (G,) surface quadrature weights (1 for N = 1)
    dim: np.ndarray          # (G,) coordinate normal to the edge
    sign: np.ndarray         # (G,) +1 on the hi side, -1 on the lo side


@dataclass
class Local:
    sid: int
    basis: Basis
    X: np.ndarray            # (Q, N) volume nodes
    w: np.ndarray            # (Q,) volume weights
    chi: np.ndarray          # (Q,) partition-of-unity weights
    A: np.ndarray = None
    Kf: np.ndarray = None    # int grad v . grad v
    V: np.ndarray = None
    Qx: np.ndarray = None    # sum_e <x_e v, v>
    R: np.ndarray = None     # Robin boundary mass on the interior interfaces
    Achi: np.ndarray = None
    Hchi: np.ndarray = None  # kappa*Kf_chi + V_chi (energy numerator)
    Qchi: np.ndarray = None
    Ht: np.ndarray = None    # H~ = kappa (Kf + mu R) + V
    gamma: GammaSet = None
    own_vals: np.ndarray = None   # (G, K) basis values on Gamma nodes
    contrib: list = None     # per Gamma node: list of contributing subdomains
    c0: np.ndarray = None


def overlap_1d(inst, basis: "Basis", d: int) -> np.ndarray:
    """S_d[a][c] = int phi_a phi_c over the subdomain's interval of coordinate d
    (the composite Gauss-Legendre rule of the volume quadrature)."""
    x, w = nodes_1d(inst, basis.midx[d])
    F = phi(x[:, None], basis.centres[d][None, :], basis.delta)
    return F.T @ (w[:, None] * F)


def orth_coordinate(S: np.ndarray, tau: float):
    """Per-coordinate orthogonalisation of Sec. 2's Gaussian basis (reading:
    the Gaussian overlaps are ill-conditioned, so the basis is reduced when
    they are numerically singular).  Cholesky S = L L^T succeeds when every
    pivot is at least tau times the largest diagonal entry: the whole basis is
    kept (None).  Otherwise canonical orthogonalisation: S = U diag(lam) U^T,
    keep the eigenvectors with lam > tau * lam_max, X = U_r lam_r^(-1/2)."""
    n = S.shape[0]
    dmax = float(np.max(np.diag(S)))
    Lc = np.array(S, dtype=float)
    ok = True
    for j in range(n):  # plain right-looking Cholesky, pivot by pivot
        pj = Lc[j, j] - float(np.dot(Lc[j, :j], Lc[j, :j]))
        if not pj > tau * dmax:
            ok = False
            break
        Lc[j, j] = math.sqrt(pj)
        for i in range(j + 1, n):
            Lc[i, j] = (Lc[i, j] - float(np.dot(Lc[i, :j], Lc[j, :j]))) / Lc[j, j]
    if ok:
        return None
    lam, U = np.linalg.eigh(S)
    keep = lam > tau * float(np.max(lam))
    return U[:, keep] / np.sqrt(lam[keep])[None, :]


def gamma_nodes(inst, sid: int) -> GammaSet:
    midx = sub_multi_index(inst, sid)
    N = inst.n_elec
    Xs, ws, dims, signs = [], [], [], []
    for d in range(N):
        k = midx[d]
        lo, hi = sub_interval(inst, k)
        for side, pos, sgn in ((0, lo, -1.0), (1, hi, 1.0)):
            interior = (k > 0) if side == 0 else (k < inst.L - 1)
            if not interior:
                continue
            if N == 1:
                Xs.append(np.array([[pos]]))
                ws.append(np.array([1.0]))
            else:
                o = 1 - d
                xo, wo = nodes_1d(inst, midx[o])
                P = np.zeros((xo.size, 2))
                P[:, d] = pos
                P[:, o] = xo
                Xs.append(P)
                ws.append(wo)
            dims.append(np.full(ws[-1].size, d))
            signs.append(np.full(ws[-1].size, sgn))
    if not Xs:
        return GammaSet(np.zeros((0, N)), np.zeros(0), np.zeros(0, int), np.zeros(0))
    return GammaSet(np.concatenate(Xs), np.concatenate(ws),
                    np.concatenate(dims).astype(int), np.concatenate(signs))


def phi0_values(inst, X):
    X = np.atleast_2d(X)
    r2 = np.zeros(X.shape[0])
    for d in range(inst.n_elec):
        r2 += (X[:, d] - inst.phi0_center[d]) ** 2
    return np.exp(-inst.phi0_gamma * r2)


def build_local(inst, sid: int) -> Local:
    """Galerkin matrices of Omega_sid by straightforward quadrature on the
    tensor grid of composite Gauss-Legendre nodes (Sec. 5.1), in the basis
    kept by the per-coordinate orthogonalisation test (orth_coordinate)."""
    raw = Basis(inst, sid)
    basis = Basis(inst, sid, [orth_coordinate(overlap_1d(inst, raw, d), inst.orth_tau) for d in range(raw.N)])
    midx = basis.midx
    N = inst.n_elec
    x1, w1 = nodes_1d(inst, midx[0])
    if N == 1:
        X = x1[:, None]
        w = w1.copy()
    else:
        x2, w2 = nodes_1d(inst, midx[1])
        # point p = q1 + q*q2
        X = np.stack([np.tile(x1, x2.size), np.repeat(x2, x1.size)], axis=1)
        w = np.tile(w1, x2.size) * np.repeat(w2, x1.size)
    chi = np.array([1.0 / cover_count(inst, x) for x in X])
    loc = Local(sid=sid, basis=basis, X=X, w=w, chi=chi)

    B = basis.values(X)
    G = [basis.grad(X, d) for d in range(N)]
    Vx = potential(inst, X)
    xsum = X.sum(axis=1)
    loc.A = B.T @ (w[:, None] * B)
    loc.Kf = sum(g.T @ (w[:, None] * g) for g in G)
    loc.V = B.T @ ((w * Vx)[:, None] * B)
    loc.Qx = B.T @ ((w * xsum)[:, None] * B)
    wc = w * chi
    loc.Achi = B.T @ (wc[:, None] * B)
    loc.Hchi = inst.kinetic * sum(g.T @ (wc[:, None] * g) for g in G) + B.T @ ((wc * Vx)[:, None] * B)
    loc.Qchi = B.T @ ((wc * xsum)[:, None] * B)

    gam = gamma_nodes(inst, sid)
    loc.gamma = gam
    Bg = basis.values(gam.X) if gam.w.size else np.zeros((0, basis.K))
    loc.own_vals = Bg
    loc.R = Bg.T @ (gam.w[:, None] * Bg)
    loc.Ht = inst.kinetic * (loc.Kf + inst.mu * loc.R) + loc.V
    if np.iscomplexobj(loc.Ht) and np.all(np.imag(loc.Ht) == 0):
        loc.Ht = np.real(loc.Ht)
    # contributors of every interface node: the other subdomains whose closure holds it
    loc.contrib = [[j for j in range(inst.n_sub) if j != sid and contains_closed(inst, j, x)]
                   for x in gam.X]
    # initial data: c~_l = <phi0, v_l>_{Omega_i}, A c = c~  (Sec. 6.1)
    ct = B.T @ (w * phi0_values(inst, X))
    loc.c0 = np.linalg.solve(loc.A, ct)
    return loc


# ------------------------------------------------------------------ traces

class TraceOps:
    """Per target subdomain i: value / normal-derivative rows of every
    contributing subdomain j at i's interface nodes."""

    def __init__(self, inst, locs: List[Local]):
        self.inst = inst
        self.locs = locs
        self.ops = []
        for li in locs:
            gam = li.gamma
            G = gam.w.size
            per_j: Dict[int, tuple] = {}
            cnt = np.array([len(c) for c in li.contrib], dtype=float)
            for j in range(inst.n_sub):
                rows = [g for g in range(G) if j in li.contrib[g]]
                if not rows:
                    continue
                rows = np.array(rows)
                bj = locs[j].basis
                P = gam.X[rows]
                vals = bj.values(P)
                ders = np.zeros_like(vals)
                for r, g in enumerate(rows):
                    ders[r] = gam.sign[g] * bj.grad(P[r:r + 1], gam.dim[g])[0]
                per_j[j] = (rows, vals, ders)
            self.ops.append((per_j, cnt))

    def robin_data(self, coeffs: List[np.ndarray]) -> List[np.ndarray]:
        """g_i = (1/|J|) sum_{j in J} (n_i . grad + mu) psi_j at i's nodes
        (Eq. RTC); for the classical SWR (Dirichlet condition psi_i = psi_j,
        Sec. 4) imposed by penalty with the same boundary term, the data is
        (1/|J|) sum_{j in J} mu psi_j."""
        mu = self.inst.mu
        robin = getattr(self.inst, "tc", "robin") != "dirichlet"
        out = []
        for i, (per_j, cnt) in enumerate(self.ops):
            G = cnt.size
            dt = complex if (np.iscomplexobj(coeffs[0]) or np.iscomplexobj(mu)) else float
            g = np.zeros(G, dtype=dt)
            for j, (rows, vals, ders) in per_j.items():
                g[rows] += (ders @ coeffs[j] if robin else 0.0) + mu * (vals @ coeffs[j])
            with np.errstate(invalid="ignore", divide="ignore"):
                g = np.where(cnt > 0, g / np.maximum(cnt, 1), 0.0)
            out.append(g)
        return out

    def own_values(self, coeffs: List[np.ndarray]) -> List[np.ndarray]:
        return [li.own_vals @ c for li, c in zip(self.locs, coeffs)]


# ------------------------------------------------------------------ solver

@dataclass
class IterRecord:
    k: int
    res: float
    n_win: int
    cvtot: Optional[float] = None
    # ||c^{n} - c^{n-1}||_chi of the inner NGF stop test (Sec. 5.2) at the last
    # steps of the window: {n: value} for n = n_win - 1, n_win (imaginary time with
    # the stop test only)
    stop_values: Optional[dict] = None
    energy: Optional[float] = None
    norm2: Optional[float] = None
    dipole: Optional[float] = None


@dataclass
class SWRResult:
    records: List[IterRecord] = field(default_factory=list)
    coeffs: List[np.ndarray] = None          # final coefficients (last step, last iteration)
    own_traces: List[np.ndarray] = None       # u_i at Gamma nodes, (n_win+1, G_i)
    robin: List[np.ndarray] = None            # g_i at Gamma nodes, (n_win+1, G_i)
    locs: List[Local] = None
    converged: bool = False

    @property
    def res(self):
        return [r.res for r in self.records]


def pou_norm2(locs, coeffs):
    return float(np.real(sum(np.vdot(c, l.Achi @ c) for l, c in zip(locs, coeffs))))


def energy(locs, coeffs):
    """PoU-weighted Rayleigh quotient sum_i int chi_i (kappa|grad psi_i|^2 + V|psi_i|^2)
    / sum_i int chi_i |psi_i|^2."""
    num = sum(np.vdot(c, l.Hchi @ c) for l, c in zip(locs, coeffs))
    return float(np.real(num)) / pou_norm2(locs, coeffs)


def psi_at_nodes(loc: Local, c: np.ndarray) -> np.ndarray:
    """psi_i at the subdomain's own volume nodes (point p = q1 + q*q2)."""
    return loc.basis.values(loc.X) @ c


def reconstruct_at(inst, locs, coeffs, X):
    """Averaged global wavefunction (Sec. 5.3): mean of psi_j over every
    subdomain whose closure contains the point."""
    X = np.atleast_2d(X)
    out = np.zeros(X.shape[0], dtype=complex if np.iscomplexobj(coeffs[0]) else float)
    for p, x in enumerate(X):
        js = [j for j in range(inst.n_sub) if contains_closed(inst, j, x)]
        out[p] = sum(locs[j].basis.values(x[None, :])[0] @ coeffs[j] for j in js) / len(js)
    return out


def schwarz_residual(locs, dt: float, u_hist, u_prev) -> float:
    """Res(k) of Eq. residueIT (Sec. 6.3) / Eq. residueRT (Sec. 6.2): the
    L2(0,T) norm in time of the sum over subdomains of the L2 norm on the
    interior interfaces of u_i^(k) - u_i^(k-1).

    u_hist[i]: (W+1, G_i) own traces of iteration k at steps 0..W; u_prev the
    same for iteration k-1 (None for k = 1: u^(0) = 0).  Time integral by the
    rectangle rule with weight dt at t_1..t_max(W, W'); a window shorter than
    the other is held at its last value.  Interface integral by the surface
    quadrature weights of the Gamma nodes."""
    n_done = u_hist[0].shape[0] - 1
    n_cmp = max(n_done, 0 if u_prev is None else u_prev[0].shape[0] - 1)
    r2 = 0.0
    for i, loc in enumerate(locs):
        w = loc.gamma.w
        for n in range(1, n_cmp + 1):
            a = u_hist[i][min(n, n_done)]
            b = np.zeros_like(a) if u_prev is None else u_prev[i][min(n, u_prev[i].shape[0] - 1)]
            r2 += dt * float(np.sum(w * np.abs(a - b) ** 2))
    return math.sqrt(r2)


def interface_mismatch(locs, ops: "TraceOps", hist, dt: float) -> float:
    """CVTOT of Eq. CVTOT (Sec. 4.1) and Eq. CVTOT2 (Sec. 4.2): at each time,
    the sum over ordered pairs (i, j) of the L2(Gamma_{i;j}) norm of
    psi_i^(k) - psi_j^(k), Gamma_{i;j} the part of the interior boundary of
    Omega_i inside closure(Omega_j); then the L2(0,T) norm of that sum.

    hist: iterates c^n of iteration k for n = 0..W (list over steps of lists
    over subdomains; the normalised state in imaginary time).  Reading: the
    same rectangle rule in time as Res(k) (weight dt at t_1..t_W), the surface
    quadrature of the Gamma nodes on each Gamma_{i;j}.  Unlike Res(k) it does
    not tend to 0: at the discrete fixed point psi_i and psi_j still differ on
    Gamma_{i;j} by the discretisation error."""
    total = 0.0
    for n in range(1, len(hist)):
        coeffs = hist[n]
        c_n = 0.0
        for i, (per_j, _cnt) in enumerate(ops.ops):
            loc = locs[i]
            for j, (rows, vals, _ders) in per_j.items():
                diff = loc.own_vals[rows] @ coeffs[i] - vals @ coeffs[j]
                c_n += math.sqrt(float(np.sum(loc.gamma.w[rows] * np.abs(diff) ** 2)))
        total += dt * c_n * c_n
    return math.sqrt(total)


def assemble(inst) -> List[Local]:
    return [build_local(inst, s) for s in range(inst.n_sub)]


def run_swr(inst, kmax: int = 50, tol: float = 1e-8, locs: Optional[List[Local]] = None,
            g_init: Optional[List[np.ndarray]] = None, k_min: int = 1,
            keep_all: bool = False, step_energies: bool = False) -> SWRResult:
    """Schwarz iteration loop of Sec. 5.4 (steps 1-5) for the imaginary-time
    (TISE/NGF or heat, implicit Euler) or real-time (TDSE, Crank-Nicolson)
    local problems, with Robin transmission conditions.

    g_init: optional Robin data of a zeroth iteration, list over subdomains
    of arrays (n0+1, G_i) indexed by time step (row 0 = t_0).
    """
    if locs is None:
        locs = assemble(inst)
    ops = TraceOps(inst, locs)
    S = inst.n_sub
    kappa = inst.kinetic
    dt = inst.dt
    tdse = inst.mode == TDSE
    fixed = inst.window()
    cplx = tdse or np.iscomplexobj(inst.mu)

    def b_vec(i, g):  # b_l = sum_Gamma w g v_l
        return locs[i].own_vals.T @ (locs[i].gamma.w * g)

    # antisymmetric states (Appendix A: psi_sigma(i)(x1, x2) = -psi_i(x2, x1) with
    # sigma the mirror subdomain across x1 = x2): every step acts on the
    # antisymmetric part of its input, P(c)_i = (c_i - swap(c_sigma(i))) / 2,
    # swap transposing the (coordinate-2, coordinate-1) coefficient matrix
    anti = getattr(inst, "symmetry", "none") == "antisymmetric"

    def mirror(i):
        return (i // inst.L) + inst.L * (i % inst.L)

    def proj(vecs):
        out = []
        for i in range(S):
            j = mirror(i)
            r1, r2 = locs[j].basis.r
            out.append(0.5 * (vecs[i] - vecs[j].reshape(r2, r1).T.reshape(-1)))
        return out

    # initial data (step 1), normalised for the NGF; antisymmetric states start
    # from the antisymmetric part of the projected initial Gaussian
    c0 = [l.c0.astype(complex if cplx else float) for l in locs]
    if anti:
        c0 = proj(c0)
    if inst.mode == TISE and inst.normalize:
        s0 = math.sqrt(pou_norm2(locs, c0))
        c0 = [c / s0 for c in c0]

    if g_init is not None:
        g_prev = [np.asarray(g) for g in g_init]
        n_prev = g_prev[0].shape[0] - 1
    else:
        g_prev = None
        n_prev = 0
    u_prev = None

    # imaginary time: (A + dt H~) c~^{n+1} = A c^n + kappa dt b^{n+1}
    lu_ie = None
    if not tdse:
        lu_ie = [sla.lu_factor(l.A + dt * l.Ht) for l in locs]

    result = SWRResult(locs=locs)
    for k in range(1, kmax + 1):
        def g_at(i, n):
            if g_prev is None or n_prev < 0:
                return np.zeros(locs[i].gamma.w.size)
            return g_prev[i][min(n, n_prev)]

        coeffs = [c.copy() for c in c0]
        hist = [coeffs]          # normalised iterates c^n (solution at t_n^+)
        hist_raw = [coeffs]      # iterates before normalisation (solution at t_n^-)
        n_win = fixed if fixed > 0 else inst.max_steps
        n_done = 0
        stop_q = {}
        for n in range(n_win):
            new = []
            if tdse:
                t0, t1 = n * dt, (n + 1) * dt
                e0, e1 = field_e(inst, t0), field_e(inst, t1)
                for i, l in enumerate(locs):
                    M1 = l.A + 0.5j * dt * (l.Ht + e1 * l.Qx)
                    M0 = l.A - 0.5j * dt * (l.Ht + e0 * l.Qx)
                    rhs = M0 @ coeffs[i] + 0.5j * dt * kappa * (b_vec(i, g_at(i, n + 1)) + b_vec(i, g_at(i, n)))
                    new.append(np.linalg.solve(M1, rhs))
            else:
                cin = proj(coeffs) if anti else coeffs
                bin_ = [b_vec(i, g_at(i, n + 1)) for i in range(S)]
                if anti:
                    bin_ = proj(bin_)
                for i, l in enumerate(locs):
                    rhs = l.A @ cin[i] + kappa * dt * bin_[i]
                    new.append(sla.lu_solve(lu_ie[i], rhs))
                raw = new
                if inst.normalize:
                    s = math.sqrt(pou_norm2(locs, new))
                    new = [c / s for c in new]
            n_done = n + 1
            hist_raw.append(new if tdse else raw)
            if step_energies and k == 1:
                result.__dict__.setdefault("step_energy", []).append(energy(locs, new))
            diff = [a - b for a, b in zip(new, coeffs)]
            coeffs = new
            hist.append(coeffs)
            if fixed == 0 and not tdse:
                q = math.sqrt(max(0.0, pou_norm2(locs, diff)))
                stop_q[n_done] = q
                stop_q.pop(n_done - 2, None)
                if q <= inst.ngf_tol:
                    break
        # traces of this iteration for all steps 0..n_done
        u_hist = [np.array([locs[i].own_vals @ h[i] for h in hist]) for i in range(S)]
        # Robin data for the next iteration: the transmission condition on
        # (t_n, t_{n+1}) sees the neighbour before the normalisation at t_{n+1}
        # (system SIT of Sec. 5.2), i.e. the un-normalised iterate.
        g_hist_steps = [ops.robin_data(h) for h in hist_raw]
        g_hist = [np.array([g_hist_steps[n][i] for n in range(len(hist))]) for i in range(S)]
        # residual against the previous iteration (hold-last beyond a window)
        res = schwarz_residual(locs, dt, u_hist, u_prev)
        rec = IterRecord(k=k, res=res, n_win=n_done, cvtot=interface_mismatch(locs, ops, hist, dt),
                         stop_values=dict(stop_q) if stop_q else None)
        if tdse:
            rec.norm2 = pou_norm2(locs, coeffs)
            rec.dipole = float(np.real(sum(np.vdot(c, l.Qchi @ c) for l, c in zip(locs, coeffs)))) / rec.norm2
        else:
            rec.energy = energy(locs, coeffs)
        result.records.append(rec)
        result.coeffs = coeffs
        result.own_traces = u_hist
        result.robin = g_hist
        if keep_all:
            result.__dict__.setdefault("all_coeffs", []).append(coeffs)
        u_prev = u_hist
        g_prev = g_hist
        n_prev = n_done
        if res <= tol and k >= k_min:
            result.converged = True
            break
    return result


# ---------------------------------------------------- single-domain helpers

def generalized_eigs(loc: Local, kinetic_only_h=False):
    """Eigenvalues of H~ c = lambda A c for one subdomain (brute force check)."""
    return sla.eigh(np.real(loc.Ht), loc.A, eigvals_only=True)
