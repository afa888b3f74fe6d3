"""Seeded, synthetic problem definitions for the SWR-Galerkin sweep.

This module holds input descriptions only: geometry, basis sizes, physical
parameters and time-stepping settings of each workload, plus the seeded
generator of the batched uneven workload.  It performs none of the method's
arithmetic (no quadrature, no matrices, no solves), so both the CPU oracle and
the CUDA path can take their inputs from here without sharing any numerics.

Parameter meaning follows the paper's statement of the problem:
  * Hamiltonian H0 with P fixed nuclei (Sec. 1.1) and the length-gauge dipole
    term x.E(t) (Sec. 1.2, Eq. LG);
  * soft-Coulomb regularised potentials -Z/sqrt((x-x_A)^2+eta^2)
    (Sec. 6.3, Eq. pseudo), used here for electron-nucleus and
    electron-electron terms;
  * global box [a,b]^N cut into L^N overlapping hypercubes with overlap
    bands of width eps (opening of Sec. 6);
  * 1-D Gaussian primitives exp(-delta (x-alpha)^2) with evenly spaced centres
    (Sec. 2, Eq. gauss1d; Sec. 6.1);
  * Robin constant mu (Sec. 5.1, Eq. RTC);
  * implicit Euler + normalisation for the imaginary-time problem and
    Crank-Nicolson for the real-time one (Sec. 5.4, step 2).
"""
from __future__ import annotations

import dataclasses
import math
import random
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple, Union

TISE = "tise"
TDSE = "tdse"


@dataclass
class Instance:
    """One SWR problem (one global box, L^N subdomains)."""

    n_elec: int = 1                      # N (d = 1): 1 or 2
    box: Tuple[float, float] = (-10.0, 10.0)  # [a, b] in every coordinate
    L: int = 2                           # subdomains per coordinate
    overlap: float = 1.0                 # eps: width of each overlap band
    K_d: Union[int, Sequence[int]] = 40  # Gaussians per coordinate (int or per subdomain)
    delta: Union[float, Sequence[float]] = 4.0  # Gaussian exponent (scalar or per subdomain)
    q_p: int = 14                        # Gauss-Legendre nodes per panel
    n_mid: int = 9                       # equal panels of the non-overlapped middle zone
    nuclei: Tuple[Tuple[float, float], ...] = ((0.0, 1.0),)  # (x_A, Z_A)
    eta_en: float = 1.0                  # electron-nucleus softening
    eta_ee: float = 0.5                  # electron-electron softening
    ee_coef: float = 1.0                 # prefactor of the e-e repulsion (0 disables it)
    harmonic: float = 0.0                # adds harmonic * x^2 / 2 per electron
    kinetic: float = 0.5                 # kappa in -kappa*Laplacian (1/2: Schroedinger, 1: heat equation)
    mu: complex = 10.0                   # Robin constant (real > 0 imaginary time; i*R_- real time)
    mode: str = TISE                     # "tise" (implicit Euler NGF) or "tdse" (Crank-Nicolson)
    normalize: bool = True               # TISE: renormalise after every step
    dt: float = 0.1
    n_steps: int = 0                     # fixed window length (TDSE, or TISE with ngf_tol <= 0)
    ngf_tol: float = 1e-12               # TISE inner stop on ||phi^{n+1}-phi^n||
    max_steps: int = 5000                # TISE window cap
    field: Tuple[float, float, float, float] = (0.0, 1.0, 0.0, 0.0)  # (E0, T, omega, phase)
    phi0_gamma: float = 1.0              # phi0 = exp(-gamma |x - x0|^2)
    phi0_center: Tuple[float, float] = (0.0, 0.0)
    orth_tau: float = 1e-12              # per-coordinate overlap: Cholesky if every pivot >= tau * max diagonal,
                                         # else canonical (eigenvectors with lambda > tau * lambda_max)
    tc: str = "robin"                    # transmission condition: "robin" (Eq. RTC) or "dirichlet"
                                         # (classical SWR, imposed by penalty with constant mu)
    symmetry: str = "none"               # "antisymmetric": N = 2 imaginary time restricted to states with
                                         # psi(x2, x1) = -psi(x1, x2) (Appendix A, mirror subdomains)

    @property
    def n_sub(self) -> int:
        return self.L ** self.n_elec

    def k_d_of(self, sid: int) -> int:
        if isinstance(self.K_d, int):
            return self.K_d
        return int(self.K_d[sid])

    def delta_of(self, sid: int) -> float:
        if isinstance(self.delta, (int, float)):
            return float(self.delta)
        return float(self.delta[sid])

    def window(self) -> int:
        """Number of time steps of a fixed window, 0 when the TISE stop decides."""
        if self.mode == TDSE:
            return self.n_steps
        return self.n_steps if self.ngf_tol <= 0 else 0

    def replace(self, **kw) -> "Instance":
        return dataclasses.replace(self, **kw)


def mid_panels(box: Tuple[float, float], L: int, overlap: float) -> int:
    """Number of equal panels for the middle zone [lo+eps, hi-eps] of a
    subdomain coordinate so that they are about as long as an overlap band."""
    H = (box[1] - box[0]) / L
    return max(1, int(round((H - overlap) / overlap)))


def spacing_rule_delta(box: Tuple[float, float], L: int, overlap: float, k_d: int) -> float:
    """Exponent for which the Gaussian width equals the centre spacing h.

    The workloads without a stated width take delta = 1/(2 h^2), h the spacing
    of K_d evenly spaced centres on a subdomain interval of length
    (b - a)/L + eps.  This is an input choice, recorded with each workload.
    """
    h = ((box[1] - box[0]) / L + overlap) / (k_d - 1)
    return 1.0 / (2.0 * h * h)


# ---------------------------------------------------------------- workloads

def tise_1d_two_subdomains(q_p: int = 14) -> Instance:
    """1 electron in 1-D, [-10,10], 2 subdomains with overlap 1.0, 40 Gaussians
    of width 0.5 (read as exp(-((x-alpha)/0.5)^2), delta = 4), soft-Coulomb
    -1/sqrt(x^2+1), Robin mu = 10, implicit Euler dt = 0.1."""
    return Instance(n_elec=1, box=(-10.0, 10.0), L=2, overlap=1.0, K_d=40, delta=4.0,
                    q_p=q_p, n_mid=9, nuclei=((0.0, 1.0),), eta_en=1.0, ee_coef=0.0,
                    mu=10.0, mode=TISE, dt=0.1, ngf_tol=1e-12, max_steps=5000,
                    phi0_gamma=1.0)


def harmonic_1d_two_subdomains(q_p: int = 14) -> Instance:
    """Same geometry and basis with V = x^2/2 (ground energy 1/2)."""
    return tise_1d_two_subdomains(q_p).replace(nuclei=(), harmonic=1.0)


def tise_2e_16_subdomains(q_p: int = 12) -> Instance:
    """2 electrons in 1-D, [-12,12]^2 in 4x4 subdomains, 24x24 Gaussians each,
    nuclei Z=1 at +-0.7, soft e-n and e-e with eps = 0.5, overlap 10% of the
    core width (0.6), delta by the spacing rule, mu = 10, dt = 0.1."""
    box, L, ov, kd = (-12.0, 12.0), 4, 0.6, 24
    return Instance(n_elec=2, box=box, L=L, overlap=ov, K_d=kd,
                    delta=spacing_rule_delta(box, L, ov, kd), q_p=q_p,
                    n_mid=mid_panels(box, L, ov),
                    nuclei=((-0.7, 1.0), (0.7, 1.0)), eta_en=0.5, eta_ee=0.5,
                    ee_coef=1.0, mu=10.0, mode=TISE, dt=0.1, ngf_tol=1e-12,
                    max_steps=5000, phi0_gamma=1.0)


def tdse_2e_64_subdomains(q_p: int = 14, n_steps: int = 1000) -> Instance:
    """2 electrons in 1-D, [-20,20]^2 in 8x8 subdomains, 32x32 Gaussians each,
    Crank-Nicolson dt = 0.01 for 1000 steps, mu = -10i, dipole field
    E(t) = 0.05 sin^2(pi t/10) sin(0.057 t), same molecule as the 16-subdomain
    ground-state workload, overlap 10% of the core width (0.5)."""
    box, L, ov, kd = (-20.0, 20.0), 8, 0.5, 32
    return Instance(n_elec=2, box=box, L=L, overlap=ov, K_d=kd,
                    delta=spacing_rule_delta(box, L, ov, kd), q_p=q_p,
                    n_mid=mid_panels(box, L, ov),
                    nuclei=((-0.7, 1.0), (0.7, 1.0)), eta_en=0.5, eta_ee=0.5,
                    ee_coef=1.0, mu=-10j, mode=TDSE, dt=0.01, n_steps=n_steps,
                    field=(0.05, 10.0, 0.057, 0.0), phi0_gamma=1.0)


def batched_uneven(n_instances: int = 512, seed: int = 171002401,
                   k_lo: int = 64, k_hi: int = 1024) -> List[Instance]:
    """Seeded batch of independent ground-state problems with uneven bases.

    Per instance: N in {1,2} (50/50); 1 or 2 nuclei at U[-2,2] with Z in
    {1,2,3}; softening eps ~ U[0.3,1] (e-n and e-e); box [-12,12]^N;
    N=1: L ~ U{4..64}; N=2: L ~ U{2..8}; overlap 10% of the core width;
    per-subdomain basis size K ~ U[k_lo, k_hi] drawn for every subdomain and
    read as K_d = round(sqrt(K)) Gaussians per coordinate for both N (so the
    draw sets the per-coordinate resolution; N=2 subdomains have K = K_d^2,
    N=1 subdomains K = K_d: a 1-D basis of up to 1024 Gaussians on an
    interval of width 0.4-6.6 would be 30-100x finer than the 1-electron
    workload's 40 Gaussians on width 10.5); delta by the spacing rule per subdomain; quadrature
    panels as long as the overlap band with q_p nodes each, q_p chosen so every panel resolves the narrowest Gaussian (about 3.4 nodes per
    Gaussian of the finest subdomain); implicit Euler
    NGF dt = 0.1, mu = 10.
    """
    rng = random.Random(seed)
    out = []
    box = (-12.0, 12.0)
    for _ in range(n_instances):
        n = 1 if rng.random() < 0.5 else 2
        P = rng.choice((1, 2))
        nuc = tuple((rng.uniform(-2.0, 2.0), float(rng.choice((1, 2, 3)))) for _ in range(P))
        eps = rng.uniform(0.3, 1.0)
        L = rng.randint(4, 64) if n == 1 else rng.randint(2, 8)
        ov = 0.1 * (box[1] - box[0]) / L
        kds, deltas = [], []
        for _s in range(L ** n):
            K = rng.randint(k_lo, k_hi)
            kd = max(2, int(round(math.sqrt(K))))
            kds.append(kd)
            deltas.append(spacing_rule_delta(box, L, ov, kd))
        kmax = max(kds)
        n_mid = mid_panels(box, L, ov)
        # about 3.4 nodes per Gaussian of the finest subdomain, at least 8 per panel
        q_p = max(8, int(math.ceil(3.4 * kmax / (n_mid + 2))))
        out.append(Instance(n_elec=n, box=box, L=L, overlap=ov, K_d=kds, delta=deltas,
                            q_p=q_p, n_mid=n_mid, nuclei=nuc, eta_en=eps, eta_ee=eps, ee_coef=1.0,
                            mu=10.0, mode=TISE, dt=0.1, ngf_tol=1e-12, max_steps=5000,
                            phi0_gamma=1.0))
    return out


def small_tise_2d(L: int = 3, K_d: int = 10, q_p: int = 8, n_mid: int = 3, **kw) -> Instance:
    """Parity-sized 2-electron ground-state problem (several tiles, ragged tail)."""
    box, ov = (-6.0, 6.0), 0.4
    base = Instance(n_elec=2, box=box, L=L, overlap=ov, K_d=K_d,
                    delta=spacing_rule_delta(box, L, ov, K_d), q_p=q_p, n_mid=n_mid,
                    nuclei=((-0.7, 1.0), (0.7, 1.0)), eta_en=0.5, eta_ee=0.5,
                    ee_coef=1.0, mu=10.0, mode=TISE, dt=0.1, ngf_tol=1e-12,
                    max_steps=3000, phi0_gamma=1.0)
    return base.replace(**kw) if kw else base


def small_tdse_2d(L: int = 3, K_d: int = 10, q_p: int = 8, n_mid: int = 3, n_steps: int = 40,
                  **kw) -> Instance:
    """Parity-sized 2-electron real-time problem under a dipole field."""
    box, ov = (-6.0, 6.0), 0.4
    base = Instance(n_elec=2, box=box, L=L, overlap=ov, K_d=K_d,
                    delta=spacing_rule_delta(box, L, ov, K_d), q_p=q_p, n_mid=n_mid,
                    nuclei=((-0.7, 1.0), (0.7, 1.0)), eta_en=0.5, eta_ee=0.5,
                    ee_coef=1.0, mu=-10j, mode=TDSE, dt=0.01, n_steps=n_steps,
                    field=(0.5, 0.4, 8.0, 0.3), phi0_gamma=1.0)
    return base.replace(**kw) if kw else base


PRESETS = {
    "tise_1d_2sd": tise_1d_two_subdomains,
    "harmonic_1d_2sd": harmonic_1d_two_subdomains,
    "tise_2e_16sd": tise_2e_16_subdomains,
    "tdse_2e_64sd": tdse_2e_64_subdomains,
}


def learned_trace_family(n_instances: int, seed: int = 5) -> List[Instance]:
    """Seeded real-time problems for the learned initial traces, on a reduced
    grid: 2 electrons, [-6,6]^2 in 2x2 subdomains, 8x8 Gaussians, 40
    Crank-Nicolson steps (dt = 0.01), mu = -10i, field
    0.5 sin^2(pi t/0.4) sin(8 t + phase) with phase ~ U[0, 2 pi); 1 or 2
    nuclei at U[-1.5, 1.5] with Z in {1, 2}; softening ~ U[0.3, 1]."""
    rng = random.Random(seed)
    box, L, ov, kd = (-6.0, 6.0), 2, 0.6, 8
    out = []
    for _ in range(n_instances):
        P = rng.choice((1, 2))
        nuc = tuple((rng.uniform(-1.5, 1.5), float(rng.choice((1, 2)))) for _ in range(P))
        eps = rng.uniform(0.3, 1.0)
        phase = rng.uniform(0.0, 2.0 * math.pi)
        out.append(Instance(n_elec=2, box=box, L=L, overlap=ov, K_d=kd,
                            delta=spacing_rule_delta(box, L, ov, kd), q_p=6, n_mid=mid_panels(box, L, ov),
                            nuclei=nuc, eta_en=eps, eta_ee=eps, ee_coef=1.0, mu=-10j, mode=TDSE,
                            dt=0.01, n_steps=40, field=(0.5, 0.4, 8.0, phase), phi0_gamma=1.0))
    return out



def learned_trace_family_16sd(n_instances: int, seed: int = 7) -> List[Instance]:
    """Seeded real-time problems for the learned initial traces with the
    64-subdomain real-time workload's subdomain geometry (cores of width 5,
    overlap 0.5) on a 4 x 4 grid: 2 electrons, [-10,10]^2, 10 x 10 Gaussians
    per subdomain, 100 Crank-Nicolson steps (dt = 0.01), mu = -10i, field
    0.5 sin^2(pi t) sin(8 t + phase) with phase ~ U[0, 2 pi); 1 or 2 nuclei
    at U[-2, 2] with Z in {1, 2, 3}; softening ~ U[0.3, 1]."""
    rng = random.Random(seed)
    box, L, ov, kd = (-10.0, 10.0), 4, 0.5, 10
    out = []
    for _ in range(n_instances):
        P = rng.choice((1, 2))
        nuc = tuple((rng.uniform(-2.0, 2.0), float(rng.choice((1, 2, 3)))) for _ in range(P))
        eps = rng.uniform(0.3, 1.0)
        phase = rng.uniform(0.0, 2.0 * math.pi)
        out.append(Instance(n_elec=2, box=box, L=L, overlap=ov, K_d=kd,
                            delta=spacing_rule_delta(box, L, ov, kd), q_p=8, n_mid=mid_panels(box, L, ov),
                            nuclei=nuc, eta_en=eps, eta_ee=eps, ee_coef=1.0, mu=-10j, mode=TDSE,
                            dt=0.01, n_steps=100, field=(0.5, 1.0, 8.0, phase), phi0_gamma=1.0))
    return out