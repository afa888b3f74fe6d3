"""Writes the stored expected values of the full-size parity tests.

Calls only the FP64 CPU oracle (oracle/swr_oracle.py) and the seeded problem
definitions (paper_1710_02401_gb300/problems.py); no value here comes from
the CUDA path.  Run from the repository root:

    python tests/golden/make_golden.py [case ...]

Cases (one .npz each, beside this script):
  tise_2e_16sd_k3     the 2-electron ground-state workload at full size
                      (4 x 4 subdomains, 24 x 24 Gaussians, K = 576), first
                      three Schwarz iterations
  tdse_2e_k1024_4sd   the real-time workload's subdomain shape (32 x 32 complex
                      Gaussians, K = 1024, width 5.5, the same quadrature and
                      pulse) on a 2 x 2 decomposition of [-5, 5]^2, 20
                      Crank-Nicolson steps, two Schwarz iterations
  batched_k1024       instances 95, 209 (2 electrons, subdomains up to
                      K = 1024) and 262 (1 electron, 4 subdomains) of the
                      seeded 512-instance uneven batch, two Schwarz iterations

Stored per Schwarz iteration: window length, Res(k), CVTOT(k), energy (or
norm^2 and dipole in real time), and in imaginary time the NGF stop
quantity ||c^n - c^(n-1)|| of the window's last two steps (stop_prev,
stop_last).  For the last iteration: the own traces u_i and the Robin data
g_i at every interface node of the steps listed in `steps`, plus `n_samples` seeded (subdomain, step, node) samples over the
whole window; psi at every `psi_stride`-th volume node.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import swr_oracle as O  # noqa: E402
from paper_1710_02401_gb300 import problems as P  # noqa: E402


def case_instances(name):
    """(instances, Schwarz iterations) of a stored case."""
    if name == "tise_2e_16sd_k3":
        return [P.tise_2e_16_subdomains()], 3
    if name == "tdse_2e_k1024_4sd":
        full = P.tdse_2e_64_subdomains(n_steps=20)
        box, L = (-5.0, 5.0), 2  # the same subdomain width (b - a)/L + eps = 5.5 as on 8 x 8 of [-20, 20]
        return [full.replace(box=box, L=L, delta=P.spacing_rule_delta(box, L, full.overlap, full.K_d),
                             n_mid=P.mid_panels(box, L, full.overlap))], 2
    if name == "batched_k1024":
        b = P.batched_uneven(512)
        return [b[95], b[209], b[262]], 2
    raise KeyError(name)


PSI_STRIDE = 7
N_SAMPLES = 4000


def steps_of(W):
    return sorted({0, 1, 2, W // 3, W // 2, max(W - 1, 0), W})


def run_case(name):
    insts, kmax = case_instances(name)
    out = {}
    rng = np.random.default_rng(20250101)
    for ii, inst in enumerate(insts):
        t0 = time.time()
        r = O.run_swr(inst, kmax=kmax, tol=0.0)
        p = f"i{ii}_"
        out[p + "win"] = np.array([rec.n_win for rec in r.records], dtype=np.int64)
        out[p + "res"] = np.array([rec.res for rec in r.records])
        out[p + "cvtot"] = np.array([rec.cvtot for rec in r.records])
        if r.records[0].stop_values:
            out[p + "stop_prev"] = np.array([rec.stop_values[rec.n_win - 1] for rec in r.records])
            out[p + "stop_last"] = np.array([rec.stop_values[rec.n_win] for rec in r.records])
        if inst.mode == P.TDSE:
            out[p + "norm2"] = np.array([rec.norm2 for rec in r.records])
            out[p + "dipole"] = np.array([rec.dipole for rec in r.records])
        else:
            out[p + "energy"] = np.array([rec.energy for rec in r.records])
        W = r.records[-1].n_win
        st = np.array(steps_of(W), dtype=np.int64)
        out[p + "steps"] = st
        for i in range(inst.n_sub):
            u, g = r.own_traces[i], r.robin[i]
            out[p + f"u{i}"] = u[st]
            out[p + f"g{i}"] = g[st]
            psi = O.psi_at_nodes(r.locs[i], r.coeffs[i])
            out[p + f"psi{i}"] = psi[::PSI_STRIDE]
        # seeded samples over the whole window: (subdomain, step, node, u, g)
        subs = [i for i in range(inst.n_sub) if r.own_traces[i].shape[1] > 0]
        smp = []
        for _ in range(N_SAMPLES):
            i = int(rng.choice(subs))
            n = int(rng.integers(0, W + 1))
            k = int(rng.integers(0, r.own_traces[i].shape[1]))
            smp.append((i, n, k))
        smp = np.array(smp, dtype=np.int64)
        out[p + "smp_idx"] = smp
        out[p + "smp_u"] = np.array([r.own_traces[i][n, k] for i, n, k in smp])
        out[p + "smp_g"] = np.array([r.robin[i][n, k] for i, n, k in smp])
        print(f"{name} instance {ii}: windows {out[p + 'win'].tolist()} res {out[p + 'res'].tolist()} "
              f"({time.time() - t0:.1f} s)", flush=True)
    out["n_inst"] = np.array(len(insts))
    out["psi_stride"] = np.array(PSI_STRIDE)
    np.savez_compressed(os.path.join(HERE, name + ".npz"), **out)


if __name__ == "__main__":
    names = sys.argv[1:] or ["tise_2e_16sd_k3", "tdse_2e_k1024_4sd", "batched_k1024"]
    for nm in names:
        run_case(nm)
