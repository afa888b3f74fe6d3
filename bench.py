"""Benchmark of the SWR-Galerkin sweep on GB300.

One step = the whole hot path on the 2-electron ground-state workload
([-12,12]^2, 4x4 subdomains, 24x24 Gaussians each): swr_assemble (quadrature,
local Galerkin systems, orthonormalisation, step-matrix inverses, projection
of phi0) followed by swr_iterate until the interface residual Res(k) <= 1e-8.
Metric: local subdomain solves per second (one solve = one time step of one
subdomain), with the time-to-residual reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Under torchrun every rank solves its own replica of the workload on its own
GPU (independent problems, no data-path collective; weak scaling); the time
is the max over ranks.  `--impl reference` times the FP64 CPU oracle on the
host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

TOL = 1e-8
KMAX = 200
METRIC = "SWR time-to-1e-8 interface residual; subdomain solves/s vs plain FP64 GPU path"
# FP64 and FP32 (non-tensor) FMA rates of one GB300, measured on this machine with
# independent FMA chains over all SMs (the ceilings of the window kernel)
FP64_PEAK_TFLOPS = 1.01
FP32_PEAK_TFLOPS = 67.7
# DRAM bytes per launch of the window kernels from one ncu capture (profiles/), valid
# only while the kernel source is the one that was profiled (sha256 prefix of swr_window.cu)
PROFILED_TRAFFIC = {
    "k_window_df32": ("9feb1703488c26c7", 327.6e6, "profiles/k_window_df32_tise_2e_16sd.md"),
    "k_window_fp64": ("9feb1703488c26c7", 280.5e6, "profiles/k_window_fp64_tise_2e_16sd.md"),
}


def profiled_traffic(kernel):
    import hashlib
    src = os.path.join(ROOT, "paper_1710_02401_gb300", "csrc", "swr_window.cu")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    rec = PROFILED_TRAFFIC.get(kernel)
    if rec is None or rec[0] != h:
        return None, None
    return rec[1], rec[2]


def workload(name: str):
    from paper_1710_02401_gb300 import problems as P
    if name == "tise_2e_16sd":
        return P.tise_2e_16_subdomains()
    if name == "tise_1d_2sd":
        return P.tise_1d_two_subdomains()
    if name == "tdse_2e_64sd":
        return P.tdse_2e_64_subdomains()
    raise SystemExit(f"unknown workload {name}")


def workload_config(name: str, inst) -> dict:
    return {"workload": name, "n_elec": inst.n_elec, "box": list(inst.box), "L": inst.L,
            "subdomains": inst.n_sub, "K_d": inst.K_d, "K": inst.K_d ** inst.n_elec,
            "nodes_per_coord": (inst.n_mid + 2) * inst.q_p, "dt": inst.dt, "mu": str(inst.mu),
            "tol": TOL, "kmax": KMAX, "l2": "flushed (256 MB write) before every step",
            "parallelism": "replicas (one independent problem per GPU)"}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def oracle_sample(inst, gpu_solves_per_iter=None):
    """Times the FP64 CPU oracle on this host: assembly of all local systems,
    then the first Schwarz iteration (zero initial traces).  Returns
    (solves/s of the iteration, description, assembly seconds)."""
    from oracle import swr_oracle as O
    t0 = time.perf_counter()
    locs = O.assemble(inst)
    t_asm = time.perf_counter() - t0
    t1 = time.perf_counter()
    r = O.run_swr(inst, kmax=1, tol=0.0, locs=locs)
    t_it = time.perf_counter() - t1
    solves = r.records[0].n_win * inst.n_sub
    desc = (f"oracle (numpy FP64, dense quadrature + LU) on the same workload: first Schwarz "
            f"iteration, {solves} local step solves in {t_it:.2f} s; local assembly of all "
            f"{inst.n_sub} subdomains took {t_asm:.2f} s and is not in the rate")
    return solves / t_it, desc, t_asm


def run_reference(args, inst, name):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import swr_oracle as O
    locs = O.assemble(inst)
    for _ in range(args.warmup):
        O.run_swr(inst, kmax=1, tol=0.0, locs=locs)
    t_tot, solves = 0.0, 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = O.run_swr(inst, kmax=1, tol=0.0, locs=locs)
        t_tot += time.perf_counter() - t0
        solves += r.records[0].n_win * inst.n_sub
    value = solves / t_tot
    cores = os.cpu_count()
    sample = ("each step: first Schwarz iteration (zero initial traces) of the FP64 oracle on the "
              "full workload, local systems assembled once before the timed steps")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "subdomain solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(name, inst),
        "cpu_baseline": {"value": value, "unit": "subdomain solves/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "subdomain solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="tise_2e_16sd")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                    help="precision of the headline line; the other path is timed beside it")
    ap.add_argument("--no-compare", action="store_true", help="skip the timing of the other precision")
    ap.add_argument("--iterations", type=int, default=0,
                    help="fixed Schwarz iterations per step instead of iterating to Res <= 1e-8 "
                         "(for the long real-time workload)")
    args = ap.parse_args()
    name = args.workload
    inst = workload(name)
    if args.impl == "reference":
        run_reference(args, inst, name)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1710_02401_gb300 import build as B
    B.build()
    from paper_1710_02401_gb300 import swr as S

    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    prec_of = {"mixed": S.PREC_MIXED, "fp64": S.PREC_FP64}

    def timed(prec_name, steps, warmup, sample_clocks):
        """W untimed + K timed steps (assemble + iterate to Res <= TOL), CUDA
        events on the library's stream, L2 flushed before every step."""
        s = S.SWR(inst, precision=prec_of[prec_name], device=str(dev), stream=stream)
        for _ in range(warmup):
            s.assemble()
            s.iterate(TOL if not args.iterations else 0.0, args.iterations or KMAX)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        sampler = ClockSampler(local) if sample_clocks else None
        if sampler:
            sampler.start()
        c0 = s.counters()
        times, reps = [], []
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.assemble()
            rep, hist = s.iterate(TOL if not args.iterations else 0.0, args.iterations or KMAX)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            reps.append(rep)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        c1 = s.counters()
        clocks = sampler.stop() if sampler else None
        t_ms = sum(times)
        solves = sum(r.subdomain_solves for r in reps)
        t_max, solves_all = t_ms, solves
        if world > 1:
            t = torch.tensor([t_ms], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            t_max = float(t.item())
            n = torch.tensor([solves], dtype=torch.float64, device=dev)
            dist.all_reduce(n, op=dist.ReduceOp.SUM)
            solves_all = int(n.item())
        d = {k: c1[k] - c0[k] for k in c1}
        return dict(s=s, value=solves_all / (t_max * 1e-3), t_max=t_max, reps=reps, counters=d, clocks=clocks,
                    plan=s.window_plan())

    main_run = timed(args.precision, args.steps, args.warmup, True)
    other = None
    if not args.no_compare:
        other_name = "fp64" if args.precision == "mixed" else "mixed"
        other = timed(other_name, max(1, min(args.steps, 2)), 1, False)
        other["name"] = other_name
    s = main_run["s"]
    reps = main_run["reps"]
    cnt = main_run["counters"]
    w_ms, w_launch, w_flops = cnt["window_ms"], cnt["window_launches"], cnt["window_flops"]
    # dominant kernel: the persistent time-window kernel
    achieved = w_flops / (w_ms * 1e-3) / 1e12 if w_ms > 0 else 0.0
    if inst.mode == "tdse" and args.precision == "mixed":
        gbs = cnt["window_bytes"] / (w_ms * 1e-3) / 1e9 if w_ms > 0 else 0.0
        hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] \
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
        roof = {"kernel": "k_cmv_df32 + Crank-Nicolson element-wise kernels", "bound": "hbm", "achieved": gbs,
                "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)",
                "algorithmic": "16 bytes of G0 (four FP32 planes) per complex matrix element and sweep, "
                               "(1 + m) sweeps per Crank-Nicolson step; G0 (1.07 GB) does not fit in L2"}
    elif inst.mode == "tdse":
        roof = {"kernel": "k_cmv + Crank-Nicolson element-wise kernels", "bound": "alu", "achieved": achieved,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "peak_source": "FP64 FMA rate measured on this pool's GB300 (probe of independent FMA chains)",
                "algorithmic": "8 K^2 flops per complex matvec with G0, (1 + m) matvecs per Crank-Nicolson step"}
    elif args.precision == "mixed":
        # double-single matvec: ~12 FP32 operations per matrix element on the FP32 pipes
        peak = FP32_PEAK_TFLOPS / 6.0
        kname = "k_window_fused" if main_run["plan"]["variant"] == S.WINDOW_FUSED else "k_window_2ph<true>"
        roof = {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": "measured FP32 FMA rate of this pool's GB300 (67.7 TFLOP/s) / 6: the "
                               "double-single product-sum spends 12 FP32 operations per 2 FP64-equivalent flops",
                "algorithmic": "2 K^2 FP64-equivalent flops per local step solve (matvec with the step-matrix inverse)"}
    else:
        roof = {"kernel": "k_window_2ph<false>", "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "peak_source": "FP64 FMA rate measured on this pool's GB300 (probe of independent FMA chains)",
                "algorithmic": "2 K^2 flops per local step solve (FP64 matvec with the step-matrix inverse)"}
    traffic, src = profiled_traffic(roof["kernel"])
    roof["traffic"] = traffic
    roof["traffic_source"] = src
    roof["window_ms_per_launch"] = w_ms / max(w_launch, 1)
    roof["step_us"] = 1e3 * w_ms / max(1.0, cnt["solves"] / inst.n_sub)
    launches = int(cnt["kernel_launches"])

    # end to end through the public API: setup from host descriptors, assembly,
    # iterations, read-back of energies and psi at all nodes, teardown
    e2e_val, h2d, d2h = None, 0, 0
    if args.e2e_steps > 0:
        e_solves, e_time = 0, 0.0
        for _ in range(args.e2e_steps):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            se = S.SWR(inst, precision=prec_of[args.precision], device=str(dev), stream=stream)
            se.assemble()
            rep_e, _ = se.iterate(TOL if not args.iterations else 0.0, args.iterations or KMAX)
            energy = se.energy()
            psi = se.psi_nodes()
            ce = se.counters()
            se.close()
            torch.cuda.synchronize(dev)
            e_time += time.perf_counter() - t0
            e_solves += rep_e.subdomain_solves
            h2d, d2h = int(ce["h2d_bytes"]), int(ce["d2h_bytes"])
            del se
        e2e_val = e_solves / e_time

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, desc, t_asm = oracle_sample(inst)
        cpu = {"value": v, "unit": "subdomain solves/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": desc}
    out = {
        "metric": METRIC, "value": main_run["value"], "unit": "subdomain solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": main_run["t_max"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32x2 (double-single) step matrices, f64 reductions" if args.precision == "mixed" else "f64",
        "data": "synthetic", "config": workload_config(name, inst),
        "precision": args.precision,
        "time_to_residual_s": main_run["t_max"] / args.steps * 1e-3,
        "schwarz_iterations": [r.iterations for r in reps], "converged": all(r.converged for r in reps),
        "res_last": [r.res_last for r in reps],
        "energy": float(s.energy()[0]),
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": "subdomain solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": main_run["clocks"],
    }
    if other is not None:
        o_reps = other["reps"]
        out["other_precision"] = {
            "precision": other["name"], "value": other["value"],
            "time_to_residual_s": other["t_max"] / len(o_reps) * 1e-3,
            "schwarz_iterations": [r.iterations for r in o_reps],
            "energy": float(other["s"].energy()[0]),
            "speedup_of_headline": main_run["value"] / other["value"],
        }
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
