"""Learned initial interface traces.

The paper starts every SWR solve from zero Robin data, g^(0) = 0.  Here a
small BF16 perceptron maps a descriptor of each subdomain (its box, the
nuclei, the softening, the field phase) to the code of its converged Robin
data (swr_trace_codec: orthonormal polynomials along each edge times in the
step index), and the solve starts from the decoded prediction.  Training data
come from the SWR solver itself, on the GPU; training runs on the GPU with
the library's own forward/backward/Adam kernels.  The zero-guess solve stays
the fallback and decides the prediction's error: the residual that decides
convergence is the same Res(k) of the plain method.

Every numerical step runs in libswr.so; this module only arranges the data
(descriptors, the affine output standardisation folded into the last layer).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Sequence

import numpy as np

from . import problems as P
from . import swr as S

CODE_S, CODE_T = 8, 16
N_FEATURES = 16


def descriptors(instances: Sequence[P.Instance]) -> np.ndarray:
    """One row per subdomain, subdomains in solver order."""
    rows = []
    for inst in instances:
        a, b = inst.box
        H = (b - a) / inst.L
        scale = max(abs(a), abs(b))
        nuc = list(inst.nuclei) + [(0.0, 0.0)] * (3 - len(inst.nuclei))
        E0, T, om, ph = inst.field
        for sid in range(inst.n_sub):
            i1, i2 = sid % inst.L, sid // inst.L
            lo1, hi1 = a + i1 * H - inst.overlap / 2, a + (i1 + 1) * H + inst.overlap / 2
            lo2, hi2 = a + i2 * H - inst.overlap / 2, a + (i2 + 1) * H + inst.overlap / 2
            f = [lo1 / scale, hi1 / scale, lo2 / scale, hi2 / scale]
            for (x, z) in nuc:
                f += [x / 2.0, z / 2.0]
            f += [inst.eta_en, inst.eta_ee, math.sin(ph), math.cos(ph), E0, 1.0]
            rows.append(f)
    return np.asarray(rows, dtype=np.float32)


def solve(instances, tol: float, kmax: int, init_codes=None):
    """Runs one batched SWR solve; returns (context, per-instance iteration
    counts to Res <= tol (kmax + 1 when not reached), residual history)."""
    s = S.SWR(list(instances))
    s.assemble()
    s.trace_codec(CODE_S, CODE_T)
    if init_codes is not None:
        s.trace_decode_set(init_codes)
    n = len(instances)
    done = np.full(n, kmax + 1)
    hist = []
    for k in range(1, kmax + 1):
        s.step()
        r = s.residual()
        hist.append(r.copy())
        newly = (r <= tol) & (done > kmax)
        done[newly] = k
        if np.all(done <= kmax):
            break
    return s, done, np.array(hist)


@dataclass
class Model:
    mlp: S.MLP
    dims: List[int]


def init_params(dims: Sequence[int], seed: int) -> np.ndarray:
    """Seeded Glorot-uniform initial weights, zero biases (drawn here and
    passed to the kernels as input)."""
    rng = np.random.default_rng(seed)
    out = []
    for l in range(len(dims) - 1):
        lim = math.sqrt(6.0 / (dims[l] + dims[l + 1]))
        out.append(rng.uniform(-lim, lim, size=dims[l] * dims[l + 1]))
        out.append(np.zeros(dims[l + 1]))
    return np.concatenate(out).astype(np.float32)


def fold_output_affine(params: np.ndarray, dims: Sequence[int], mean: np.ndarray, std: np.ndarray) -> np.ndarray:
    """Last layer of a model trained on standardised targets -> raw targets."""
    p = params.astype(np.float64).copy()
    o = sum(dims[l] * dims[l + 1] + dims[l + 1] for l in range(len(dims) - 2))
    din, dout = dims[-2], dims[-1]
    W = p[o:o + din * dout].reshape(din, dout)
    b = p[o + din * dout:o + din * dout + dout]
    p[o:o + din * dout] = (W * std[None, :]).ravel()
    p[o + din * dout:o + din * dout + dout] = b * std + mean
    return p.astype(np.float32)


def train(x: np.ndarray, y: np.ndarray, width: int = 256, n_hidden: int = 3, steps: int = 1500,
          lr: float = 1e-3, seed: int = 0, log=None):
    """Trains on standardised targets with full-batch Adam on the GPU kernels;
    returns the model with the standardisation folded into its last layer."""
    import torch
    mean = y.mean(axis=0)
    std = y.std(axis=0) + 1e-6
    yz = (y - mean) / std
    dims = [x.shape[1]] + [width] * n_hidden + [y.shape[1]]
    mlp = S.MLP(x.shape[1], width, n_hidden, y.shape[1])
    mlp.set_params(init_params(dims, seed))
    xd = torch.as_tensor(x, dtype=torch.float32, device="cuda")
    yd = torch.as_tensor(yz, dtype=torch.float32, device="cuda")
    losses = []
    for it in range(steps):
        cur = lr * (0.1 ** (it / steps))
        loss, _ = mlp.train_step(xd, yd, cur)
        losses.append(loss)
        if log and it % 250 == 0:
            log(f"step {it} loss {loss:.4e}")
    mlp.set_params(fold_output_affine(mlp.get_params(), dims, mean, std))
    return Model(mlp, dims), losses


def gather_training_set(instances, tol=1e-8, kmax=60):
    """Converged trace codes (GPU solve + encode) and descriptors."""
    s, done, _ = solve(instances, tol, kmax)
    codes = s.trace_encode().cpu().numpy()
    return descriptors(instances), codes, done


def predict_codes(model: Model, instances):
    import torch
    x = torch.as_tensor(descriptors(instances), dtype=torch.float32, device="cuda")
    return model.mlp.forward(x)


def compare(model: Model, instances, tol=1e-8, kmax=60):
    """Iterations to Res <= tol from zero traces and from the learned guess."""
    _, zero, _ = solve(instances, tol, kmax)
    _, learned, _ = solve(instances, tol, kmax, init_codes=predict_codes(model, instances))
    return zero, learned


def compare_timed(model: Model, instances, tol=1e-8, kmax=60, repeats=3):
    """Wall time of the batched solve to Res <= tol of every instance, from
    zero traces and from the learned guess (descriptor upload, MLP inference
    and decoding of the codes into Robin data and sources included), best of
    `repeats`; setup and assembly of the context are inside both timings."""
    import time
    import torch

    def timed(learned: bool):
        best, out = float("inf"), None
        for _ in range(repeats):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s = S.SWR(list(instances))
            s.assemble()
            s.trace_codec(CODE_S, CODE_T)
            t_inf = 0.0
            if learned:
                ti = time.perf_counter()
                s.trace_decode_set(predict_codes(model, instances))
                torch.cuda.synchronize()
                t_inf = time.perf_counter() - ti
            n = len(instances)
            done = np.full(n, kmax + 1)
            for k in range(1, kmax + 1):
                s.step()
                r = s.residual()
                done[(r <= tol) & (done > kmax)] = k
                if np.all(done <= kmax):
                    break
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            s.close()
            if dt < best:
                best, out = dt, (done, t_inf)
        return best, out[0], out[1]

    t_zero, it_zero, _ = timed(False)
    t_learned, it_learned, t_inf = timed(True)
    return {"seconds_zero_guess": t_zero, "seconds_learned": t_learned, "seconds_inference_decode": t_inf,
            "iterations_zero_guess": float(np.mean(it_zero)), "iterations_learned": float(np.mean(it_learned)),
            "batch_iterations_zero_guess": int(np.max(it_zero)), "batch_iterations_learned": int(np.max(it_learned))}
