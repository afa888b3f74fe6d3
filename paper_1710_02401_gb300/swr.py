"""ctypes binding of the SWR-Galerkin C ABI (include/swr.h).

Argument marshalling only: every step of the sweep runs in the CUDA kernels of
libswr.so.  PyTorch provides the device workspace (a caller-owned uint8
tensor handed to swr_setup) and the CUDA stream; nothing here computes any
part of the method.  The binding fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Iterable, List, Optional, Sequence

import numpy as np

from . import problems as P

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libswr.so")

SWR_OK, SWR_EINVAL, SWR_ENOMEM, SWR_ECUDA, SWR_ESINGULAR, SWR_ENUMERIC, SWR_ENOTCONV, SWR_ETIMEOUT, SWR_ESTATE = range(9)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ESINGULAR", "ENUMERIC", "ENOTCONV", "ETIMEOUT", "ESTATE"]
MODE_TISE, MODE_TDSE = 0, 1
PREC_FP64, PREC_MIXED, PREC_FP32_REFINED = 0, 1, 2
WINDOW_AUTO, WINDOW_TWO_PHASE, WINDOW_FUSED, WINDOW_SPLIT, WINDOW_RESIDENT, WINDOW_CLUSTER = 0, 1, 2, 3, 4, 5
TC_ROBIN, TC_DIRICHLET = 0, 1
SYM_NONE, SYM_ANTISYMMETRIC = 0, 1
LAUNCH_GRAPH, LAUNCH_DIRECT = 0, 1
CONTRACT_AUTO, CONTRACT_FP64, CONTRACT_TENSOR = 0, 1, 2
GET, SET = 0, 1
(FIELD_ENERGY, FIELD_NORM2, FIELD_DIPOLE, FIELD_RES, FIELD_WINDOW, FIELD_PSI_NODES, FIELD_OWN_TRACES,
 FIELD_ROBIN, FIELD_TRACE_BYTES, FIELD_NODE_COUNTS, FIELD_K_MAX, FIELD_COUNTERS, FIELD_CVTOT) = range(13)


class swr_instance(C.Structure):
    _fields_ = [
        ("n_elec", C.c_int), ("box_lo", C.c_double), ("box_hi", C.c_double), ("L", C.c_int),
        ("overlap", C.c_double), ("K_d", C.c_int), ("K_d_per_sub", C.POINTER(C.c_int)),
        ("delta", C.c_double), ("delta_per_sub", C.POINTER(C.c_double)), ("q_p", C.c_int),
        ("n_mid", C.c_int), ("n_nuclei", C.c_int), ("x_nuc", C.c_double * 3), ("Z_nuc", C.c_double * 3),
        ("eta_en", C.c_double), ("eta_ee", C.c_double), ("ee_coef", C.c_double), ("harmonic", C.c_double),
        ("kinetic", C.c_double), ("mu_re", C.c_double), ("mu_im", C.c_double), ("mode", C.c_int),
        ("normalize", C.c_int), ("dt", C.c_double), ("n_steps", C.c_int), ("ngf_tol", C.c_double),
        ("max_steps", C.c_int), ("field_E0", C.c_double), ("field_T", C.c_double),
        ("field_omega", C.c_double), ("field_phase", C.c_double), ("phi0_gamma", C.c_double),
        ("phi0_center", C.c_double * 2), ("orth_tau", C.c_double), ("tc", C.c_int), ("symmetry", C.c_int),
    ]


class swr_problem(C.Structure):
    _fields_ = [("n_instances", C.c_int), ("instances", C.POINTER(swr_instance)), ("precision", C.c_int),
                ("stream", C.c_void_p), ("workspace", C.c_void_p), ("workspace_bytes", C.c_size_t),
                ("window_variant", C.c_int), ("rows_per_task", C.c_int), ("launch_mode", C.c_int),
                ("refine_res", C.c_double), ("spin_limit", C.c_longlong), ("contraction_path", C.c_int),
                ("cvtot_each_iteration", C.c_int)]


class swr_tune_report(C.Structure):
    _fields_ = [("variant", C.c_int), ("rows_per_task", C.c_int), ("tasks", C.c_int), ("ctas", C.c_int),
                ("task_state_global", C.c_int), ("candidates", C.c_int), ("graph", C.c_int),
                ("seconds_per_step", C.c_double),
                ("seconds_default", C.c_double), ("tensor_contractions", C.c_int)]


class swr_iter_report(C.Structure):
    _fields_ = [("k", C.c_int), ("res", C.c_double), ("window_max", C.c_int),
                ("subdomain_solves", C.c_longlong), ("seconds", C.c_double), ("cvtot", C.c_double),
                ("fp32_matrices", C.c_int)]


class swr_report(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("res_last", C.c_double),
                ("subdomain_solves", C.c_longlong), ("seconds", C.c_double), ("fp32_iterations", C.c_int)]


class swr_trace_view(C.Structure):
    _fields_ = [("host", C.c_void_p), ("bytes", C.c_size_t)]


class swr_lsd_problem(C.Structure):
    _fields_ = [("box_lo", C.c_double), ("box_hi", C.c_double), ("L", C.c_int), ("overlap", C.c_double),
                ("n_nuclei", C.c_int), ("x_nuc", C.c_double * 3), ("Z_nuc", C.c_double * 3),
                ("eta_en", C.c_double), ("eta_ee", C.c_double), ("ee_coef", C.c_double), ("harmonic", C.c_double),
                ("M", C.c_int), ("K", C.c_int), ("kd", C.c_int), ("delta", C.c_double), ("xb_factor", C.c_double),
                ("eps_b", C.c_double), ("v_inf", C.c_double), ("q_p", C.c_int), ("panel", C.c_double)]


class swr_lsd_result(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("lam", "coef", "S1", "h1", "J1", "pairs", "S_lsd", "H_lsd", "G_next")]


EXPORTS = ["swr_workspace_size", "swr_setup", "swr_assemble", "swr_step", "swr_iterate", "swr_traces",
           "swr_get", "swr_field_bytes", "swr_trace_codec", "swr_trace_encode", "swr_trace_decode_set",
           "swr_mlp_create", "swr_mlp_param_count", "swr_mlp_set_params", "swr_mlp_get_params",
           "swr_mlp_forward", "swr_mlp_train_step", "swr_mlp_destroy", "swr_mlp_last_error",
           "swr_residual_noalloc", "swr_autotune", "swr_window_plan", "swr_set_spin_limit", "swr_destroy",
           "swr_last_error", "swr_lsd_build"]

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libswr.so (raises when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libswr.so not found at {path}: run paper_1710_02401_gb300/build.py "
                           "(the SWR sweep has no CPU fallback)")
    lib = C.CDLL(path)
    lib.swr_workspace_size.argtypes = [C.POINTER(swr_problem), C.POINTER(C.c_size_t)]
    lib.swr_setup.argtypes = [C.POINTER(swr_problem), C.POINTER(C.c_void_p)]
    lib.swr_assemble.argtypes = [C.c_void_p]
    lib.swr_step.argtypes = [C.c_void_p, C.POINTER(swr_iter_report)]
    lib.swr_iterate.argtypes = [C.c_void_p, C.c_double, C.c_int, C.POINTER(swr_report), C.POINTER(C.c_double)]
    lib.swr_traces.argtypes = [C.c_void_p, C.c_int, C.POINTER(swr_trace_view)]
    lib.swr_get.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t]
    lib.swr_field_bytes.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_size_t)]
    lib.swr_residual_noalloc.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.c_size_t]
    lib.swr_set_spin_limit.argtypes = [C.c_void_p, C.c_longlong]
    lib.swr_autotune.argtypes = [C.c_void_p, C.c_int, C.POINTER(swr_tune_report)]
    lib.swr_window_plan.argtypes = [C.c_void_p, C.POINTER(swr_tune_report)]
    lib.swr_trace_codec.argtypes = [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_size_t)]
    lib.swr_trace_encode.argtypes = [C.c_void_p, C.c_void_p]
    lib.swr_trace_decode_set.argtypes = [C.c_void_p, C.c_void_p]
    lib.swr_mlp_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]
    lib.swr_mlp_param_count.argtypes = [C.c_void_p, C.POINTER(C.c_size_t)]
    lib.swr_mlp_set_params.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t]
    lib.swr_mlp_get_params.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t]
    lib.swr_mlp_forward.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
    lib.swr_mlp_train_step.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_float,
                                       C.POINTER(C.c_float), C.c_void_p]
    lib.swr_mlp_destroy.argtypes = [C.c_void_p]
    lib.swr_mlp_destroy.restype = None
    lib.swr_mlp_last_error.argtypes = [C.c_void_p]
    lib.swr_mlp_last_error.restype = C.c_char_p
    lib.swr_destroy.argtypes = [C.c_void_p]
    lib.swr_destroy.restype = None
    lib.swr_last_error.argtypes = [C.c_void_p]
    lib.swr_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("swr_destroy", "swr_last_error", "swr_mlp_destroy", "swr_mlp_last_error"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


class SWRError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


def _to_c_instance(inst: P.Instance, keep: list) -> swr_instance:
    ci = swr_instance()
    ci.n_elec = inst.n_elec
    ci.box_lo, ci.box_hi = float(inst.box[0]), float(inst.box[1])
    ci.L = inst.L
    ci.overlap = float(inst.overlap)
    if isinstance(inst.K_d, int):
        ci.K_d = inst.K_d
        ci.K_d_per_sub = None
    else:
        arr = (C.c_int * len(inst.K_d))(*[int(k) for k in inst.K_d])
        keep.append(arr)
        ci.K_d = int(inst.K_d[0])
        ci.K_d_per_sub = C.cast(arr, C.POINTER(C.c_int))
    if isinstance(inst.delta, (int, float)):
        ci.delta = float(inst.delta)
        ci.delta_per_sub = None
    else:
        arr = (C.c_double * len(inst.delta))(*[float(d) for d in inst.delta])
        keep.append(arr)
        ci.delta = float(inst.delta[0])
        ci.delta_per_sub = C.cast(arr, C.POINTER(C.c_double))
    ci.q_p = inst.q_p
    ci.n_mid = inst.n_mid
    ci.n_nuclei = len(inst.nuclei)
    for a, (x, z) in enumerate(inst.nuclei):
        ci.x_nuc[a] = float(x)
        ci.Z_nuc[a] = float(z)
    ci.eta_en, ci.eta_ee = float(inst.eta_en), float(inst.eta_ee)
    ci.ee_coef = float(inst.ee_coef)
    ci.harmonic = float(inst.harmonic)
    ci.kinetic = float(inst.kinetic)
    mu = complex(inst.mu)
    ci.mu_re, ci.mu_im = mu.real, mu.imag
    ci.mode = MODE_TDSE if inst.mode == P.TDSE else MODE_TISE
    ci.normalize = 1 if inst.normalize else 0
    ci.dt = float(inst.dt)
    ci.n_steps = int(inst.n_steps)
    ci.ngf_tol = float(inst.ngf_tol)
    ci.max_steps = int(inst.max_steps)
    ci.field_E0, ci.field_T, ci.field_omega, ci.field_phase = (float(f) for f in inst.field)
    ci.phi0_gamma = float(inst.phi0_gamma)
    ci.phi0_center[0], ci.phi0_center[1] = float(inst.phi0_center[0]), float(inst.phi0_center[1])
    ci.orth_tau = float(inst.orth_tau)
    ci.tc = TC_DIRICHLET if inst.tc == "dirichlet" else TC_ROBIN
    ci.symmetry = SYM_ANTISYMMETRIC if inst.symmetry == "antisymmetric" else SYM_NONE
    return ci


def workspace_bytes(instances, precision: int = PREC_FP64, window_variant: int = 0,
                    rows_per_task: int = 0) -> int:
    """Device bytes a context over `instances` needs (swr_workspace_size)."""
    lib = load_library()
    if isinstance(instances, P.Instance):
        instances = [instances]
    keep: list = []
    arr = (swr_instance * len(instances))()
    for i, inst in enumerate(instances):
        arr[i] = _to_c_instance(inst, keep)
    prob = swr_problem()
    prob.n_instances = len(instances)
    prob.instances = C.cast(arr, C.POINTER(swr_instance))
    prob.precision = precision
    prob.window_variant = int(window_variant)
    prob.rows_per_task = int(rows_per_task)
    n = C.c_size_t(0)
    st = lib.swr_workspace_size(C.byref(prob), C.byref(n))
    if st != SWR_OK:
        msg = lib.swr_last_error(None)
        raise SWRError(st, msg.decode() if msg else "")
    return int(n.value)


class SWR:
    """One SWR context over a batch of instances (all subdomains of all
    instances in one sweep).  Device memory is a torch uint8 tensor owned by
    this object; work is ordered on `stream` (default: torch's current)."""

    def __init__(self, instances, precision: int = PREC_FP64, device: str = "cuda:0", stream=None,
                 use_torch_workspace: bool = True, window_variant: int = 0, rows_per_task: int = 0,
                 launch_mode: int = 0, spin_limit: int = 0, refine_res: float = 0.0, contraction_path: int = 0,
                 cvtot_each_iteration: bool = False):
        import torch
        self.lib = load_library()
        if isinstance(instances, P.Instance):
            instances = [instances]
        self.instances = list(instances)
        self._keep: list = []
        arr = (swr_instance * len(self.instances))()
        for i, inst in enumerate(self.instances):
            arr[i] = _to_c_instance(inst, self._keep)
        self._arr = arr
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        prob = swr_problem()
        prob.n_instances = len(self.instances)
        prob.instances = C.cast(arr, C.POINTER(swr_instance))
        prob.precision = precision
        prob.stream = C.c_void_p(self.stream.cuda_stream)
        prob.window_variant = int(window_variant)
        prob.rows_per_task = int(rows_per_task)
        prob.launch_mode = int(launch_mode)
        prob.spin_limit = int(spin_limit)
        prob.refine_res = float(refine_res)
        prob.contraction_path = int(contraction_path)
        prob.cvtot_each_iteration = 1 if cvtot_each_iteration else 0
        nbytes = C.c_size_t(0)
        self._check(self.lib.swr_workspace_size(C.byref(prob), C.byref(nbytes)), None)
        self.workspace = None
        if use_torch_workspace:
            self.workspace = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8, device=self.device)
            base = self.workspace.data_ptr()
            aligned = (base + 255) & ~255
            prob.workspace = C.c_void_p(aligned)
            prob.workspace_bytes = int(nbytes.value)
        self.workspace_bytes = int(nbytes.value)
        self._prob = prob
        ctx = C.c_void_p(None)
        self._check(self.lib.swr_setup(C.byref(prob), C.byref(ctx)), None)
        self.ctx = ctx

    # ------------------------------------------------------------ plumbing
    def _check(self, st: int, ctx) -> None:
        if st != SWR_OK:
            msg = self.lib.swr_last_error(ctx if ctx is not None else None)
            raise SWRError(st, msg.decode() if msg else "")

    def close(self) -> None:
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            self.lib.swr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ the ABI
    def assemble(self) -> None:
        self._check(self.lib.swr_assemble(self.ctx), self.ctx)

    def step(self) -> swr_iter_report:
        rep = swr_iter_report()
        self._check(self.lib.swr_step(self.ctx, C.byref(rep)), self.ctx)
        return rep

    def autotune(self, steps: int = 24) -> dict:
        """Times the window plans on a fixed window and keeps the fastest."""
        rep = swr_tune_report()
        self._check(self.lib.swr_autotune(self.ctx, int(steps), C.byref(rep)), self.ctx)
        return {f: getattr(rep, f) for f, _ in swr_tune_report._fields_}

    def window_plan(self) -> dict:
        rep = swr_tune_report()
        self._check(self.lib.swr_window_plan(self.ctx, C.byref(rep)), self.ctx)
        return {f: getattr(rep, f) for f, _ in swr_tune_report._fields_}

    def iterate(self, tol: float, kmax: int, raise_on_notconv: bool = False):
        rep = swr_report()
        hist = (C.c_double * kmax)()
        st = self.lib.swr_iterate(self.ctx, float(tol), int(kmax), C.byref(rep), hist)
        if st != SWR_OK and not (st == SWR_ENOTCONV and not raise_on_notconv):
            self._check(st, self.ctx)
        return rep, list(hist[: rep.iterations])

    def field_bytes(self, field: int) -> int:
        n = C.c_size_t(0)
        self._check(self.lib.swr_field_bytes(self.ctx, field, C.byref(n)), self.ctx)
        return int(n.value)

    def get(self, field: int, dtype=np.float64) -> np.ndarray:
        nb = self.field_bytes(field)
        out = np.empty(nb // np.dtype(dtype).itemsize, dtype=dtype)
        self._check(self.lib.swr_get(self.ctx, field, out.ctypes.data_as(C.c_void_p), nb), self.ctx)
        return out

    def set_spin_limit(self, polls: int) -> None:
        """Polls before a device-side wait gives up (0: the default)."""
        self._check(self.lib.swr_set_spin_limit(self.ctx, int(polls)), self.ctx)

    def residual_noalloc(self) -> np.ndarray:
        """Res(k) of the last iteration recomputed by the allocation-free entry point."""
        out = np.empty(len(self.instances), dtype=np.float64)
        self._check(self.lib.swr_residual_noalloc(self.ctx, out.ctypes.data_as(C.POINTER(C.c_double)),
                                                  out.size), self.ctx)
        return out

    # ------------------------------------------------------ trace codes
    def trace_codec(self, S: int, Tm: int) -> int:
        n = C.c_size_t(0)
        self._check(self.lib.swr_trace_codec(self.ctx, S, Tm, C.byref(n)), self.ctx)
        self.code_floats = int(n.value)
        return self.code_floats

    def n_sub_total(self) -> int:
        return sum(inst.n_sub for inst in self.instances)

    def trace_encode(self):
        """Codes of the last iteration's Robin data as a CUDA float32 tensor [n_sub, floats]."""
        import torch
        out = torch.empty(self.n_sub_total(), self.code_floats, dtype=torch.float32, device=self.device)
        self._check(self.lib.swr_trace_encode(self.ctx, C.c_void_p(out.data_ptr())), self.ctx)
        return out

    def trace_decode_set(self, code) -> None:
        """Start the next Schwarz iteration from the decoded codes (CUDA float32 tensor)."""
        code = code.contiguous()
        self._check(self.lib.swr_trace_decode_set(self.ctx, C.c_void_p(code.data_ptr())), self.ctx)

    def trace_bytes(self) -> int:
        return int(self.get(FIELD_TRACE_BYTES, dtype=np.uint64)[0])

    def traces_get(self) -> np.ndarray:
        buf = np.empty(self.trace_bytes(), dtype=np.uint8)
        view = swr_trace_view(buf.ctypes.data_as(C.c_void_p), buf.nbytes)
        self._check(self.lib.swr_traces(self.ctx, GET, C.byref(view)), self.ctx)
        return buf

    def traces_set(self, buf: np.ndarray) -> None:
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        view = swr_trace_view(buf.ctypes.data_as(C.c_void_p), buf.nbytes)
        self._check(self.lib.swr_traces(self.ctx, SET, C.byref(view)), self.ctx)

    # ------------------------------------------------------------ results
    def counters(self) -> dict:
        c = self.get(FIELD_COUNTERS)
        keys = ["window_ms", "window_launches", "kernel_launches", "window_flops", "window_bytes",
                "solves", "assemble_ms", "step_ms", "h2d_bytes", "d2h_bytes", "window_bytes_alg"]
        return dict(zip(keys, (float(x) for x in c)))

    def energy(self) -> np.ndarray:
        return self.get(FIELD_ENERGY)

    def residual(self) -> np.ndarray:
        return self.get(FIELD_RES)

    def cvtot(self) -> np.ndarray:
        """Interface mismatch CVTOT(k) of the last iteration per instance (Eq. CVTOT / CVTOT2)."""
        return self.get(FIELD_CVTOT)

    def window(self) -> np.ndarray:
        return self.get(FIELD_WINDOW, dtype=np.int32)

    def node_counts(self) -> np.ndarray:
        return self.get(FIELD_NODE_COUNTS, dtype=np.int32).reshape(-1, 3)

    @property
    def complex(self) -> bool:
        return self.instances[0].mode == P.TDSE

    def dipole(self) -> np.ndarray:
        return self.get(FIELD_DIPOLE)

    def norm2(self) -> np.ndarray:
        return self.get(FIELD_NORM2)

    def psi_nodes(self) -> List[np.ndarray]:
        """psi_i at the volume nodes of every subdomain (node p = q1 + q*q2);
        complex in real time."""
        flat = self.get(FIELD_PSI_NODES)
        nch = 2 if self.complex else 1
        out, o = [], 0
        for (q, ng, K), inst_sub in zip(self.node_counts(), self._sub_n()):
            n = q ** inst_sub
            blk = flat[o:o + n * nch]
            out.append(blk[0::2] + 1j * blk[1::2] if nch == 2 else blk)
            o += n * nch
        return out

    def _sub_n(self):
        for inst in self.instances:
            for _ in range(inst.n_sub):
                yield inst.n_elec

    def own_traces(self) -> List[np.ndarray]:
        return self._per_sub_steps(FIELD_OWN_TRACES)

    def robin_data(self) -> List[np.ndarray]:
        return self._per_sub_steps(FIELD_ROBIN)

    def _per_sub_steps(self, field):
        flat = self.get(field)
        win = self.window()
        nch = 2 if self.complex else 1
        out, o, s = [], 0, 0
        counts = self.node_counts()
        for i, inst in enumerate(self.instances):
            for _ in range(inst.n_sub):
                ng = int(counts[s][1])
                n = (int(win[i]) + 1) * ng * nch
                blk = flat[o:o + n].reshape(int(win[i]) + 1, nch, ng)
                out.append(blk[:, 0, :] + 1j * blk[:, 1, :] if nch == 2 else blk[:, 0, :])
                o += n
                s += 1
        return out


class MLP:
    """BF16 multilayer perceptron with its own CUDA forward/backward/Adam
    kernels (tanh hidden layers).  Device arrays are torch CUDA tensors."""

    def __init__(self, n_in: int, width: int, n_hidden: int, n_out: int, stream=None, device="cuda:0"):
        import torch
        self.lib = load_library()
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.dims = [n_in] + [width] * n_hidden + [n_out]
        h = C.c_void_p(None)
        st = self.lib.swr_mlp_create(n_in, width, n_hidden, n_out, C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != SWR_OK:
            raise SWRError(st, "swr_mlp_create")
        self.h = h
        n = C.c_size_t(0)
        self.lib.swr_mlp_param_count(self.h, C.byref(n))
        self.n_params = int(n.value)

    def _check(self, st):
        if st != SWR_OK:
            raise SWRError(st, self.lib.swr_mlp_last_error(self.h).decode())

    def set_params(self, p: np.ndarray) -> None:
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(self.lib.swr_mlp_set_params(self.h, p.ctypes.data_as(C.c_void_p), p.size))

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        self._check(self.lib.swr_mlp_get_params(self.h, out.ctypes.data_as(C.c_void_p), out.size))
        return out

    def forward(self, x):
        import torch
        x = x.contiguous()
        y = torch.empty(x.shape[0], self.dims[-1], dtype=torch.float32, device=self.device)
        self._check(self.lib.swr_mlp_forward(self.h, C.c_void_p(x.data_ptr()), x.shape[0], C.c_void_p(y.data_ptr())))
        return y

    def train_step(self, x, t, lr: float, want_grad: bool = False):
        x = x.contiguous()
        t = t.contiguous()
        loss = C.c_float(0.0)
        g = np.empty(self.n_params, dtype=np.float32) if want_grad else None
        self._check(self.lib.swr_mlp_train_step(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(t.data_ptr()),
                                                x.shape[0], float(lr), C.byref(loss),
                                                g.ctypes.data_as(C.c_void_p) if g is not None else None))
        return float(loss.value), g

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.swr_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lsd_build(box=(-8.0, 8.0), L=5, overlap=0.32, nuclei=((-0.5, 1.0), (0.5, 1.0)), eta_en=0.5, eta_ee=0.5,
              ee_coef=1.0, harmonic=0.0, M=10, K=45, kd=40, delta=0.0, xb_factor=0.5, eps_b=0.4, v_inf=100.0,
              q_p=12, panel=0.2) -> dict:
    """Local orbitals and local Slater determinants (swr_lsd_build): orbital
    energies and coefficients, one-electron integrals, and per 2-D subdomain
    the determinants' (l, p), Gram, H0 and Gram against the next subdomain in
    x1.  Argument meaning as in include/swr.h."""
    lib = load_library()
    lib.swr_lsd_build.argtypes = [C.POINTER(swr_lsd_problem), C.POINTER(swr_lsd_result)]
    lib.swr_lsd_build.restype = C.c_int
    p = swr_lsd_problem()
    p.box_lo, p.box_hi, p.L, p.overlap = float(box[0]), float(box[1]), int(L), float(overlap)
    p.n_nuclei = len(nuclei)
    for a, (x, z) in enumerate(nuclei):
        p.x_nuc[a], p.Z_nuc[a] = float(x), float(z)
    p.eta_en, p.eta_ee, p.ee_coef, p.harmonic = float(eta_en), float(eta_ee), float(ee_coef), float(harmonic)
    p.M, p.K, p.kd, p.delta = int(M), int(K), int(kd), float(delta)
    p.xb_factor, p.eps_b, p.v_inf, p.q_p, p.panel = float(xb_factor), float(eps_b), float(v_inf), int(q_p), float(panel)
    LM = L * M
    out = {"lam": np.zeros((L, M)), "coef": np.zeros((L, kd, M)), "S1": np.zeros((LM, LM)),
           "h1": np.zeros((LM, LM)), "J1": np.zeros((LM, LM)), "pairs": np.zeros((L * L, K, 2), dtype=np.int32),
           "S_lsd": np.zeros((L * L, K, K)), "H_lsd": np.zeros((L * L, K, K)), "G_next": np.zeros((L * L, K, K))}
    r = swr_lsd_result(*[out[k].ctypes.data for k, _ in swr_lsd_result._fields_])
    st = lib.swr_lsd_build(C.byref(p), C.byref(r))
    if st != SWR_OK:
        msg = lib.swr_last_error(None)
        raise SWRError(st, msg.decode() if msg else "")
    return out
