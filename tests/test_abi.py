"""The C ABI: the library builds for sm_103a, loads, exports every function
that include/swr.h declares, and the ctypes mirror of its structs has the
C layout.  CPU only (no CUDA call is made)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

from paper_1710_02401_gb300 import build as B
from paper_1710_02401_gb300 import problems as P
from paper_1710_02401_gb300 import swr as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "swr.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return S.load_library()


def declared_functions():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:swr_status|void|const char\*)\s+(swr_\w+)\s*\(", txt, re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (swr_\w+)", out))
    for n in names:
        assert n in exported, n
        assert hasattr(lib, n)
    assert set(S.EXPORTS) == set(names)


def test_struct_layout_matches_c(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(f'''
#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
#define F(T, m) printf("%s.%s %zu\\n", #T, #m, offsetof(T, m));
int main(void) {{
  printf("swr_instance %zu\\n", sizeof(swr_instance));
  printf("swr_problem %zu\\n", sizeof(swr_problem));
  printf("swr_iter_report %zu\\n", sizeof(swr_iter_report));
  printf("swr_report %zu\\n", sizeof(swr_report));
  printf("swr_trace_view %zu\\n", sizeof(swr_trace_view));
  printf("swr_tune_report %zu\\n", sizeof(swr_tune_report));
  F(swr_instance, delta_per_sub) F(swr_instance, x_nuc) F(swr_instance, mode) F(swr_instance, phi0_center)
  F(swr_instance, max_steps) F(swr_instance, orth_tau) F(swr_instance, tc) F(swr_problem, workspace_bytes) F(swr_iter_report, seconds)
  F(swr_problem, window_variant) F(swr_problem, rows_per_task) F(swr_problem, launch_mode)
  F(swr_problem, spin_limit) F(swr_iter_report, cvtot) F(swr_problem, refine_res) F(swr_iter_report, fp32_matrices)
  F(swr_report, fp32_iterations) F(swr_problem, contraction_path) F(swr_problem, cvtot_each_iteration)
  F(swr_tune_report, graph) F(swr_tune_report, seconds_default) F(swr_tune_report, tensor_contractions)
  printf("swr_lsd_problem %zu\\n", sizeof(swr_lsd_problem));
  printf("swr_lsd_result %zu\\n", sizeof(swr_lsd_result));
  F(swr_lsd_problem, L) F(swr_lsd_problem, overlap) F(swr_lsd_problem, x_nuc) F(swr_lsd_problem, M)
  F(swr_lsd_problem, kd) F(swr_lsd_problem, delta) F(swr_lsd_problem, q_p) F(swr_lsd_problem, panel)
  F(swr_lsd_result, pairs) F(swr_lsd_result, G_next)
  return 0;
}}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", str(prog), "-o", str(exe)], check=True)
    got = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split("\n") if line)
    assert int(got["swr_instance"]) == C.sizeof(S.swr_instance)
    assert int(got["swr_problem"]) == C.sizeof(S.swr_problem)
    assert int(got["swr_iter_report"]) == C.sizeof(S.swr_iter_report)
    assert int(got["swr_report"]) == C.sizeof(S.swr_report)
    assert int(got["swr_trace_view"]) == C.sizeof(S.swr_trace_view)
    for key in ["delta_per_sub", "x_nuc", "mode", "phi0_center", "max_steps", "orth_tau", "tc"]:
        assert int(got[f"swr_instance.{key}"]) == getattr(S.swr_instance, key).offset, key
    assert int(got["swr_problem.workspace_bytes"]) == S.swr_problem.workspace_bytes.offset
    assert int(got["swr_iter_report.seconds"]) == S.swr_iter_report.seconds.offset
    assert int(got["swr_tune_report"]) == C.sizeof(S.swr_tune_report)
    for key in ["window_variant", "rows_per_task", "launch_mode", "spin_limit", "refine_res", "contraction_path",
                "cvtot_each_iteration"]:
        assert int(got[f"swr_problem.{key}"]) == getattr(S.swr_problem, key).offset, key
    for key in ["cvtot", "fp32_matrices"]:
        assert int(got[f"swr_iter_report.{key}"]) == getattr(S.swr_iter_report, key).offset, key
    assert int(got["swr_report.fp32_iterations"]) == S.swr_report.fp32_iterations.offset
    assert int(got["swr_tune_report.seconds_default"]) == S.swr_tune_report.seconds_default.offset
    assert int(got["swr_tune_report.graph"]) == S.swr_tune_report.graph.offset
    assert int(got["swr_tune_report.tensor_contractions"]) == S.swr_tune_report.tensor_contractions.offset
    assert int(got["swr_lsd_problem"]) == C.sizeof(S.swr_lsd_problem)
    assert int(got["swr_lsd_result"]) == C.sizeof(S.swr_lsd_result)
    for key in ["L", "overlap", "x_nuc", "M", "kd", "delta", "q_p", "panel"]:
        assert int(got[f"swr_lsd_problem.{key}"]) == getattr(S.swr_lsd_problem, key).offset, key
    for key in ["pairs", "G_next"]:
        assert int(got[f"swr_lsd_result.{key}"]) == getattr(S.swr_lsd_result, key).offset, key


def _problem(insts, keep):
    arr = (S.swr_instance * len(insts))()
    for i, inst in enumerate(insts):
        arr[i] = S._to_c_instance(inst, keep)
    keep.append(arr)
    p = S.swr_problem()
    p.n_instances = len(insts)
    p.instances = C.cast(arr, C.POINTER(S.swr_instance))
    p.precision = S.PREC_FP64
    return p


def test_workspace_size_and_validation_on_host(lib):
    keep = []
    n = C.c_size_t(0)
    p = _problem([P.small_tise_2d()], keep)
    assert lib.swr_workspace_size(C.byref(p), C.byref(n)) == S.SWR_OK
    assert n.value > 0
    # a bigger window needs more memory
    p2 = _problem([P.small_tise_2d().replace(max_steps=6000)], keep)
    n2 = C.c_size_t(0)
    assert lib.swr_workspace_size(C.byref(p2), C.byref(n2)) == S.SWR_OK
    assert n2.value > n.value
    bad = [
        P.small_tise_2d().replace(n_elec=3),
        P.small_tise_2d().replace(overlap=0.0),
        P.small_tise_2d().replace(overlap=5.0),
        P.small_tise_2d().replace(q_p=0),
        P.small_tise_2d().replace(dt=0.0),
        P.small_tise_2d().replace(K_d=1),
        P.small_tise_2d().replace(delta=-1.0),
        P.small_tise_2d().replace(mu=1 + 1j),
        P.small_tise_2d().replace(ngf_tol=0.0, n_steps=0),
    ]
    for inst in bad:
        st = lib.swr_workspace_size(C.byref(_problem([inst], keep)), C.byref(n))
        assert st == S.SWR_EINVAL, inst
        assert len(lib.swr_last_error(None)) > 0
    empty = S.swr_problem()
    assert lib.swr_workspace_size(C.byref(empty), C.byref(n)) == S.SWR_EINVAL
    neg = _problem([P.small_tise_2d()], keep)
    neg.spin_limit = -1
    assert lib.swr_workspace_size(C.byref(neg), C.byref(n)) == S.SWR_EINVAL
    neg = _problem([P.small_tise_2d()], keep)
    neg.refine_res = -1.0
    assert lib.swr_workspace_size(C.byref(neg), C.byref(n)) == S.SWR_EINVAL
    neg = _problem([P.small_tise_2d()], keep)
    neg.contraction_path = 3
    assert lib.swr_workspace_size(C.byref(neg), C.byref(n)) == S.SWR_EINVAL
    # the tensor-core inverse needs slice scratch: a larger workspace
    tc = _problem([P.small_tise_2d()], keep)
    tc.contraction_path = S.CONTRACT_TENSOR
    n_tc = C.c_size_t(0)
    assert lib.swr_workspace_size(C.byref(tc), C.byref(n_tc)) == S.SWR_OK
    assert n_tc.value > n.value


def test_mixed_modes_rejected(lib):
    keep = []
    n = C.c_size_t(0)
    p = _problem([P.small_tise_2d(), P.small_tdse_2d()], keep)
    assert lib.swr_workspace_size(C.byref(p), C.byref(n)) == S.SWR_EINVAL


def test_window_plan_requests_on_host(lib):
    keep = []
    n = C.c_size_t(0)
    p = _problem([P.small_tise_2d()], keep)
    p.launch_mode = 2
    assert lib.swr_workspace_size(C.byref(p), C.byref(n)) == S.SWR_EINVAL
    p.launch_mode = S.LAUNCH_DIRECT
    for variant, rows, prec, ok in [
        (S.WINDOW_TWO_PHASE, 0, S.PREC_FP64, True),
        (S.WINDOW_TWO_PHASE, 256, S.PREC_MIXED, True),
        (S.WINDOW_FUSED, 0, S.PREC_MIXED, True),
        (S.WINDOW_FUSED, 0, S.PREC_FP64, False),    # the fused kernel is the mixed one
        (S.WINDOW_FUSED, 256, S.PREC_MIXED, False),  # 256-row tasks do not fit its shared memory
        (S.WINDOW_SPLIT, 0, S.PREC_MIXED, True),
        (S.WINDOW_SPLIT, 256, S.PREC_MIXED, True),   # task state in global memory: any task size
        (S.WINDOW_SPLIT, 0, S.PREC_FP64, False),     # the split kernel is the mixed one
        (S.WINDOW_SPLIT, 0, S.PREC_FP32_REFINED, True),
        (S.WINDOW_FUSED, 0, S.PREC_FP32_REFINED, True),
        (0, 0, S.PREC_FP32_REFINED, True),
        (S.WINDOW_TWO_PHASE, 0, S.PREC_FP32_REFINED, False),  # reads both planes: no FP32 phase
        (S.WINDOW_RESIDENT, 0, S.PREC_MIXED, True),
        (S.WINDOW_RESIDENT, 0, S.PREC_FP32_REFINED, True),
        (S.WINDOW_RESIDENT, 0, S.PREC_FP64, False),    # the resident kernel is a mixed one
        (S.WINDOW_RESIDENT, 256, S.PREC_MIXED, False),  # 256-row tasks do not fit its shared memory
        (S.WINDOW_CLUSTER, 0, S.PREC_MIXED, True),
        (S.WINDOW_CLUSTER, 0, S.PREC_FP32_REFINED, True),
        (S.WINDOW_CLUSTER, 0, S.PREC_FP64, False),     # the cluster kernel is a mixed one
        (6, 0, S.PREC_MIXED, False),
        (0, 0, 3, False),
        (0, 4, S.PREC_FP64, False),
        (0, 257, S.PREC_FP64, False),
    ]:
        p.window_variant, p.rows_per_task, p.precision = variant, rows, prec
        st = lib.swr_workspace_size(C.byref(p), C.byref(n))
        assert (st == S.SWR_OK) == ok, (variant, rows, prec, lib.swr_last_error(None))
    # a batch with more row tasks per CTA than shared memory holds plans with the
    # task state in global memory; requesting the two-phase variant never
    # allocates W (nor the Robin response the split window reads), and the
    # fused variant cannot run such a batch
    big = P.batched_uneven(24, seed=3)
    pb = _problem(big, keep)
    pb.precision = S.PREC_MIXED
    auto, two = C.c_size_t(0), C.c_size_t(0)
    assert lib.swr_workspace_size(C.byref(pb), C.byref(auto)) == S.SWR_OK
    pb.window_variant = S.WINDOW_TWO_PHASE
    assert lib.swr_workspace_size(C.byref(pb), C.byref(two)) == S.SWR_OK
    assert two.value <= auto.value
    pb.window_variant = S.WINDOW_FUSED
    assert lib.swr_workspace_size(C.byref(pb), C.byref(n)) == S.SWR_EINVAL
    pb.window_variant = S.WINDOW_SPLIT  # runs it, without W but with the Robin response of every step
    assert lib.swr_workspace_size(C.byref(pb), C.byref(n)) == S.SWR_OK
    assert n.value > two.value
    ps = _problem([P.small_tdse_2d()], keep)
    ps.precision, ps.window_variant = S.PREC_MIXED, S.WINDOW_SPLIT
    assert lib.swr_workspace_size(C.byref(ps), C.byref(n)) == S.SWR_EINVAL  # imaginary time only
    ps.window_variant = S.WINDOW_CLUSTER
    assert lib.swr_workspace_size(C.byref(ps), C.byref(n)) == S.SWR_EINVAL
    # the cluster plan needs one SM per CTA and one cluster per subdomain: a
    # 512-instance batch has more subdomains than the device has SMs
    pb.window_variant = S.WINDOW_CLUSTER
    assert lib.swr_workspace_size(C.byref(pb), C.byref(n)) == S.SWR_EINVAL


def test_transmission_and_symmetry_requests_on_host(lib):
    keep = []
    n = C.c_size_t(0)

    def status(inst, precision=S.PREC_FP64, variant=0, raw=None):
        p = _problem([inst], keep)
        p.precision, p.window_variant = precision, variant
        if raw:  # set a raw field of the C instance (values the Python side does not produce)
            arr = C.cast(p.instances, C.POINTER(S.swr_instance))
            setattr(arr[0], *raw)
        return lib.swr_workspace_size(C.byref(p), C.byref(n))

    anti = P.small_tise_2d().replace(symmetry="antisymmetric", phi0_center=(0.8, -0.8))
    assert status(P.small_tise_2d().replace(tc="dirichlet")) == S.SWR_OK
    assert status(P.small_tise_2d(), raw=("tc", 2)) == S.SWR_EINVAL
    assert status(P.small_tise_2d(), raw=("symmetry", 2)) == S.SWR_EINVAL
    assert status(anti) == S.SWR_OK
    assert status(anti, S.PREC_MIXED) == S.SWR_OK                              # split window
    assert status(anti, S.PREC_MIXED, S.WINDOW_FUSED) == S.SWR_EINVAL          # not the fused one
    assert status(anti, S.PREC_MIXED, S.WINDOW_RESIDENT) == S.SWR_EINVAL       # nor the resident one
    assert status(anti, S.PREC_MIXED, S.WINDOW_CLUSTER) == S.SWR_EINVAL        # nor the cluster one
    assert status(P.tise_1d_two_subdomains().replace(symmetry="antisymmetric")) == S.SWR_EINVAL  # N = 1
    assert status(P.small_tdse_2d().replace(symmetry="antisymmetric")) == S.SWR_OK             # real time too
    kd = [8, 9, 8, 9]  # subdomain (1, 0) and its mirror (0, 1) differ
    assert status(P.small_tise_2d(L=2, K_d=8).replace(K_d=kd, symmetry="antisymmetric")) == S.SWR_EINVAL
    assert status(P.small_tise_2d(L=2, K_d=8).replace(K_d=[8, 9, 9, 8], symmetry="antisymmetric")) == S.SWR_OK
