"""The C ABI without a GPU: libgpe.so loads, exports every entry point that
include/gpe.h declares, the ctypes structures match the C layout, and
argument errors are reported before any CUDA call."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from paper_1611_02045_gb300 import gpe as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gpe.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gpe_[A-Za-z_0-9]+)\s*\(", text)))


def test_header_declares_the_expected_entry_points():
    names = declared_functions()
    for need in ("gpe_create", "gpe_destroy", "gpe_apply_H", "gpe_precond", "gpe_energy", "gpe_pcg_solve",
                 "gpe_last_error", "gpe_solve_opts_default"):
        assert need in names


def test_library_exports_every_declared_symbol(built_lib):
    lib = C.CDLL(str(built_lib))
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(G.EXPORTED) <= set(declared_functions())


def test_ctypes_layout_matches_c(built_lib):
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "gpe.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(gpe_problem), offsetof(gpe_problem, eta), offsetof(gpe_problem, prec));
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(gpe_solve_opts), offsetof(gpe_solve_opts, switch_res), offsetof(gpe_solve_opts, use_graph),
         offsetof(gpe_solve_opts, refine_restart), offsetof(gpe_solve_opts, precond), offsetof(gpe_solve_opts, beta_rule),
         offsetof(gpe_solve_opts, line_search), offsetof(gpe_solve_opts, wait_polls));
  printf("%zu %zu %zu %zu %zu\n", sizeof(gpe_report), offsetof(gpe_report, res_l2), offsetof(gpe_report, log),
         offsetof(gpe_report, loop_kind), offsetof(gpe_report, iters_fp64));
  printf("%zu %zu %zu %zu\n", sizeof(gpe_tune_report), offsetof(gpe_tune_report, us_before),
         offsetof(gpe_tune_report, E), offsetof(gpe_tune_report, width));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "lay.c")
        exe = os.path.join(d, "lay")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    got = list(map(int, out))
    want = [C.sizeof(G.gpe_problem), G.gpe_problem.eta.offset, G.gpe_problem.prec.offset,
            C.sizeof(G.gpe_solve_opts), G.gpe_solve_opts.switch_res.offset, G.gpe_solve_opts.use_graph.offset,
            G.gpe_solve_opts.refine_restart.offset, G.gpe_solve_opts.precond.offset, G.gpe_solve_opts.beta_rule.offset,
            G.gpe_solve_opts.line_search.offset, G.gpe_solve_opts.wait_polls.offset,
            C.sizeof(G.gpe_report), G.gpe_report.res_l2.offset, G.gpe_report.log.offset,
            G.gpe_report.loop_kind.offset, G.gpe_report.iters_fp64.offset,
            C.sizeof(G.gpe_tune_report), G.gpe_tune_report.us_before.offset, G.gpe_tune_report.E.offset,
            G.gpe_tune_report.width.offset]
    assert got == want


def test_solve_opts_defaults(built_lib):
    o = G.solve_opts_default()
    assert o.tol_res_inf == 1e-8 and o.max_iter == 20000 and o.theta_default == 0.1
    assert o.max_backtracks == 30 and o.cg == 1 and o.use_graph == 3 and o.refine_restart == 1
    assert o.precond == G.GPE_PRECOND_C and o.beta_rule == G.GPE_BETA_PR and o.line_search == G.GPE_LINE_MODEL
    assert o.wait_polls == 0
    assert G.lib().gpe_solve_opts_default(None) == G.GPE_ERR_ARG


@pytest.mark.parametrize("bad", [
    dict(dim=4), dict(n=(12, 16)), dict(n=(4, 16)), dict(n=(1024, 16)), dict(L=(-1.0, 1.0)),
    dict(L=(float("nan"), 1.0)), dict(eta=float("inf")), dict(prec=7),
])
def test_create_rejects_bad_arguments_before_cuda(built_lib, bad):
    p = G.gpe_problem()
    args = dict(dim=2, n=(16, 16), L=(4.0, 4.0), eta=1.0, omega=0.5, prec=0)
    args.update(bad)
    p.dim = args["dim"]
    for i in range(3):
        p.n[i] = args["n"][i] if i < len(args["n"]) else 8
        p.L[i] = args["L"][i] if i < len(args["L"]) else 1.0
    p.eta, p.omega, p.prec = args["eta"], args["omega"], args["prec"]
    V = np.zeros(256)
    ctx = C.c_void_p()
    lib = G.lib()
    s = lib.gpe_create(C.byref(p), V.ctypes.data, None, C.byref(ctx))
    assert s == G.GPE_ERR_ARG
    assert ctx.value is None
    assert lib.gpe_last_error(None).decode() != ""


def test_null_arguments(built_lib):
    lib = G.lib()
    assert lib.gpe_create(None, None, None, None) == G.GPE_ERR_ARG
    assert lib.gpe_destroy(None) == G.GPE_OK
    assert lib.gpe_apply_H(None, None, None, None) == G.GPE_ERR_ARG
    assert lib.gpe_energy(None, None, None) == G.GPE_ERR_ARG
    assert lib.gpe_pcg_solve(None, None, None, None) == G.GPE_ERR_ARG
    assert lib.gpe_set_problem(None, None, 1.0, 0.0) == G.GPE_ERR_ARG
    assert lib.gpe_energy_grad(None, None, None, None, None) == G.GPE_ERR_ARG
    assert lib.gpe_tangent_solve(None, None, None, None, 1e-10, 10, None, None) == G.GPE_ERR_ARG
    assert lib.gpe_density_adjoint(None, None, None, None, 1e-10, 10, None, None) == G.GPE_ERR_ARG
    out = C.c_void_p()
    assert lib.gpe_batch_create(0, None, None, None, C.byref(out)) == G.GPE_ERR_ARG and not out.value
    assert lib.gpe_batch_create(1, None, None, None, None) == G.GPE_ERR_ARG
    assert lib.gpe_batch_solve(None, None, None, None) == G.GPE_ERR_ARG
    assert lib.gpe_batch_destroy(None) == G.GPE_OK
    assert lib.gpe_batch_last_error(None) is not None
    assert lib.gpe_autotune(None, 10, 1, None) == G.GPE_ERR_ARG
    assert lib.gpe_set_plan(None, 0, 0, 8, 1) == G.GPE_ERR_ARG
    assert lib.gpe_get_plan(None, 0, 0, None, None) == G.GPE_ERR_ARG
    assert lib.gpe_batch_autotune(None, 10) == G.GPE_ERR_ARG
    assert lib.gpe_thomas_fermi(None, None, None) == G.GPE_ERR_ARG
    assert lib.gpe_interpolate(None, None, None, None) == G.GPE_ERR_ARG


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(G, "_lib", None)
    monkeypatch.setattr(G, "_LIB_PATH", tmp_path / "missing.so")
    with pytest.raises(RuntimeError):
        G.lib()
