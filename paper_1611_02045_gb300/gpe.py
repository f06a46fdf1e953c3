"""Thin ctypes binding of libgpe (include/gpe.h): argument marshalling only.

Every computation runs in libgpe's CUDA kernels.  There is no CPU fallback:
if libgpe.so is missing or cannot be loaded, every call raises.

Field arguments may be torch tensors (device or host), numpy arrays (host) or
raw integer addresses.  PyTorch is used only to hold device memory and to
provide the stream.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "libgpe.so"

GPE_OK, GPE_ERR_ARG, GPE_ERR_CUDA, GPE_ERR_NOT_CONVERGED, GPE_ERR_NONFINITE, GPE_ERR_PRECOND, \
    GPE_ERR_TIMEOUT, GPE_ERR_UNSUPPORTED = range(8)
GPE_FP64, GPE_MIXED = 0, 1
GPE_PRECOND_C, GPE_PRECOND_DELTA, GPE_PRECOND_V, GPE_PRECOND_C1, GPE_PRECOND_C2, GPE_PRECOND_NONE = range(6)
GPE_BETA_PR, GPE_BETA_FR = 0, 1
GPE_LINE_MODEL, GPE_LINE_EXACT = 0, 1
GPE_LOG_FIELDS = 12
LOG_COLUMNS = ("n", "phase", "E", "lam", "res_inf", "res_l2", "alpha", "beta", "theta", "dE",
               "fallback", "backtracks")
STATUS_NAMES = {0: "ok", 1: "arg", 2: "cuda", 3: "not_converged", 4: "nonfinite", 5: "precond",
                6: "timeout", 7: "unsupported"}


class gpe_problem(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("L", C.c_double * 3), ("eta", C.c_double),
                ("omega", C.c_double), ("prec", C.c_int)]


class gpe_solve_opts(C.Structure):
    _fields_ = [("tol_res_inf", C.c_double), ("tol_dE", C.c_double), ("max_iter", C.c_int),
                ("theta_default", C.c_double), ("max_backtracks", C.c_int), ("cg", C.c_int),
                ("stall_window", C.c_int), ("switch_res", C.c_double), ("max_iter_lo", C.c_int),
                ("use_graph", C.c_int), ("refine_restart", C.c_int), ("precond", C.c_int),
                ("beta_rule", C.c_int), ("line_search", C.c_int), ("wait_polls", C.c_int)]


class gpe_report(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("iters_lo", C.c_int), ("fallbacks", C.c_int),
                ("backtracks", C.c_int), ("E", C.c_double), ("lambda_", C.c_double), ("res_inf", C.c_double),
                ("res_l2", C.c_double), ("log_cap", C.c_int), ("log_len", C.c_int),
                ("log", C.POINTER(C.c_double)), ("loop_kind", C.c_int), ("iters_fp64", C.c_int)]


class gpe_tune_report(C.Structure):
    _fields_ = [("cached", C.c_int), ("candidates", C.c_int), ("us_before", C.c_double * 3),
                ("us_after", C.c_double * 3), ("E", (C.c_int * 3) * 3), ("width", (C.c_int * 3) * 3)]


class GpeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libgpe status {status} ({STATUS_NAMES.get(status, '?')}): {msg}")
        self.status = status


_lib = None
EXPORTED = ("gpe_solve_opts_default", "gpe_create", "gpe_destroy", "gpe_apply_H", "gpe_apply_H_batch", "gpe_precond",
            "gpe_energy", "gpe_set_problem", "gpe_energy_grad", "gpe_tangent_solve", "gpe_density_adjoint",
            "gpe_pcg_solve", "gpe_last_error", "gpe_batch_create", "gpe_batch_solve", "gpe_batch_destroy",
            "gpe_batch_last_error", "gpe_autotune", "gpe_set_plan", "gpe_get_plan", "gpe_batch_autotune",
            "gpe_thomas_fermi", "gpe_interpolate", "gpe_alu_peak")
MODE_NAMES = ("complex64", "fp64", "refinement")
_STRING_RETURNING = ("gpe_last_error", "gpe_batch_last_error")


def lib():
    """Load libgpe.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not _LIB_PATH.exists():
            raise RuntimeError(f"{_LIB_PATH} not built; run paper_1611_02045_gb300.build.build()")
        L = C.CDLL(str(_LIB_PATH))
        vp = C.c_void_p
        L.gpe_solve_opts_default.argtypes = [C.POINTER(gpe_solve_opts)]
        L.gpe_create.argtypes = [C.POINTER(gpe_problem), vp, vp, C.POINTER(vp)]
        L.gpe_destroy.argtypes = [vp]
        L.gpe_apply_H.argtypes = [vp, vp, vp, vp]
        L.gpe_apply_H_batch.argtypes = [vp, C.c_int, vp, vp, vp]
        L.gpe_precond.argtypes = [vp, vp, vp, C.c_double, vp]
        L.gpe_energy.argtypes = [vp, vp, C.POINTER(C.c_double)]
        L.gpe_set_problem.argtypes = [vp, vp, C.c_double, C.c_double]
        L.gpe_energy_grad.argtypes = [vp, vp, vp, vp, C.POINTER(C.c_double)]
        L.gpe_tangent_solve.argtypes = [vp, vp, vp, vp, C.c_double, C.c_int, C.POINTER(C.c_int),
                                        C.POINTER(C.c_double)]
        L.gpe_density_adjoint.argtypes = [vp, vp, vp, vp, C.c_double, C.c_int, C.POINTER(C.c_int),
                                          C.POINTER(C.c_double)]
        L.gpe_pcg_solve.argtypes = [vp, vp, C.POINTER(gpe_solve_opts), C.POINTER(gpe_report)]
        L.gpe_last_error.argtypes = [vp]
        L.gpe_last_error.restype = C.c_char_p
        L.gpe_batch_create.argtypes = [C.c_int, C.POINTER(gpe_problem), C.POINTER(vp), vp, C.POINTER(vp)]
        L.gpe_batch_solve.argtypes = [vp, C.POINTER(vp), C.POINTER(gpe_solve_opts), C.POINTER(gpe_report)]
        L.gpe_batch_destroy.argtypes = [vp]
        L.gpe_batch_last_error.argtypes = [vp]
        L.gpe_batch_last_error.restype = C.c_char_p
        L.gpe_autotune.argtypes = [vp, C.c_int, C.c_int, C.POINTER(gpe_tune_report)]
        L.gpe_set_plan.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int]
        L.gpe_get_plan.argtypes = [vp, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.gpe_batch_autotune.argtypes = [vp, C.c_int]
        L.gpe_thomas_fermi.argtypes = [vp, vp, C.POINTER(C.c_double)]
        L.gpe_interpolate.argtypes = [vp, vp, vp, vp]
        L.gpe_alu_peak.argtypes = [C.c_int, vp, C.POINTER(C.c_double)]
        for name in EXPORTED:
            if name not in _STRING_RETURNING:
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _addr(x):
    """Address of a tensor / array / integer pointer."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("field tensors must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("field arrays must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported field type {type(x)}")


ALU_KINDS = {"fp64_fma": 0, "fp32_fma": 1, "fp32x2_fma": 2}


def alu_peak(kind, stream=None):
    """gpe_alu_peak: GFLOP/s of FP64 fma, FP32 fma or packed FP32x2 fma on the current device."""
    out = C.c_double(0.0)
    s = lib().gpe_alu_peak(ALU_KINDS[kind], _stream_handle(stream), C.byref(out))
    if s != GPE_OK:
        raise GpeError(s, "gpe_alu_peak failed")
    return out.value


def solve_opts_default():
    o = gpe_solve_opts()
    lib().gpe_solve_opts_default(C.byref(o))
    return o


class Context:
    """Owns one gpe_ctx.  Mirrors the C entry points by name."""

    def __init__(self, n, L, eta, omega, V, prec=GPE_FP64, stream=None):
        L_ = lib()
        p = gpe_problem()
        p.dim = len(n)
        for i in range(3):
            p.n[i] = int(n[i]) if i < len(n) else 1
            p.L[i] = float(L[i]) if i < len(L) else 1.0
        p.eta, p.omega, p.prec = float(eta), float(omega), int(prec)
        self.n, self.L, self.prec, self.dim = tuple(n), tuple(L), int(prec), len(n)
        self.eta, self.omega = float(eta), float(omega)
        self._V = V  # keep alive during create
        if isinstance(V, np.ndarray):
            V = np.ascontiguousarray(V, dtype=np.float64)
            self._V = V
        ctx = C.c_void_p()
        st = _stream_handle(stream)
        s = L_.gpe_create(C.byref(p), _addr(V), st, C.byref(ctx))
        if s != GPE_OK:
            raise GpeError(s, L_.gpe_last_error(None).decode())
        self._ctx = ctx

    def _check(self, s):
        if s != GPE_OK:
            raise GpeError(s, lib().gpe_last_error(self._ctx).decode())
        return s

    def apply_H(self, phi, f, out):
        return self._check(lib().gpe_apply_H(self._ctx, _addr(phi), _addr(f), _addr(out)))

    def apply_H_batch(self, nbatch, phi, f, out):
        return self._check(lib().gpe_apply_H_batch(self._ctx, int(nbatch), _addr(phi), _addr(f), _addr(out)))

    def precond(self, phi, r, alpha, out):
        return self._check(lib().gpe_precond(self._ctx, _addr(phi), _addr(r), float(alpha), _addr(out)))

    def energy(self, phi):
        out = (C.c_double * 8)()
        self._check(lib().gpe_energy(self._ctx, _addr(phi), out))
        keys = ("kin", "pot", "int", "rot", "total", "lam", "lam_tilde", "norm2")
        return dict(zip(keys, list(out)))

    def set_problem(self, V=None, eta=None, omega=None):
        """Replace V (float64, host or device; None keeps it), eta and omega (None keeps them)."""
        Vp = V
        if isinstance(V, np.ndarray):
            Vp = np.ascontiguousarray(V, dtype=np.float64)
        eta = self.eta if eta is None else float(eta)
        omega = self.omega if omega is None else float(omega)
        self._check(lib().gpe_set_problem(self._ctx, _addr(Vp), eta, omega))
        self.eta, self.omega = eta, omega

    def energy_grad(self, phi, grad_phi=None, grad_V=None):
        """E and its derivatives at phi (gpe_energy_grad); fills grad_phi / grad_V when given."""
        out = (C.c_double * 5)()
        self._check(lib().gpe_energy_grad(self._ctx, _addr(phi), _addr(grad_phi), _addr(grad_V), out))
        keys = ("E", "dE_deta", "dE_domega", "lam", "norm2")
        return dict(zip(keys, list(out)))

    def autotune(self, iters=20, use_cache=True):
        """gpe_autotune: returns dict(cached, candidates, us_before, us_after, plans) with
        plans[mode_name] = [(E, width) per axis] for the modes the context uses."""
        r = gpe_tune_report()
        self._check(lib().gpe_autotune(self._ctx, int(iters), int(bool(use_cache)), C.byref(r)))
        plans = {MODE_NAMES[m]: [(r.E[m][a], r.width[m][a]) for a in range(self.dim)]
                 for m in range(3) if r.E[m][0]}
        return dict(cached=bool(r.cached), candidates=r.candidates, us_before=list(r.us_before),
                    us_after=list(r.us_after), plans=plans)

    def thomas_fermi(self, phi_out):
        """gpe_thomas_fermi: fills phi_out (complex128, host or device); returns mu."""
        mu = C.c_double(0.0)
        self._check(lib().gpe_thomas_fermi(self._ctx, _addr(phi_out), C.byref(mu)))
        return mu.value

    def interpolate_to(self, fine, phi_c, phi_f):
        """gpe_interpolate: phi_c (this context's grid) onto fine's grid into phi_f."""
        s = lib().gpe_interpolate(self._ctx, _addr(phi_c), fine._ctx, _addr(phi_f))
        if s != GPE_OK:
            raise GpeError(s, lib().gpe_last_error(fine._ctx).decode())

    def set_plan(self, mode, axis, E, width):
        return self._check(lib().gpe_set_plan(self._ctx, int(mode), int(axis), int(E), int(width)))

    def get_plan(self, mode, axis):
        E, w = C.c_int(0), C.c_int(0)
        self._check(lib().gpe_get_plan(self._ctx, int(mode), int(axis), C.byref(E), C.byref(w)))
        return E.value, w.value

    def tangent_solve(self, phi, rhs, z, tol=1e-10, max_iter=2000, check=True):
        """gpe_tangent_solve: z with <phi, z> = 0 solving P K z = P rhs.  Returns
        dict(status, iters, rel_res); raises on failure when check is true."""
        it, res = C.c_int(0), C.c_double(0.0)
        s = lib().gpe_tangent_solve(self._ctx, _addr(phi), _addr(rhs), _addr(z), float(tol), int(max_iter),
                                    C.byref(it), C.byref(res))
        if check:
            self._check(s)
        return dict(status=s, iters=it.value, rel_res=res.value)

    def density_adjoint(self, phi, g_rho, grad_V, tol=1e-10, max_iter=2000, check=True):
        """gpe_density_adjoint: dL/dV for a loss of |phi*|^2 with cotangent g_rho (float64)."""
        it, res = C.c_int(0), C.c_double(0.0)
        s = lib().gpe_density_adjoint(self._ctx, _addr(phi), _addr(g_rho), _addr(grad_V), float(tol), int(max_iter),
                                      C.byref(it), C.byref(res))
        if check:
            self._check(s)
        return dict(status=s, iters=it.value, rel_res=res.value)

    def pcg_solve(self, phi_inout, opts=None, log_cap=0, check=False):
        """Run the solver in place on phi_inout (complex128, host or device).
        Returns a dict with the report and, if log_cap > 0, the per-iteration log."""
        if opts is None:
            opts = solve_opts_default()
        rep = gpe_report()
        logbuf = None
        if log_cap > 0:
            logbuf = np.zeros((log_cap, GPE_LOG_FIELDS), dtype=np.float64)
            rep.log_cap = log_cap
            rep.log = logbuf.ctypes.data_as(C.POINTER(C.c_double))
        s = lib().gpe_pcg_solve(self._ctx, _addr(phi_inout), C.byref(opts), C.byref(rep))
        if s in (GPE_ERR_ARG, GPE_ERR_CUDA) or (check and s != GPE_OK):
            self._check(s)
        out = dict(status=rep.status, status_name=STATUS_NAMES.get(rep.status), iters=rep.iters,
                   iters_lo=rep.iters_lo, fallbacks=rep.fallbacks, backtracks=rep.backtracks, E=rep.E,
                   lam=rep.lambda_, res_inf=rep.res_inf, res_l2=rep.res_l2, loop_kind=rep.loop_kind,
                   iters_fp64=rep.iters_fp64, note=lib().gpe_last_error(self._ctx).decode())
        if logbuf is not None:
            out["log"] = logbuf[: rep.log_len].copy()
        return out

    def close(self):
        if getattr(self, "_ctx", None):
            lib().gpe_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _problem(n, L, eta, omega, prec):
    p = gpe_problem()
    p.dim = len(n)
    for i in range(3):
        p.n[i] = int(n[i]) if i < len(n) else 1
        p.L[i] = float(L[i]) if i < len(L) else 1.0
    p.eta, p.omega, p.prec = float(eta), float(omega), int(prec)
    return p


class Batch:
    """Owns one gpe_batch: many independent solves in one graph launch.

    instances: sequence of dicts with n, L, eta, omega, V (float64 host array or
    device tensor) and optionally prec (default GPE_MIXED)."""

    def __init__(self, instances, stream=None):
        L_ = lib()
        cnt = len(instances)
        probs = (gpe_problem * cnt)()
        Vs = (C.c_void_p * cnt)()
        self._keep = []
        for i, w in enumerate(instances):
            probs[i] = _problem(w["n"], w["L"], w["eta"], w["omega"], w.get("prec", GPE_MIXED))
            V = w["V"]
            if isinstance(V, np.ndarray):
                V = np.ascontiguousarray(V, dtype=np.float64)
            self._keep.append(V)
            Vs[i] = _addr(V)
        b = C.c_void_p()
        s = L_.gpe_batch_create(cnt, probs, Vs, _stream_handle(stream), C.byref(b))
        self._keep = None
        if s != GPE_OK:
            raise GpeError(s, L_.gpe_batch_last_error(None).decode())
        self._b = b
        self.count = cnt

    def solve(self, phis, opts=None, check=False):
        """Solve all instances in place (phis: complex128 tensors/arrays, one per
        instance).  Returns (status, list of per-instance report dicts)."""
        if len(phis) != self.count:
            raise ValueError("one initial guess per instance")
        if opts is None:
            opts = solve_opts_default()
        ptrs = (C.c_void_p * self.count)(*[_addr(p) for p in phis])
        reps = (gpe_report * self.count)()
        s = lib().gpe_batch_solve(self._b, ptrs, C.byref(opts), reps)
        msg = lib().gpe_batch_last_error(self._b).decode()
        if s in (GPE_ERR_ARG, GPE_ERR_CUDA) or (check and s != GPE_OK):
            raise GpeError(s, msg)
        out = [dict(status=r.status, status_name=STATUS_NAMES.get(r.status), iters=r.iters, iters_lo=r.iters_lo,
                    fallbacks=r.fallbacks, backtracks=r.backtracks, E=r.E, lam=r.lambda_, res_inf=r.res_inf,
                    res_l2=r.res_l2, loop_kind=r.loop_kind, iters_fp64=r.iters_fp64) for r in reps]
        return s, out

    def autotune(self, iters=20):
        s = lib().gpe_batch_autotune(self._b, int(iters))
        if s != GPE_OK:
            raise GpeError(s, lib().gpe_batch_last_error(self._b).decode())

    def close(self):
        if getattr(self, "_b", None):
            lib().gpe_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream
