"""Multigrid continuation (Section 6): solve on a coarse grid, interpolate the
ground state spectrally onto a grid twice as fine (gpe_interpolate), solve
again from it, up to the finest grid.  Orchestration only: every solve and
every interpolation runs in libgpe's kernels.

    phi, reports = multigrid_solve([64, 128, 256, 512], L=(16.0, 16.0), eta=500.0,
                                   omega=0.9, V_of=lambda n, L: inputs.harmonic(n, L))
"""
from __future__ import annotations

import numpy as np

from . import gpe as G


def multigrid_solve(levels, L, eta, omega, V_of, prec=G.GPE_MIXED, phi0=None, opts=None, coarse_tol=1e-10,
                    device="cuda"):
    """levels: grid sizes per axis (each twice the previous; an int for a cube or
    square of that size, or a tuple); V_of(n, L) -> float64 potential on grid n.
    The coarsest solve starts from phi0 (complex128, host or device) or, when
    None, from the Thomas-Fermi state (gpe_thomas_fermi).  Coarse levels stop at
    ||r||_inf < coarse_tol, the finest at opts.tol_res_inf.  Returns (phi on the
    finest grid as a torch complex128 tensor, list of per-level reports)."""
    import torch

    dim = len(L)
    grids = [tuple([lv] * dim) if np.isscalar(lv) else tuple(lv) for lv in levels]
    final_opts = opts or G.solve_opts_default()
    reports, prev_ctx, phi = [], None, None
    try:
        for i, n in enumerate(grids):
            ctx = G.Context(n, L, eta, omega, V_of(n, L), prec=prec)
            shape = tuple(reversed(n))
            cur = torch.empty(shape, dtype=torch.complex128, device=device)
            if prev_ctx is None:
                if phi0 is None:
                    ctx.thomas_fermi(cur)
                else:
                    cur.copy_(torch.as_tensor(phi0, dtype=torch.complex128))
            else:
                prev_ctx.interpolate_to(ctx, phi, cur)
                prev_ctx.close()
            o = G.gpe_solve_opts.from_buffer_copy(final_opts)
            if i < len(grids) - 1:
                o.tol_res_inf = coarse_tol
            rep = ctx.pcg_solve(cur, o)
            rep["grid"] = n
            reports.append(rep)
            prev_ctx, phi = ctx, cur
    finally:
        if prev_ctx is not None:
            prev_ctx.close()
    return phi, reports
