"""torch.autograd wrappers over libgpe's derivative entry points.

Argument marshalling only: every value comes from libgpe's kernels
(gpe_energy_grad, gpe_pcg_solve, gpe_density_adjoint); the wrappers move
tensors in and out and multiply the cotangent by the returned derivatives.

Complex gradients follow PyTorch's convention for a real loss: the gradient of
L with respect to a complex tensor phi is dL/dRe phi + i dL/dIm phi, which is
what gpe_energy_grad returns for the energy (2 h^d H_phi phi, Section 2).

  energy(phi, V, eta, omega, ctx)       E at a fixed phi; differentiable in
                                        phi, V, eta and omega.
  ground_state_energy(V, eta, omega, ctx, phi0)
                                        E* of the ground state reached from
                                        phi0; differentiable in V, eta, omega
                                        through the Hellmann-Feynman identities
                                        dE*/dV = h^d |phi*|^2,
                                        dE*/deta = 1/2 int |phi*|^4,
                                        dE*/domega = -<phi*, L_z phi*>.
  ground_state_density(V, ctx, phi0)    rho* = |phi*|^2; differentiable in V
                                        through the tangent-space adjoint solve.

The context `ctx` (gpe.Context of the same grid) is re-targeted to the given
V, eta, omega with gpe_set_problem on every call.
"""
from __future__ import annotations

import torch

from . import gpe as G


def _scalar(x):
    return float(x.detach().item()) if torch.is_tensor(x) else float(x)


def _work_dtype(ctx):
    return torch.complex128 if ctx.prec == G.GPE_FP64 else torch.complex64


def _retarget(ctx, V, eta, omega):
    Vd = V.detach().to(torch.float64).contiguous()
    ctx.set_problem(Vd, _scalar(eta), _scalar(omega))
    return Vd


def _grad_like(x, value):
    """A cotangent for input x (None when x is not a tensor that needs it)."""
    if not torch.is_tensor(x) or not x.requires_grad:
        return None
    return torch.as_tensor(value, dtype=x.dtype, device=x.device).expand_as(x).clone()


class _Energy(torch.autograd.Function):
    @staticmethod
    def forward(fctx, phi, V, eta, omega, ctx):
        Vd = _retarget(ctx, V, eta, omega)
        ph = phi.detach().to(_work_dtype(ctx)).contiguous()
        gphi = torch.empty_like(ph)
        gV = torch.empty_like(Vd)
        out = ctx.energy_grad(ph, gphi, gV)
        fctx.save_for_backward(gphi, gV)
        fctx.d_eta, fctx.d_omega = out["dE_deta"], out["dE_domega"]
        fctx.phi_dtype = phi.dtype
        fctx.inputs = (eta, omega)
        return torch.tensor(out["E"], dtype=torch.float64, device=phi.device)

    @staticmethod
    def backward(fctx, g):
        gphi, gV = fctx.saved_tensors
        eta, omega = fctx.inputs
        d_phi = (g * gphi).to(fctx.phi_dtype) if fctx.needs_input_grad[0] else None
        d_V = g * gV if fctx.needs_input_grad[1] else None
        d_eta = g * fctx.d_eta if fctx.needs_input_grad[2] else None
        d_omega = g * fctx.d_omega if fctx.needs_input_grad[3] else None
        if d_eta is not None and torch.is_tensor(eta):
            d_eta = d_eta.to(eta.dtype).reshape(eta.shape)
        if d_omega is not None and torch.is_tensor(omega):
            d_omega = d_omega.to(omega.dtype).reshape(omega.shape)
        return d_phi, d_V, d_eta, d_omega, None


def energy(phi, V, eta, omega, ctx):
    """E(phi; V, eta, omega) (Section 2) at a fixed phi, differentiable in all four."""
    return _Energy.apply(phi, V, eta, omega, ctx)


def _solve(ctx, phi0, opts):
    phi = phi0.detach().to(torch.complex128).contiguous().clone()
    rep = ctx.pcg_solve(phi, opts)
    if rep["status"] != G.GPE_OK:
        raise G.GpeError(rep["status"], f"ground-state solve did not converge: {rep}")
    return phi, rep


class _GroundStateEnergy(torch.autograd.Function):
    @staticmethod
    def forward(fctx, V, eta, omega, ctx, phi0, opts):
        Vd = _retarget(ctx, V, eta, omega)
        phi, rep = _solve(ctx, phi0, opts)
        ph = phi.to(_work_dtype(ctx))
        gV = torch.empty_like(Vd)
        out = ctx.energy_grad(ph, None, gV)
        fctx.save_for_backward(gV)
        fctx.d_eta, fctx.d_omega = out["dE_deta"], out["dE_domega"]
        fctx.inputs = (eta, omega)
        fctx.mark_non_differentiable(phi)
        return torch.tensor(rep["E"], dtype=torch.float64, device=V.device), phi

    @staticmethod
    def backward(fctx, gE, _gphi):
        (gV,) = fctx.saved_tensors
        eta, omega = fctx.inputs
        d_V = gE * gV if fctx.needs_input_grad[0] else None
        d_eta = gE * fctx.d_eta if fctx.needs_input_grad[1] else None
        d_omega = gE * fctx.d_omega if fctx.needs_input_grad[2] else None
        if d_eta is not None and torch.is_tensor(eta):
            d_eta = d_eta.to(eta.dtype).reshape(eta.shape)
        if d_omega is not None and torch.is_tensor(omega):
            d_omega = d_omega.to(omega.dtype).reshape(omega.shape)
        return d_V, d_eta, d_omega, None, None, None


def ground_state_energy(V, eta, omega, ctx, phi0, opts=None):
    """(E*, phi*) of the ground state reached from phi0; E* differentiable in
    V, eta and omega (Hellmann-Feynman), phi* returned without gradient."""
    return _GroundStateEnergy.apply(V, eta, omega, ctx, phi0, opts)


class _GroundStateDensity(torch.autograd.Function):
    @staticmethod
    def forward(fctx, V, ctx, phi0, opts, tol, max_iter):
        _retarget(ctx, V, ctx.eta, ctx.omega)
        phi, _ = _solve(ctx, phi0, opts)
        fctx.ctx, fctx.tol, fctx.max_iter = ctx, tol, max_iter
        fctx.save_for_backward(phi)
        return (phi.real * phi.real + phi.imag * phi.imag)

    @staticmethod
    def backward(fctx, g_rho):
        (phi,) = fctx.saved_tensors
        ctx = fctx.ctx
        gV = torch.empty(phi.shape, dtype=torch.float64, device=phi.device)
        ph = phi.to(_work_dtype(ctx)).contiguous()
        ctx.density_adjoint(ph, g_rho.detach().to(torch.float64).contiguous(), gV, fctx.tol, fctx.max_iter)
        return gV, None, None, None, None, None


def ground_state_density(V, ctx, phi0, opts=None, tol=1e-10, max_iter=2000):
    """rho* = |phi*|^2 of the ground state of V (the context's eta, omega)
    reached from phi0, differentiable in V through gpe_density_adjoint."""
    return _GroundStateDensity.apply(V, ctx, phi0, opts, tol, max_iter)
