"""Derivatives on the GPU (gpe_energy_grad, gpe_tangent_solve,
gpe_density_adjoint and the torch.autograd wrappers) against the FP64 CPU
oracle and against central finite differences of GPU ground-state solves.

Tolerances
  * gradients at a fixed phi (complex128): max|gpu - oracle| <= 1e-12 max|oracle|
    (the same H_phi passes as gpe_apply_H, scaled);
  * complex64 contexts: 2e-5 relative (FP32 transforms);
  * Hellmann-Feynman against central differences of FP64 solves with h = 1e-6:
    the ground-state energies agree to ~1e-15 relative, so the quotient carries
    ~1e-15 |E| / h ~ 1e-8 absolute error on derivatives of size 1e-3 .. 1;
    rel 1e-5;
  * tangent solve against the oracle's at the same phi and rhs: both stop at
    ||r|| <= 1e-12 ||P rhs||; the solutions differ by ~ cond(K) 1e-12: rel 1e-8;
  * density-loss gradient against differences of solves (h = 1e-6): rel 1e-4.
"""
import numpy as np
import pytest

from oracle import gpe_oracle as O
from paper_1611_02045_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G(built_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_02045_gb300 import gpe
    return gpe


@pytest.fixture(scope="module")
def AG(G):
    from paper_1611_02045_gb300 import autograd
    return autograd


def dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def small_problem(n=(64, 64), L=(8.0, 8.0), eta=50.0, omega=0.4, seed=11):
    V = I.harmonic(n, L) + 0.3 * I.smooth_bumps(n, L, seed)
    return n, L, eta, omega, V


FP64_OPTS_TOL = 1e-11


def solve(G, ctx, phi0, tol=FP64_OPTS_TOL):
    opts = G.solve_opts_default()
    opts.tol_res_inf = tol
    phi = dev(phi0) if not torch.is_tensor(phi0) else phi0.clone()
    rep = ctx.pcg_solve(phi, opts)
    assert rep["status"] == G.GPE_OK, rep
    return phi, rep


# ------------------------------------------------------------ fixed-phi derivatives
@pytest.mark.parametrize("case", ["2d", "2d_omega0", "3d", "2d_nonsquare"])
def test_energy_grad_matches_oracle_fp64(G, case):
    if case == "3d":
        n, L = (16, 32, 16), (4.0, 5.0, 4.0)
        V, eta, omega = I.harmonic(n, L, [1.0, 1.0, 2.0]), 30.0, 0.5
    else:
        n, L = ((32, 64), (5.0, 8.0)) if case == "2d_nonsquare" else ((64, 64), (8.0, 8.0))
        _, _, eta, omega, V = small_problem(n, L)
        if case == "2d_omega0":
            omega = 0.0
    if len(n) == 2:
        phi = I.phi_d(n, L, 0.6)
    else:
        phi = I.normalise(I.anisotropic_gaussian(n, L, [1.0, 1.0, 2.0]) * (1 + 0.5j * I.mesh(n, L)[0]), n, L)
    phi = phi * (1 + 0.1 * I.random_field(5, n, L))
    po = O.Problem(n, L, eta, omega, V)
    with G.Context(n, L, eta, omega, V, prec=G.GPE_FP64) as ctx:
        gphi = torch.empty(phi.shape, dtype=torch.complex128, device="cuda")
        gV = torch.empty(phi.shape, dtype=torch.float64, device="cuda")
        out = ctx.energy_grad(dev(phi), gphi, gV)
    want_g = O.energy_gradient(po, phi)
    d = O.energy_parameter_derivatives(po, phi)
    assert relmax(host(gphi), want_g) < 1e-12
    assert relmax(host(gV), d["dV"]) < 1e-13
    assert abs(out["dE_deta"] - d["deta"]) <= 1e-13 * abs(d["deta"])
    assert abs(out["dE_domega"] - d["domega"]) <= 1e-12 * max(abs(d["domega"]), 1e-3)
    assert abs(out["E"] - O.energy(po, phi)) <= 1e-12 * abs(out["E"])
    assert abs(out["lam"] - O.chemical_potential(po, phi)) <= 1e-12 * abs(out["lam"])


def test_energy_grad_complex64(G):
    n, L, eta, omega, V = small_problem()
    phi = I.phi_d(n, L, 0.6) * (1 + 0.1 * I.random_field(5, n, L))
    po = O.Problem(n, L, eta, omega, V)
    with G.Context(n, L, eta, omega, V, prec=G.GPE_MIXED) as ctx:
        gphi = torch.empty(phi.shape, dtype=torch.complex64, device="cuda")
        gV = torch.empty(phi.shape, dtype=torch.float64, device="cuda")
        ph32 = phi.astype(np.complex64)
        out = ctx.energy_grad(dev(ph32, torch.complex64), gphi, gV)
    ph = ph32.astype(np.complex128)
    assert relmax(host(gphi).astype(np.complex128), O.energy_gradient(po, ph)) < 2e-5
    d = O.energy_parameter_derivatives(po, ph)
    assert relmax(host(gV), d["dV"]) < 1e-12
    assert abs(out["dE_deta"] - d["deta"]) <= 2e-6 * abs(d["deta"])
    assert abs(out["dE_domega"] - d["domega"]) <= 2e-5 * abs(d["domega"])


def test_set_problem_retargets_every_loop(G):
    """gpe_set_problem: energies and a solve after the change equal a fresh
    context's (captured graphs of the old problem are discarded)."""
    n, L, eta, omega, V = small_problem()
    V2 = I.harmonic(n, L) + 0.3 * I.smooth_bumps(n, L, 12)
    phi0 = I.perturbed(I.phi_d(n, L, 0.3), 3, n, L)
    with G.Context(n, L, eta, omega, V, prec=G.GPE_FP64) as a, G.Context(n, L, 70.0, 0.2, V2, prec=G.GPE_FP64) as b:
        solve(G, a, phi0, 1e-8)  # captures the graph for the first problem
        a.set_problem(V2, 70.0, 0.2)
        f = dev(phi0)
        ea, eb = a.energy(f), b.energy(f)
        for k in ea:
            assert abs(ea[k] - eb[k]) <= 1e-13 * max(abs(eb[k]), 1e-300)
        pa, ra = solve(G, a, phi0, 1e-9)
        pb, rb = solve(G, b, phi0, 1e-9)
    assert ra["iters"] == rb["iters"] and abs(ra["E"] - rb["E"]) <= 1e-14 * abs(rb["E"])


# ------------------------------------------------------------ Hellmann-Feynman
@pytest.fixture(scope="module")
def gs_c5(G):
    """Instance 0 of the differentiation batch (256^2, eta 500, omega 0.7,
    V = r^2/2 + 0.1 S): FP64 ground state."""
    w = I.workload("grad256_2d", 0)
    ctx = G.Context(w["n"], w["L"], w["eta"], w["omega"], w["V"], prec=G.GPE_FP64)
    phi, rep = solve(G, ctx, w["phi0"])
    yield w, ctx, phi, rep
    ctx.close()


def _resolve(G, ctx, w, phi, eta=None, omega=None, V=None):
    ctx.set_problem(w["V"] if V is None else V, w["eta"] if eta is None else eta,
                    w["omega"] if omega is None else omega)
    _, rep = solve(G, ctx, phi)
    return rep["E"]


def test_hellmann_feynman_matches_differences_of_solves(G, gs_c5):
    w, ctx, phi, rep = gs_c5
    gV = torch.empty(phi.shape, dtype=torch.float64, device="cuda")
    ctx.set_problem(w["V"], w["eta"], w["omega"])
    out = ctx.energy_grad(phi, None, gV)
    h = 1e-6
    fd = (_resolve(G, ctx, w, phi, eta=w["eta"] + h) - _resolve(G, ctx, w, phi, eta=w["eta"] - h)) / (2 * h)
    assert abs(fd - out["dE_deta"]) <= 1e-5 * abs(out["dE_deta"]), (fd, out)
    fd = (_resolve(G, ctx, w, phi, omega=w["omega"] + h) - _resolve(G, ctx, w, phi, omega=w["omega"] - h)) / (2 * h)
    assert abs(fd - out["dE_domega"]) <= 1e-5 * abs(out["dE_domega"]), (fd, out)
    S = I.smooth_bumps(w["n"], w["L"], 99)
    fd = (_resolve(G, ctx, w, phi, V=w["V"] + h * S) - _resolve(G, ctx, w, phi, V=w["V"] - h * S)) / (2 * h)
    an = float(np.sum(host(gV) * S))
    assert abs(fd - an) <= 1e-5 * abs(an), (fd, an)
    ctx.set_problem(w["V"], w["eta"], w["omega"])
    # and the closed forms, evaluated by the oracle at the same state
    po = O.Problem(w["n"], w["L"], w["eta"], w["omega"], w["V"])
    d = O.energy_parameter_derivatives(po, host(phi))
    assert abs(out["dE_deta"] - d["deta"]) <= 1e-12 * abs(d["deta"])
    assert abs(out["dE_domega"] - d["domega"]) <= 1e-12 * abs(d["domega"])


# ------------------------------------------------------------ tangent-space adjoint
@pytest.fixture(scope="module")
def gs_small(G):
    n, L, eta, omega, V = small_problem(n=(32, 32), L=(6.0, 6.0), eta=20.0, omega=0.3)
    ctx = G.Context(n, L, eta, omega, V, prec=G.GPE_FP64)
    phi, _ = solve(G, ctx, I.perturbed(I.phi_a(n, L), 12, n, L, amp=1e-2), 1e-12)
    yield (n, L, eta, omega, V), ctx, phi
    ctx.close()


def test_tangent_solve_matches_oracle(G, gs_small):
    (n, L, eta, omega, V), ctx, phi = gs_small
    po = O.Problem(n, L, eta, omega, V)
    ph = host(phi)
    lam = O.chemical_potential(po, ph)
    rhs = I.random_field(41, n, L) * np.abs(ph)
    z = torch.empty_like(phi)
    r = ctx.tangent_solve(phi, dev(rhs), z, tol=1e-12, max_iter=1000)
    zo, it, res = O.tangent_solve(po, ph, lam, rhs, tol=1e-12)
    assert r["rel_res"] <= 1e-12 and res <= 1e-12
    assert abs(r["iters"] - it) <= max(3, it // 10), (r, it)
    zg = host(z)
    assert np.linalg.norm(zg - zo) <= 1e-8 * np.linalg.norm(zo)
    assert abs(O.inner(po, ph, zg)) < 1e-12 * O.norm(po, zg)


def test_density_adjoint_matches_oracle(G, gs_small):
    (n, L, eta, omega, V), ctx, phi = gs_small
    po = O.Problem(n, L, eta, omega, V)
    ph = host(phi)
    rho = np.abs(I.normalise(I.anisotropic_gaussian(n, L, [1.3, 0.8]), n, L)) ** 2
    g_rho = 2.0 * po.weight * (np.abs(ph) ** 2 - rho)  # dL/drho for L = h^d sum (rho - rho_t)^2
    gV = torch.empty(ph.shape, dtype=torch.float64, device="cuda")
    r = ctx.density_adjoint(phi, torch.from_numpy(g_rho).cuda(), gV, tol=1e-12, max_iter=1000)
    want, _, _ = O.density_loss_gradient_V(po, ph, rho)
    assert r["rel_res"] <= 1e-12
    assert relmax(host(gV), want) < 1e-8


def test_density_loss_gradient_matches_differences_of_solves(G, AG, gs_c5):
    """The differentiation workload: gradient of int (|phi*|^2 - rho)^2 with
    respect to V through the autograd wrapper, against central differences
    (h = 1e-6) of FP64 ground-state solves along two smooth directions."""
    w, ctx, phi, _ = gs_c5
    n, L = w["n"], w["L"]
    wt = I.weight(n, L)
    rho_t = torch.from_numpy(np.abs(I.normalise(I.anisotropic_gaussian(n, L, [0.05, 0.04]), n, L)) ** 2).cuda()
    opts = ctx_opts(G)
    V = torch.from_numpy(w["V"]).cuda().requires_grad_(True)
    ctx.set_problem(w["V"], w["eta"], w["omega"])
    rho = AG.ground_state_density(V, ctx, phi, opts, tol=1e-11, max_iter=3000)
    loss = wt * torch.sum((rho - rho_t) ** 2)
    loss.backward()
    gV = host(V.grad)

    def L_of(Vn):
        ctx.set_problem(Vn, w["eta"], w["omega"])
        p, _ = solve(G, ctx, phi)
        r = torch.abs(p) ** 2
        return float(wt * torch.sum((r - rho_t) ** 2))

    h = 1e-6
    for seed in (97, 98):
        S = I.smooth_bumps(n, L, seed)
        fd = (L_of(w["V"] + h * S) - L_of(w["V"] - h * S)) / (2 * h)
        an = float(np.sum(gV * S))
        assert abs(fd - an) <= 1e-4 * abs(an), (seed, fd, an)
    ctx.set_problem(w["V"], w["eta"], w["omega"])


def ctx_opts(G):
    o = G.solve_opts_default()
    o.tol_res_inf = FP64_OPTS_TOL
    return o


# ------------------------------------------------------------ autograd wrappers
def test_autograd_energy_matches_oracle(G, AG):
    n, L, eta, omega, V = small_problem()
    po = O.Problem(n, L, eta, omega, V)
    phi_np = I.phi_d(n, L, 0.6) * (1 + 0.1 * I.random_field(5, n, L))
    with G.Context(n, L, eta, omega, V, prec=G.GPE_FP64) as ctx:
        phi = dev(phi_np).requires_grad_(True)
        Vt = torch.from_numpy(V).cuda().requires_grad_(True)
        et = torch.tensor(eta, dtype=torch.float64, device="cuda", requires_grad=True)
        om = torch.tensor(omega, dtype=torch.float64, device="cuda", requires_grad=True)
        E = AG.energy(phi, Vt, et, om, ctx)
        (3.0 * E).backward()
    Ev = float(E.detach())
    assert abs(Ev - O.energy(po, phi_np)) <= 1e-12 * abs(Ev)
    d = O.energy_parameter_derivatives(po, phi_np)
    assert relmax(host(phi.grad), 3.0 * O.energy_gradient(po, phi_np)) < 1e-12
    assert relmax(host(Vt.grad), 3.0 * d["dV"]) < 1e-13
    assert abs(float(et.grad) - 3.0 * d["deta"]) <= 1e-12 * abs(3.0 * d["deta"])
    assert abs(float(om.grad) - 3.0 * d["domega"]) <= 1e-12 * abs(3.0 * d["domega"])


def test_autograd_ground_state_energy_hellmann_feynman(G, AG, gs_small):
    (n, L, eta, omega, V), ctx, phi = gs_small
    Vt = torch.from_numpy(V).cuda().requires_grad_(True)
    et = torch.tensor(eta, dtype=torch.float64, device="cuda", requires_grad=True)
    om = torch.tensor(omega, dtype=torch.float64, device="cuda", requires_grad=True)
    opts = ctx_opts(G)
    E, ph = AG.ground_state_energy(Vt, et, om, ctx, phi, opts)
    E.backward()
    po = O.Problem(n, L, eta, omega, V)
    d = O.energy_parameter_derivatives(po, host(ph))
    assert relmax(host(Vt.grad), d["dV"]) < 1e-12
    assert abs(float(et.grad) - d["deta"]) <= 1e-12 * abs(d["deta"])
    assert abs(float(om.grad) - d["domega"]) <= 1e-11 * max(abs(d["domega"]), 1e-6)
