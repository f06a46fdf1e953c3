"""The differentiation workload at its full configuration: 16 independent 2D
ground states at 256^2 (eta = 500, omega = 0.7, V = r^2/2 + 0.1 S_i with S_i
seeded smooth bumps) solved together in one batched graph launch
(gpe_batch_solve, mixed precision), then per instance the Hellmann-Feynman
derivatives dE*/dV = h^d |phi*|^2, dE*/deta = 1/2 int |phi*|^4,
dE*/domega = -<phi*, L_z phi*> (gpe_energy_grad) and the gradient of the
density loss int (|phi*|^2 - rho_t)^2 with respect to V through the
tangent-space adjoint solve (gpe_density_adjoint; Section 2: Hessian and
tangent projector).

Tolerances as in test_gpu_grad: fixed-phi derivatives against the oracle at
the same state rel 1e-12; the adjoint gradient against the oracle's rel 1e-8
(both solves stop at ||r|| <= 1e-12 ||P rhs||); Hellmann-Feynman against
central differences (h = 1e-6) of FP64 re-solves rel 1e-5.
"""
import numpy as np
import pytest

from oracle import gpe_oracle as O
from paper_1611_02045_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

COUNT = 16


@pytest.fixture(scope="module")
def G(built_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_02045_gb300 import gpe
    return gpe


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def target_density(n, L):
    return np.abs(I.normalise(I.anisotropic_gaussian(n, L, [0.05, 0.04]), n, L)) ** 2


@pytest.fixture(scope="module")
def solved(G):
    """The 16 instances solved in one batched launch; per-instance derivatives."""
    ws = [I.workload("grad256_2d", i) for i in range(COUNT)]
    specs = [dict(n=w["n"], L=w["L"], eta=w["eta"], omega=w["omega"], V=w["V"], prec=G.GPE_MIXED) for w in ws]
    phis = [torch.from_numpy(w["phi0"].copy()).cuda() for w in ws]
    with G.Batch(specs) as B:
        status, reps = B.solve(phis)
    assert status == G.GPE_OK, reps
    n, L = ws[0]["n"], ws[0]["L"]
    rho_t = target_density(n, L)
    wt = I.weight(n, L)
    out = []
    with G.Context(n, L, ws[0]["eta"], ws[0]["omega"], ws[0]["V"], prec=G.GPE_FP64) as ctx:
        for w, phi in zip(ws, phis):
            ctx.set_problem(w["V"], w["eta"], w["omega"])
            gV = torch.empty(phi.shape, dtype=torch.float64, device="cuda")
            d = ctx.energy_grad(phi, None, gV)
            g_rho = torch.from_numpy(2.0 * wt * (np.abs(host(phi)) ** 2 - rho_t)).cuda()
            gL = torch.empty(phi.shape, dtype=torch.float64, device="cuda")
            a = ctx.density_adjoint(phi, g_rho, gL, tol=1e-12, max_iter=3000)
            out.append(dict(w=w, phi=phi, d=d, gV=host(gV), gL=host(gL), adj=a))
    return reps, out, rho_t


def test_batch_solves_every_instance(G, solved):
    reps, out, _ = solved
    assert len(reps) == COUNT
    for r in reps:
        assert r["status"] == G.GPE_OK and r["res_inf"] < 1e-8, r
    # the instances are different problems: sixteen different energies
    Es = sorted(r["E"] for r in reps)
    assert all(b - a > 1e-9 for a, b in zip(Es, Es[1:]))


@pytest.mark.parametrize("index", [0, 7, 15])
def test_hellmann_feynman_and_density_adjoint_match_oracle(G, solved, index):
    reps, out, rho_t = solved
    o = out[index]
    w = o["w"]
    po = O.Problem(w["n"], w["L"], w["eta"], w["omega"], w["V"])
    ph = host(o["phi"]).astype(np.complex128)
    # the state the batch returned is a ground state in the oracle's eyes
    lam = O.chemical_potential(po, ph)
    assert np.max(np.abs(O.apply_H(po, ph, ph) - lam * ph)) < 1e-8
    d = O.energy_parameter_derivatives(po, ph)
    assert relmax(o["gV"], d["dV"]) < 1e-12
    assert abs(o["d"]["dE_deta"] - d["deta"]) <= 1e-12 * abs(d["deta"])
    assert abs(o["d"]["dE_domega"] - d["domega"]) <= 1e-12 * abs(d["domega"])
    assert abs(o["d"]["E"] - reps[index]["E"]) <= 1e-10 * abs(reps[index]["E"])
    want, _, res = O.density_loss_gradient_V(po, ph, rho_t)
    assert o["adj"]["rel_res"] <= 1e-12 and res <= 1e-12
    assert relmax(o["gL"], want) < 1e-8


def test_hellmann_feynman_matches_differences_of_fp64_solves(G, solved):
    """Instance 5: the batch's state polished in FP64 (||r||_inf < 1e-11), then
    dE*/deta, dE*/domega and dE*/dV along a smooth direction against central
    differences of re-solved ground-state energies (h = 1e-6, warm start)."""
    _, out, _ = solved
    o = out[5]
    w = o["w"]
    opts = G.solve_opts_default()
    opts.tol_res_inf = 1e-11
    with G.Context(w["n"], w["L"], w["eta"], w["omega"], w["V"], prec=G.GPE_FP64) as ctx:
        phi = o["phi"].clone()
        ctx.pcg_solve(phi, opts, check=True)
        gV = torch.empty(phi.shape, dtype=torch.float64, device="cuda")
        an = ctx.energy_grad(phi, None, gV)

        def E_at(eta=None, omega=None, V=None):
            ctx.set_problem(w["V"] if V is None else V, w["eta"] if eta is None else eta,
                            w["omega"] if omega is None else omega)
            p = phi.clone()
            return ctx.pcg_solve(p, opts, check=True)["E"]

        h = 1e-6
        fd = (E_at(eta=w["eta"] + h) - E_at(eta=w["eta"] - h)) / (2 * h)
        assert abs(fd - an["dE_deta"]) <= 1e-5 * abs(an["dE_deta"]), (fd, an)
        fd = (E_at(omega=w["omega"] + h) - E_at(omega=w["omega"] - h)) / (2 * h)
        assert abs(fd - an["dE_domega"]) <= 1e-5 * abs(an["dE_domega"]), (fd, an)
        S = I.smooth_bumps(w["n"], w["L"], 123)
        fd = (E_at(V=w["V"] + h * S) - E_at(V=w["V"] - h * S)) / (2 * h)
        dv = float(np.sum(host(gV) * S))
        assert abs(fd - dv) <= 1e-5 * abs(dv), (fd, dv)
