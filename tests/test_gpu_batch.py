"""Batched solves (gpe_batch_*) on the GPU: every instance of a heterogeneous
batch, solved inside one graph launch, must reproduce the single-instance
gpe_pcg_solve of the same problem from the same initial guess -- the same
kernels in the same order -- to the last bit of E and of the iteration count;
the single-instance solver is itself checked against the oracle elsewhere.
The batch's states are also re-evaluated by the oracle (energy, residual).
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.complex128)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def _instances(G):
    """Every branch kind: cluster complex64 phase (64^2, 128^2), loop-node
    complex64 phase (64 x 128, not square), FP64 (32^2), quartic trap."""
    out = []
    specs = [((64, 64), (8.0, 8.0), 100.0, 0.5, 0.0, G.GPE_MIXED, 1),
             ((128, 128), (10.0, 10.0), 250.0, 0.7, 0.05, G.GPE_MIXED, 2),
             ((64, 128), (8.0, 10.0), 60.0, 0.3, 0.0, G.GPE_MIXED, 3),
             ((32, 32), (6.0, 6.0), 30.0, 0.4, 0.0, G.GPE_FP64, 4),
             ((64, 64), (8.0, 8.0), 500.0, 0.85, 0.05, G.GPE_MIXED, 5)]
    for n, L, eta, omega, kappa, prec, seed in specs:
        V = I.harmonic_quartic(n, L, kappa)
        phi0 = I.perturbed(I.phi_d(n, L, omega), seed, n, L)
        out.append(dict(n=n, L=L, eta=eta, omega=omega, V=V, prec=prec, phi0=phi0))
    return out


def _single(G, w, opts):
    with G.Context(w["n"], w["L"], w["eta"], w["omega"], w["V"], prec=w["prec"]) as ctx:
        phi = dev(w["phi0"])
        rep = ctx.pcg_solve(phi, opts)
    return host(phi), rep


def test_batch_reproduces_single_instance_solves(G):
    ws = _instances(G)
    opts = G.solve_opts_default()
    with G.Batch(ws) as B:
        phis = [dev(w["phi0"]) for w in ws]
        s, reps = B.solve(phis, opts)
        assert s == G.GPE_OK, reps
        # a second launch of the same graph from the same inputs
        phis2 = [dev(w["phi0"]) for w in ws]
        s2, reps2 = B.solve(phis2, opts)
    for i, w in enumerate(ws):
        ph1, r1 = _single(G, w, opts)
        rb = reps[i]
        assert rb["status"] == G.GPE_OK and r1["status"] == G.GPE_OK
        assert rb["iters"] == r1["iters"] and rb["iters_lo"] == r1["iters_lo"], (i, rb, r1)
        assert rb["iters_fp64"] == r1["iters_fp64"], (i, rb, r1)
        assert rb["E"] == r1["E"] and rb["res_inf"] == r1["res_inf"], (i, rb, r1)
        assert np.array_equal(host(phis[i]), ph1)
        assert reps2[i]["E"] == rb["E"] and np.array_equal(host(phis2[i]), ph1)
        want_loop = 3 if (w["prec"] == G.GPE_MIXED and w["n"][0] == w["n"][1]) else 1
        assert rb["loop_kind"] == want_loop
        po = O.Problem(w["n"], w["L"], w["eta"], w["omega"], w["V"])
        ph = ph1.astype(np.complex128)
        lam = O.chemical_potential(po, ph)
        assert np.max(np.abs(O.apply_H(po, ph, ph) - lam * ph)) < 1e-8
        assert abs(O.energy(po, ph) - rb["E"]) <= 1e-12 * abs(rb["E"])


def test_stalled_refinement_is_completed_in_fp64(G):
    """Instance 1 (quartic trap, omega 0.7) has a nearly flat energy direction:
    the refinement's single-precision step moments stall near ||r|| ~ 1e-7 and
    the FP64 completion phase must take over and converge."""
    w = _instances(G)[1]
    ph, rep = _single(G, w, G.solve_opts_default())
    assert rep["status"] == G.GPE_OK and rep["iters_fp64"] > 0, rep
    po = O.Problem(w["n"], w["L"], w["eta"], w["omega"], w["V"])
    lam = O.chemical_potential(po, ph)
    assert np.max(np.abs(O.apply_H(po, ph, ph) - lam * ph)) < 1e-8


def test_batch_with_3d_instances(G):
    """3D instances (complex64 phase as a loop node over the 3D pass kernels)
    next to a 2D one: each reproduces its single-instance solve."""
    specs = []
    for n, L, eta, om, seed in [((32, 32, 32), (6.0, 6.0, 6.0), 200.0, 0.4, 7),
                                ((16, 32, 16), (5.0, 6.0, 5.0), 50.0, 0.2, 8),
                                ((64, 64), (8.0, 8.0), 100.0, 0.5, 9)]:
        V = I.harmonic(n, L, [1.0, 1.0, 2.0][: len(n)])
        G0 = I.anisotropic_gaussian(n, L, [1.0, 1.0, 2.0][: len(n)])
        phi0 = I.perturbed(I.normalise(G0 * (1 + 0.5j * I.mesh(n, L)[0]), n, L), seed, n, L)
        specs.append(dict(n=n, L=L, eta=eta, omega=om, V=V, prec=G.GPE_MIXED, phi0=phi0))
    opts = G.solve_opts_default()
    with G.Batch(specs) as B:
        phis = [dev(w["phi0"]) for w in specs]
        s, reps = B.solve(phis, opts)
    assert s == G.GPE_OK, reps
    for i, w in enumerate(specs):
        ph1, r1 = _single(G, w, opts)
        assert reps[i]["iters"] == r1["iters"] and reps[i]["E"] == r1["E"], (i, reps[i], r1)
        assert np.array_equal(host(phis[i]), ph1)
        assert reps[i]["loop_kind"] == (3 if len(w["n"]) == 2 else 1)


def test_batch_reports_each_instance_status(G):
    """A non-finite initial guess fails its own instance only; the others
    converge and the batch returns the failing status."""
    ws = _instances(G)[:3]
    bad = ws[1]["phi0"].copy()
    bad[3, 5] = np.nan
    phis = [dev(ws[0]["phi0"]), dev(bad), dev(ws[2]["phi0"])]
    with G.Batch(ws) as B:
        s, reps = B.solve(phis, G.solve_opts_default())
    assert s == G.GPE_ERR_NONFINITE
    assert [r["status"] for r in reps] == [G.GPE_OK, G.GPE_ERR_NONFINITE, G.GPE_OK]
    assert np.isnan(host(phis[1])[3, 5])  # the failed instance keeps its input


def test_batch_iteration_cap(G):
    ws = _instances(G)[:2]
    opts = G.solve_opts_default()
    opts.max_iter = 25
    with G.Batch(ws) as B:
        s, reps = B.solve([dev(w["phi0"]) for w in ws], opts)
    assert s == G.GPE_ERR_NOT_CONVERGED
    assert all(r["status"] == G.GPE_ERR_NOT_CONVERGED and r["iters"] == 25 for r in reps)
