"""The preconditioner variants of Section 5.4 (P_C, P_Delta, P_V, P_C1, P_C2,
none) and the Fletcher-Reeves rule on the GPU against the FP64 oracle.

Tolerances as for the default solver: FP64 per-iterate E_n rel 1e-12 and
phase-aligned phi_n relative L2 1e-9 over 20 iterations (fallbacks and
backtracks equal); mixed solves to the oracle's converged energy
(rel 1e-7) with ||r||_inf < 1e-8 re-evaluated by the oracle.  The derived
scalars beta_n and theta_n are checked to 1e-6 max(|beta_n|, 1) and
1e-6 max(|theta_n|, 1e-3): beta's numerator Re<r_n - r_{n-1}, P r_n> and
theta's numerator Re<H phi, q> both cancel (nearly equal consecutive
residuals; a residual nearly orthogonal to q near convergence), so their
rounding scales with ||r_n|| ||P r_n|| and ||H phi|| ||q||, not with the
scalar; with P_Delta the FP64 GPU and oracle values differ by up to 1.2e-7
while E_n agrees to 1e-12 and phi_20 to 1e-9.
"""
import numpy as np
import pytest

from oracle import gpe_oracle as O
from paper_1611_02045_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KINDS = {"C": 0, "Delta": 1, "V": 2, "C1": 3, "C2": 4, "none": 5}


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


def phase_aligned_rel_l2(a, b):
    z = np.vdot(a, b)
    return float(np.linalg.norm(a * (z / abs(z)) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precond,beta,use_graph", [(k, "PR", 1) for k in KINDS] + [("C", "FR", 1), ("C1", "FR", 2),
                                                                                    ("V", "PR", 2)])
def test_fp64_per_iterate_parity(G, precond, beta, use_graph):
    w = I.workload("c64_2d")
    po = O.Problem(w["n"], w["L"], w["eta"], w["omega"], w["V"])
    K = 20
    _, orep = O.pcg_solve(po, w["phi0"], O.SolveOptions(max_iter=K, precond=precond, beta=beta), keep_iterates=(K,))
    with G.Context(w["n"], w["L"], w["eta"], w["omega"], w["V"], prec=G.GPE_FP64) as ctx:
        phi = dev(w["phi0"])
        o = G.solve_opts_default()
        o.max_iter = K
        o.use_graph = use_graph
        o.precond = KINDS[precond]
        o.beta_rule = 1 if beta == "FR" else 0
        rep = ctx.pcg_solve(phi, o, log_cap=64)
    assert rep["iters"] == K and rep["loop_kind"] == use_graph, rep
    assert phase_aligned_rel_l2(host(phi), orep["iterates"][K]) < 1e-9
    log = rep["log"]
    for n_ in range(K + 1):
        e = orep["log"][n_]
        assert abs(log[n_, 2] - e["E"]) <= 1e-12 * abs(e["E"]), n_
        if n_ < K:
            assert abs(log[n_, 7] - e["beta"]) <= 1e-6 * max(abs(e["beta"]), 1.0), n_
            assert abs(log[n_, 8] - e["theta"]) <= 1e-6 * max(abs(e["theta"]), 1e-3), n_
            assert int(log[n_, 10]) == int(e["fallback"]) and int(log[n_, 11]) == e["backtracks"], n_


@pytest.mark.parametrize("precond", ["V", "Delta", "C2"])
def test_mixed_cluster_solve_with_variants(G, precond):
    """The complex64 phase in the cluster kernel (its own core pass) and the
    refinement, with a non-default preconditioner: converged E against the
    oracle's FP64 solve with the same preconditioner."""
    w = I.workload("c64_2d")
    po = O.Problem(w["n"], w["L"], w["eta"], w["omega"], w["V"])
    _, orep = O.pcg_solve(po, w["phi0"], O.SolveOptions(precond=precond, max_iter=20000))
    assert orep["status"] == "converged"
    with G.Context(w["n"], w["L"], w["eta"], w["omega"], w["V"], prec=G.GPE_MIXED) as ctx:
        phi = dev(w["phi0"])
        o = G.solve_opts_default()
        o.precond = KINDS[precond]
        rep = ctx.pcg_solve(phi, o)
    assert rep["status"] == G.GPE_OK and rep["loop_kind"] == 3, rep
    assert abs(rep["E"] - orep["E"]) <= 1e-7 * abs(orep["E"])
    ph = host(phi)
    lam = O.chemical_potential(po, ph)
    assert np.max(np.abs(O.apply_H(po, ph, ph) - lam * ph)) < 1e-8


def test_bad_variant_options_are_rejected(G):
    w = I.workload("c64_2d")
    with G.Context(w["n"], w["L"], w["eta"], w["omega"], w["V"], prec=G.GPE_FP64) as ctx:
        for field, val in (("precond", 6), ("precond", -1), ("beta_rule", 2)):
            o = G.solve_opts_default()
            setattr(o, field, val)
            with pytest.raises(G.GpeError):
                ctx.pcg_solve(dev(w["phi0"]), o)


@pytest.mark.parametrize("use_graph", [1, 2])
def test_exact_line_search_per_iterate_parity(G, use_graph):
    """GPE_LINE_EXACT (Newton on the exact step polynomial) against the oracle's
    "exact" line search: E_n, phi_20 and the discrete decisions."""
    w = I.workload("c64_2d")
    po = O.Problem(w["n"], w["L"], w["eta"], w["omega"], w["V"])
    K = 20
    _, orep = O.pcg_solve(po, w["phi0"], O.SolveOptions(max_iter=K, line_search="exact"), keep_iterates=(K,))
    with G.Context(w["n"], w["L"], w["eta"], w["omega"], w["V"], prec=G.GPE_FP64) as ctx:
        phi = dev(w["phi0"])
        o = G.solve_opts_default()
        o.max_iter = K
        o.use_graph = use_graph
        o.line_search = G.GPE_LINE_EXACT
        rep = ctx.pcg_solve(phi, o, log_cap=64)
    assert rep["iters"] == K and rep["loop_kind"] == use_graph
    assert phase_aligned_rel_l2(host(phi), orep["iterates"][K]) < 1e-9
    for n_ in range(K + 1):
        e = orep["log"][n_]
        assert abs(rep["log"][n_, 2] - e["E"]) <= 1e-12 * abs(e["E"]), n_
        if n_ < K:
            assert abs(rep["log"][n_, 8] - e["theta"]) <= 1e-6 * max(abs(e["theta"]), 1e-3), n_
            assert int(rep["log"][n_, 10]) == int(e["fallback"]) and int(rep["log"][n_, 11]) == e["backtracks"], n_


def test_exact_line_search_mixed_solve_converges(G):
    w = I.workload("c64_2d")
    po = O.Problem(w["n"], w["L"], w["eta"], w["omega"], w["V"])
    _, orep = O.pcg_solve(po, w["phi0"], O.SolveOptions())
    with G.Context(w["n"], w["L"], w["eta"], w["omega"], w["V"], prec=G.GPE_MIXED) as ctx:
        phi = dev(w["phi0"])
        o = G.solve_opts_default()
        o.line_search = G.GPE_LINE_EXACT
        rep = ctx.pcg_solve(phi, o)
    assert rep["status"] == G.GPE_OK
    assert abs(rep["E"] - orep["E"]) <= 1e-7 * abs(orep["E"])


@pytest.mark.parametrize("case", ["2d_quartic", "3d"])
def test_thomas_fermi_state_matches_oracle(G, case):
    """gpe_thomas_fermi (device bisection for mu, eq. TF_App) against the
    oracle's: mu to rel 1e-12, the state to 1e-12 of its maximum, unit norm;
    then a mixed solve from it converges and the oracle verifies the answer."""
    if case == "3d":
        n, L = (64, 64, 64), (8.0, 8.0, 8.0)
        V = I.harmonic(n, L, [1.0, 1.0, 2.0])
        eta, omega = 2000.0, 0.5
    else:
        n, L = (128, 128), (12.0, 12.0)
        V = I.harmonic_quartic(n, L, 0.05)
        eta, omega = 500.0, 0.6
    po = O.Problem(n, L, eta, omega, V)
    want, mu_o = O.thomas_fermi_state(po)
    with G.Context(n, L, eta, omega, V, prec=G.GPE_MIXED) as ctx:
        phi = torch.empty(want.shape, dtype=torch.complex128, device="cuda")
        mu = ctx.thomas_fermi(phi)
        got = host(phi)
        assert abs(mu - mu_o) <= 1e-12 * abs(mu_o)
        assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
        assert abs(O.norm(po, got) - 1.0) < 1e-12
        host_out = np.zeros(want.shape, dtype=np.complex128)
        assert ctx.thomas_fermi(host_out) == mu and np.array_equal(host_out, got)
        rep = ctx.pcg_solve(phi)
    assert rep["status"] == G.GPE_OK, rep
    ph = host(phi)
    lam = O.chemical_potential(po, ph)
    assert np.max(np.abs(O.apply_H(po, ph, ph) - lam * ph)) < 1e-8
