"""GPU (libgpe CUDA kernels, through the C ABI) against the FP64 CPU oracle on
identical seeded inputs.

Tolerances
  * complex128 operators: max|gpu - oracle| <= 1e-12 max|oracle| (FFT round-off
    in FP64 is ~ eps log2(M) ~ 1e-15 of the largest Fourier-space term, times
    the largest multiplier |k|^2/2 relative to the result's scale);
  * complex64 operators: 2e-5 relative (FP32 transforms: eps32 ~ 6e-8 times
    log2(M) and the same multiplier ratio);
  * FP64 solver: per-iterate E_n to rel 1e-12 and phase-aligned phi_n to
    relative L2 1e-9 over the first 20 iterations; converged E to rel 1e-10;
  * mixed solver: converged E to rel 1e-7 and ||r||_inf < 1e-8.
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


def dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.complex128)


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def phase_aligned_rel_l2(a, b):
    """min over global phases of ||a e^{i t} - b|| / ||b||."""
    z = np.vdot(a, b)
    a2 = a * (z / abs(z))
    return float(np.linalg.norm(a2 - b) / np.linalg.norm(b))


def make(n, L, eta, omega, V, prec, G):
    return G.Context(n, L, eta, omega, V, prec=prec)


GRIDS = [((8, 8), (2.0, 2.0)), ((16, 32), (3.0, 4.0)), ((64, 64), (8.0, 8.0)), ((256, 256), (16.0, 16.0)),
         ((8, 16, 8), (2.0, 2.0, 2.0)), ((32, 32, 32), (6.0, 6.0, 6.0)), ((16, 64, 32), (4.0, 6.0, 5.0)),
         ((128, 128, 128), (8.0, 8.0, 8.0)), ((512, 512), (16.0, 16.0))]


def _fields(n, L, smooth):
    if smooth:
        phi = I.phi_d(n, L, 0.6) if len(n) == 2 else I.normalise(
            I.anisotropic_gaussian(n, L, [1.0, 1.0, 2.0]) * (1 + 0.5 * I.mesh(n, L)[0]), n, L)
        f = phi * (1 + 0.05 * I.random_field(7, n, L))
    else:
        phi, f = I.random_field(1, n, L), I.random_field(2, n, L)
    return phi, f


@pytest.mark.parametrize("n,L", GRIDS)
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_apply_H_matches_oracle(G, n, L, prec):
    V = I.harmonic(n, L, [1.0, 1.0, 2.0][: len(n)])
    eta, om = 37.0, 0.7
    po = O.Problem(n, L, eta, om, V)
    for smooth in (False, True):
        phi, f = _fields(n, L, smooth)
        dt = torch.complex128 if prec == 0 else torch.complex64
        ph_d, f_d = dev(phi, dt), dev(f, dt)
        out = torch.empty_like(f_d)
        with make(n, L, eta, om, V, prec, G) as ctx:
            ctx.apply_H(ph_d, f_d, out)
            got = host(out)
        # oracle on exactly the values the GPU saw
        want = O.apply_H(po, host(ph_d), host(f_d))
        tol = 1e-12 if prec == 0 else 2e-5
        assert relmax(got, want) < tol, (smooth, relmax(got, want))


@pytest.mark.parametrize("M", [32, 64, 128, 256])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_apply_H_batch_cluster_matches_oracle(G, M, prec):
    """gpe_apply_H_batch (one thread-block cluster per field, fields in
    distributed shared memory) against the oracle, field by field, for f = phi
    and f != phi, and against gpe_apply_H."""
    n, L = (M, M), (7.0, 5.0)
    V = I.harmonic(n, L)
    eta, om = 29.0, 0.6
    po = O.Problem(n, L, eta, om, V)
    nb = 3
    dt = torch.complex128 if prec == 0 else torch.complex64
    phis = np.stack([I.random_field(10 + b, n, L) for b in range(nb)])
    fs = np.stack([I.random_field(20 + b, n, L) for b in range(nb)])
    phi_d, f_d = dev(phis, dt), dev(fs, dt)
    tol = 1e-12 if prec == 0 else 2e-5
    with make(n, L, eta, om, V, prec, G) as ctx:
        for same in (True, False):
            out = torch.full_like(phi_d, float("nan"))
            ctx.apply_H_batch(nb, phi_d, phi_d if same else f_d, out)
            got = host(out)
            ph, ff = host(phi_d), host(phi_d if same else f_d)
            for b in range(nb):
                want = O.apply_H(po, ph[b], ff[b])
                assert relmax(got[b], want) < tol, (same, b, relmax(got[b], want))
                one = torch.empty_like(phi_d[b])
                ctx.apply_H(phi_d[b], (phi_d if same else f_d)[b], one)
                assert relmax(got[b], host(one)) < tol


def test_apply_H_batch_rejects_unsupported_grids(G):
    n, L = (64, 32), (4.0, 4.0)
    with make(n, L, 1.0, 0.0, I.harmonic(n, L), 0, G) as ctx:
        x = dev(np.zeros((32, 64)))
        with pytest.raises(G.GpeError) as e:
            ctx.apply_H_batch(1, x, x, x)
        assert e.value.status == G.GPE_ERR_UNSUPPORTED


@pytest.mark.parametrize("n,L", GRIDS)
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_precond_matches_oracle(G, n, L, prec):
    V = I.harmonic(n, L)
    eta, om = 23.0, 0.4
    po = O.Problem(n, L, eta, om, V)
    phi, r = _fields(n, L, False)
    dt = torch.complex128 if prec == 0 else torch.complex64
    ph_d, r_d = dev(phi, dt), dev(r, dt)
    out = torch.empty_like(r_d)
    tol = 1e-12 if prec == 0 else 2e-5
    with make(n, L, eta, om, V, prec, G) as ctx:
        ctx.precond(ph_d, r_d, 1.3, out)
        assert relmax(host(out), O.precond_C(po, host(ph_d), host(r_d), 1.3)) < tol
        # alpha <= 0: the adaptive shift lambda~(phi) of eq. Opt_Alpha
        ctx.precond(ph_d, r_d, 0.0, out)
        a = O.lambda_tilde(po, host(ph_d))
        assert relmax(host(out), O.precond_C(po, host(ph_d), host(r_d), a)) < tol
        # out aliasing r
        ctx.precond(ph_d, r_d, 1.3, r_d)
        assert relmax(host(r_d), O.precond_C(po, host(ph_d), r.astype(host(ph_d).dtype), 1.3)) < tol * 10


@pytest.mark.parametrize("n,L", GRIDS)
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_energy_matches_oracle(G, n, L, prec):
    V = I.harmonic(n, L, [1.0, 1.0, 2.0][: len(n)])
    eta, om = 51.0, 0.8
    po = O.Problem(n, L, eta, om, V)
    phi, _ = _fields(n, L, True)
    dt = torch.complex128 if prec == 0 else torch.complex64
    ph_d = dev(phi, dt)
    with make(n, L, eta, om, V, prec, G) as ctx:
        e = ctx.energy(ph_d)
    ph = host(ph_d)
    w = O.energy_parts(po, ph)
    tol = 1e-12 if prec == 0 else 2e-6
    for k in ("kin", "pot", "int", "rot", "total"):
        assert abs(e[k] - w[k]) <= tol * (abs(w["total"]) + abs(w[k])), k
    assert abs(e["lam"] - O.chemical_potential(po, ph)) <= tol * abs(e["lam"])
    assert abs(e["lam_tilde"] - O.lambda_tilde(po, ph)) <= tol * abs(e["lam_tilde"])
    assert abs(e["norm2"] - O.norm(po, ph) ** 2) <= tol


def test_hermitian_and_vortex_eigenfunction_on_gpu(G):
    n, L = (64, 64), (8.0, 8.0)
    V = I.harmonic(n, L)
    b = I.normalise(I.phi_b(n, L), n, L)
    with make(n, L, 0.0, 0.3, V, 0, G) as ctx:
        out = torch.empty_like(dev(b))
        ctx.apply_H(dev(b), dev(b), out)
        assert np.max(np.abs(host(out) - 1.7 * b)) < 1e-11
        f, g, phi = (I.random_field(s, n, L) for s in (3, 4, 5))
        hf, hg = torch.empty_like(dev(f)), torch.empty_like(dev(f))
        ctx.apply_H(dev(phi), dev(f), hf)
        ctx.apply_H(dev(phi), dev(g), hg)
        a = np.vdot(g, host(hf))
        c = np.conj(np.vdot(f, host(hg)))
        assert abs(a - c) < 1e-12 * abs(a)


@pytest.mark.parametrize("case", ["2d", "3d"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_linear_trap_ground_state_closed_form(G, case, prec):
    """Degenerate case with a closed form, independent of the oracle: eta = 0
    in the trap V = 1/2 sum gamma_i^2 x_i^2 has the Gaussian ground state with
    E = sum gamma_i / 2, and rotation below the trap frequency (omega < 1 about
    z with gamma_x = gamma_y = 1) leaves it the ground state (its L_z value is
    0; the states L_z = m cost m (1 - omega) more).  From a perturbed,
    off-centre start the solver must reach E = d/2 (2D: 1; 3D with gamma =
    (1, 1, 2): 2) to the tolerance of its precision."""
    if case == "2d":
        n, L, gam = (64, 64), (8.0, 8.0), [1.0, 1.0]
    else:
        n, L, gam = (32, 32, 32), (6.0, 6.0, 6.0), [1.0, 1.0, 2.0]
    V = I.harmonic(n, L, gam)
    m = I.mesh(n, L)
    start = np.exp(-0.5 * sum(((x - 0.7) / 1.3) ** 2 for x in m)).astype(np.complex128) * (1.0 + 0.3 * (m[0] + 1j * m[1]))
    phi0 = I.perturbed(start, 11, n, L, amp=1e-2)
    E_exact = 0.5 * sum(gam)
    with make(n, L, 0.0, 0.5, V, G.GPE_FP64 if prec == "fp64" else G.GPE_MIXED, G) as ctx:
        phi = dev(phi0)
        rep = ctx.pcg_solve(phi)
    assert rep["status"] == G.GPE_OK, rep
    tol = 1e-11 if prec == "fp64" else 1e-7
    assert abs(rep["E"] - E_exact) <= tol * E_exact, (rep["E"], E_exact)
    assert abs(rep["lam"] - E_exact) <= 1e-6 * E_exact  # eta = 0: lambda = E


# ------------------------------------------------------------------ solver
def _workload_problem(name):
    w = I.workload(name)
    return w, O.Problem(w["n"], w["L"], w["eta"], w["omega"], w["V"])


@pytest.mark.parametrize("use_graph", [2, 1, 0], ids=["persistent", "graph", "hostloop"])
def test_pcg_per_iterate_parity_fp64(G, use_graph):
    """Same seeded phi_0, FP64: E_n (rel 1e-12) and phi_n (phase-aligned L2 1e-9)
    over the first 20 iterations; beta_n, theta_n and the discrete decisions agree."""
    w, po = _workload_problem("c64_2d")
    K = 20
    ophi, orep = O.pcg_solve(po, w["phi0"], O.SolveOptions(max_iter=K), keep_iterates=tuple(range(K + 1)))
    with make(w["n"], w["L"], w["eta"], w["omega"], w["V"], 0, G) as ctx:
        for k in (1, 2, 5, 10, K):
            phi = dev(w["phi0"])
            o = G.solve_opts_default()
            o.max_iter = k
            o.use_graph = use_graph
            rep = ctx.pcg_solve(phi, o, log_cap=64)
            assert rep["loop_kind"] == use_graph, rep["note"]
            assert rep["iters"] == k and rep["status"] == G.GPE_ERR_NOT_CONVERGED
            assert phase_aligned_rel_l2(host(phi), orep["iterates"][k]) < 1e-9, k
        log = rep["log"]
    assert log.shape[0] == K + 1
    for n_ in range(K + 1):
        e = orep["log"][n_]
        assert abs(log[n_, 2] - e["E"]) <= 1e-12 * abs(e["E"]), n_
        assert abs(log[n_, 3] - e["lam"]) <= 1e-12 * abs(e["lam"]), n_
        # r = H phi - lambda phi carries absolute FP64 noise ~ eps |lambda| max|phi|
        assert abs(log[n_, 4] - e["res_inf"]) <= 1e-9 * e["res_inf"] + 1e-13 * abs(e["lam"]), n_
        if n_ < K:
            assert abs(log[n_, 6] - e["alpha"]) <= 1e-12 * abs(e["alpha"])
            assert abs(log[n_, 7] - e["beta"]) <= 1e-8 * max(abs(e["beta"]), 1e-3)
            assert abs(log[n_, 8] - e["theta"]) <= 1e-8 * abs(e["theta"])
            assert int(log[n_, 10]) == int(e["fallback"]) and int(log[n_, 11]) == e["backtracks"]


def test_pcg_converged_fp64_matches_oracle(G):
    w, po = _workload_problem("c64_2d")
    ophi, orep = O.pcg_solve(po, w["phi0"], O.SolveOptions())
    assert orep["status"] == "converged"
    with make(w["n"], w["L"], w["eta"], w["omega"], w["V"], 0, G) as ctx:
        phi = dev(w["phi0"])
        rep = ctx.pcg_solve(phi, check=True)
    assert rep["status"] == G.GPE_OK and rep["res_inf"] < 1e-8
    assert abs(rep["E"] - orep["E"]) <= 1e-10 * abs(orep["E"])
    # the oracle's own residual of the GPU's answer
    ph = host(phi)
    r = O.apply_H(po, ph, ph) - O.chemical_potential(po, ph) * ph
    assert np.max(np.abs(r)) < 1.01e-8
    assert abs(O.energy(po, ph) - rep["E"]) <= 1e-12 * abs(rep["E"])


def test_pcg_mixed_refinement_reaches_fp64_answer(G):
    w, po = _workload_problem("c64_2d")
    ophi, orep = O.pcg_solve(po, w["phi0"], O.SolveOptions())
    with make(w["n"], w["L"], w["eta"], w["omega"], w["V"], 1, G) as ctx:
        phi = dev(w["phi0"])
        rep = ctx.pcg_solve(phi, check=True, log_cap=4096)
    assert rep["status"] == G.GPE_OK and rep["res_inf"] < 1e-8
    assert rep["iters_lo"] > 0 and rep["iters"] > rep["iters_lo"]
    assert abs(rep["E"] - orep["E"]) <= 1e-7 * abs(orep["E"])
    ph = host(phi)
    r = O.apply_H(po, ph, ph) - O.chemical_potential(po, ph) * ph
    assert np.max(np.abs(r)) < 1.01e-8


def test_pcg_3d_per_iterate_and_converged(G):
    n, L = (32, 32, 32), (6.0, 6.0, 6.0)
    V = I.harmonic(n, L, [1.0, 1.0, 2.0])
    eta, om = 100.0, 0.5
    po = O.Problem(n, L, eta, om, V)
    m = I.mesh(n, L)
    phi0 = I.perturbed(I.normalise(I.anisotropic_gaussian(n, L, [1.0, 1.0, 2.0]) * (0.5 + 0.5 * (m[0] + 1j * m[1])), n, L), 4, n, L)
    K = 10
    _, orep = O.pcg_solve(po, phi0, O.SolveOptions(max_iter=K), keep_iterates=(K,))
    with make(n, L, eta, om, V, 0, G) as ctx:
        phi = dev(phi0)
        o = G.solve_opts_default()
        o.max_iter = K
        rep = ctx.pcg_solve(phi, o, log_cap=32)
        for n_ in range(K + 1):
            assert abs(rep["log"][n_, 2] - orep["log"][n_]["E"]) <= 1e-12 * abs(orep["log"][n_]["E"])
        assert phase_aligned_rel_l2(host(phi), orep["iterates"][K]) < 1e-9
        phi = dev(phi0)
        rep = ctx.pcg_solve(phi, check=True)
    _, oconv = O.pcg_solve(po, phi0, O.SolveOptions())
    assert abs(rep["E"] - oconv["E"]) <= 1e-10 * abs(oconv["E"])


@pytest.mark.parametrize("use_graph", [2, 1], ids=["persistent", "graph"])
def test_pcg_3d_per_iterate_64cube(G, use_graph):
    """64^3 (the persistent kernel's 3D path) against the oracle for 8 iterations."""
    n, L = (64, 64, 64), (8.0, 8.0, 8.0)
    V = I.harmonic(n, L, [1.0, 1.0, 2.0])
    eta, om = 500.0, 0.6
    po = O.Problem(n, L, eta, om, V)
    m = I.mesh(n, L)
    phi0 = I.perturbed(I.normalise(I.anisotropic_gaussian(n, L, [1.0, 1.0, 2.0]) * (0.4 + 0.6 * (m[0] + 1j * m[1])), n, L), 9, n, L)
    K = 8
    _, orep = O.pcg_solve(po, phi0, O.SolveOptions(max_iter=K), keep_iterates=(K,))
    with make(n, L, eta, om, V, 0, G) as ctx:
        phi = dev(phi0)
        o = G.solve_opts_default()
        o.max_iter = K
        o.use_graph = use_graph
        rep = ctx.pcg_solve(phi, o, log_cap=16)
        assert rep["loop_kind"] == use_graph, rep["note"]
    for n_ in range(K + 1):
        assert abs(rep["log"][n_, 2] - orep["log"][n_]["E"]) <= 1e-12 * abs(orep["log"][n_]["E"])
    assert phase_aligned_rel_l2(host(phi), orep["iterates"][K]) < 1e-9


@pytest.mark.parametrize("refine_restart", [1, 0])
def test_pcg_mixed_loop_styles_agree(G, refine_restart):
    """The persistent kernel and the graph loop run the same algorithm (their
    reductions sum in different fixed orders): both reach the same ground state."""
    w, po = _workload_problem("c64_2d")
    res = {}
    with make(w["n"], w["L"], w["eta"], w["omega"], w["V"], 1, G) as ctx:
        for ug in (2, 1):
            phi = dev(w["phi0"])
            o = G.solve_opts_default()
            o.use_graph = ug
            o.refine_restart = refine_restart
            res[ug] = ctx.pcg_solve(phi, o, check=True)
            assert res[ug]["loop_kind"] == ug, res[ug]["note"]
    assert res[2]["res_inf"] < 1e-8 and res[1]["res_inf"] < 1e-8
    assert abs(res[2]["E"] - res[1]["E"]) <= 1e-10 * abs(res[1]["E"])
    assert res[2]["iters_lo"] > 0 and res[1]["iters_lo"] > 0


@pytest.mark.parametrize("name", ["c64_2d", "fast256_2d"])
def test_cluster_complex64_phase_iterates(G, name):
    """use_graph = 3: the complex64 phase in one thread-block cluster's shared
    memory.  Its first 15 iterates against the FP64 oracle at complex64
    tolerance (E_n rel 2e-6, phi_n phase-aligned L2 2e-4), and against the same
    phase run by the graph loop."""
    w, po = _workload_problem(name)
    K = 15
    _, orep = O.pcg_solve(po, w["phi0"], O.SolveOptions(max_iter=K), keep_iterates=(K,))
    logs, phis = {}, {}
    with make(w["n"], w["L"], w["eta"], w["omega"], w["V"], 1, G) as ctx:
        for ug in (3, 1):
            phi = dev(w["phi0"])
            o = G.solve_opts_default()
            o.use_graph = ug
            o.max_iter = K
            o.switch_res = 1e-30
            o.stall_window = 1 << 30
            rep = ctx.pcg_solve(phi, o, log_cap=32)
            assert rep["loop_kind"] == ug, rep["note"]
            assert rep["iters"] == K and rep["iters_lo"] == K
            logs[ug], phis[ug] = rep["log"], host(phi)
    for n_ in range(K + 1):
        e = orep["log"][n_]["E"]
        assert abs(logs[3][n_, 2] - e) <= 2e-6 * abs(e), n_
        assert abs(logs[3][n_, 2] - logs[1][n_, 2]) <= 2e-6 * abs(e), n_
    assert phase_aligned_rel_l2(phis[3], orep["iterates"][K]) < 2e-4
    assert phase_aligned_rel_l2(phis[3], phis[1]) < 2e-4


@pytest.mark.parametrize("name", ["c64_2d", "fast256_2d"])
def test_cluster_mixed_solve_reaches_fp64_answer(G, name):
    w, po = _workload_problem(name)
    with make(w["n"], w["L"], w["eta"], w["omega"], w["V"], 1, G) as ctx:
        phi = dev(w["phi0"])
        o = G.solve_opts_default()
        o.use_graph = 3
        rep = ctx.pcg_solve(phi, o, check=True)
        assert rep["loop_kind"] == 3, rep["note"]
        ref = dev(w["phi0"])
        rep1 = ctx.pcg_solve(ref, check=True)
    assert rep["res_inf"] < 1e-8 and rep["iters_lo"] > 0
    assert abs(rep["E"] - rep1["E"]) <= 1e-10 * abs(rep1["E"])
    ph = host(phi)
    r = O.apply_H(po, ph, ph) - O.chemical_potential(po, ph) * ph
    # the stop rule, and the device's own residual reproduced by the oracle
    assert np.max(np.abs(r)) < 1e-8
    assert abs(np.max(np.abs(r)) - rep["res_inf"]) < 1e-11


def test_pcg_host_buffers_and_restart_from_solution(G):
    w, po = _workload_problem("c64_2d")
    with make(w["n"], w["L"], w["eta"], w["omega"], w["V"], 0, G) as ctx:
        phi = np.ascontiguousarray(w["phi0"].copy())
        rep = ctx.pcg_solve(phi, check=True)
        assert rep["res_inf"] < 1e-8
        rep2 = ctx.pcg_solve(phi, check=True)  # resume from the converged state
        assert rep2["iters"] == 0 and abs(rep2["E"] - rep["E"]) <= 1e-13 * abs(rep["E"])


def test_pcg_error_statuses(G):
    n, L = (16, 16), (4.0, 4.0)
    V = I.harmonic(n, L)
    with make(n, L, 10.0, 0.3, V, 0, G) as ctx:
        phi = dev(I.phi_a(n, L))
        o = G.solve_opts_default()
        o.max_iter = 3
        rep = ctx.pcg_solve(phi, o)
        assert rep["status"] == G.GPE_ERR_NOT_CONVERGED and rep["iters"] == 3
        bad = I.phi_a(n, L)
        bad[3, 4] = np.nan
        rep = ctx.pcg_solve(dev(bad))
        assert rep["status"] == G.GPE_ERR_NONFINITE
        # the context stays usable after a failed solve
        rep = ctx.pcg_solve(dev(I.phi_a(n, L)), check=True)
        assert rep["status"] == G.GPE_OK
    Vneg = V - 1e6  # alpha + V + eta|phi|^2 < 0 somewhere: P_V undefined
    with make(n, L, 10.0, 0.3, Vneg, 0, G) as ctx:
        rep = ctx.pcg_solve(dev(I.phi_a(n, L)))
        assert rep["status"] == G.GPE_ERR_PRECOND


# ----------------------------------------------------- full-size workloads
@pytest.mark.parametrize("name", ["fast256_2d", "rot128_3d"])
def test_full_size_mixed_solve_verified_by_oracle(G, name):
    """The workloads the benchmark times, in its configuration (mixed precision,
    graph loop): the oracle evaluates the returned state's energy and residual."""
    w, po = _workload_problem(name)
    with make(w["n"], w["L"], w["eta"], w["omega"], w["V"], 1, G) as ctx:
        phi = dev(w["phi0"])
        rep = ctx.pcg_solve(phi, check=True)
    assert rep["status"] == G.GPE_OK and rep["res_inf"] < 1e-8
    want = 3 if len(w["n"]) == 2 else 1  # the loops bench.py times (cluster for 2D, graph for 3D)
    assert rep["loop_kind"] == want, rep["note"]
    ph = host(phi)
    lam = O.chemical_potential(po, ph)
    res = np.max(np.abs(O.apply_H(po, ph, ph) - lam * ph))
    assert res < 1e-8
    assert abs(res - rep["res_inf"]) < 1e-11
    assert abs(O.energy(po, ph) - rep["E"]) <= 1e-12 * abs(rep["E"])
    assert abs(O.norm(po, ph) - 1.0) < 1e-12


def test_persistent_barrier_wait_gives_up_and_the_context_survives(G):
    """The persistent loop's grid barriers spin with a bound: with the bound set
    to one poll (wait_polls = 1), a block that reaches a barrier before the
    others gives up at once, every block leaves the loop, and the solve returns
    GPE_ERR_TIMEOUT; the same context then solves normally (persistent loop,
    default bound) and matches the oracle."""
    n, L = (256, 256), (8.0, 8.0)
    eta, om = 50.0, 0.3
    V = I.harmonic(n, L)
    phi0 = I.perturbed(I.phi_a(n, L), 9, n, L)
    with make(n, L, eta, om, V, 0, G) as ctx:
        o = G.solve_opts_default()
        o.use_graph = 2
        o.wait_polls = 1
        rep = ctx.pcg_solve(dev(phi0), o)
        assert rep["status"] == G.GPE_ERR_TIMEOUT, rep
        assert rep["loop_kind"] == 2, rep["note"]
        o.wait_polls = 0
        phi = dev(phi0)
        rep = ctx.pcg_solve(phi, o, check=True)
        assert rep["status"] == G.GPE_OK and rep["loop_kind"] == 2
    po = O.Problem(n, L, eta, om, V)
    _, orep = O.pcg_solve(po, phi0, O.SolveOptions(tol_res_inf=1e-8))
    assert abs(rep["E"] - orep["E"]) <= 1e-10 * abs(orep["E"])
