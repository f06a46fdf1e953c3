"""Plans of the pass kernels (values per thread E, block / tile width) and the
tuner (gpe_set_plan, gpe_autotune) on the GPU, against the FP64 CPU oracle.

A plan only changes how lines are split over threads and blocks (and so the
order of floating-point sums), so every plan must meet the same tolerances as
the default one: operators rel 1e-12 (complex128) / 2e-5 (complex64), FP64
per-iterate E_n rel 1e-12 and phase-aligned phi_n L2 1e-9 over 20 iterations,
mixed solves E rel 1e-7 of the oracle's FP64 answer with ||r||_inf < 1e-8.
"""
import numpy as np
import pytest

from oracle import gpe_oracle as O
from paper_1611_02045_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MODE_C64, MODE_FP64, MODE_REFINE = 0, 1, 2


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
    return t.detach().cpu().numpy()


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def phase_aligned_rel_l2(a, b):
    z = np.vdot(a, b)
    return float(np.linalg.norm(a * (z / abs(z)) - b) / np.linalg.norm(b))


def widths(n, axis, E, max_threads):
    """Every power-of-two width the kernels accept for this axis (as gpe_set_plan)."""
    M = n[axis]
    Tl = M // E
    out, w = [], 1
    lines = int(np.prod(n[1:]))
    while Tl * w <= max_threads and w <= (lines if axis == 0 else n[0]):
        out.append(w)
        w *= 2
    return out


PLAN_GRIDS = [((64, 64), (8.0, 8.0)), ((32, 128), (4.0, 10.0)), ((256, 256), (16.0, 16.0)),
              ((32, 64, 32), (5.0, 6.0, 5.0)), ((512, 512), (16.0, 16.0))]


@pytest.mark.parametrize("n,L", PLAN_GRIDS)
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_operators_match_oracle_under_every_E(G, n, L, prec):
    """apply_H and P_C with E = 4 and E = 8 on every axis, at the smallest,
    a middle and the largest width each axis accepts."""
    V = I.harmonic(n, L, [1.0, 1.0, 2.0][: len(n)])
    eta, om = 37.0, 0.7
    po = O.Problem(n, L, eta, om, V)
    mode, cap = (MODE_FP64, 256) if prec == 0 else (MODE_C64, 512)
    dt = torch.complex128 if prec == 0 else torch.complex64
    tol = 1e-12 if prec == 0 else 2e-5
    phi, f = I.random_field(1, n, L), I.random_field(2, n, L)
    ph_d, f_d = dev(phi, dt), dev(f, dt)
    out = torch.empty_like(f_d)
    want_H = O.apply_H(po, host(ph_d), host(f_d))
    want_P = O.precond_C(po, host(ph_d), host(f_d), 1.3)
    with G.Context(n, L, eta, om, V, prec=prec) as ctx:
        for E in (8, 4):
            ws = [widths(n, ax, E, cap) for ax in range(len(n))]
            for pick in (0, len(ws[0]) // 2, -1):
                for ax in range(len(n)):
                    ctx.set_plan(mode, ax, E, ws[ax][min(pick, len(ws[ax]) - 1) if pick >= 0 else -1])
                    assert ctx.get_plan(mode, ax)[0] == E
                ctx.apply_H(ph_d, f_d, out)
                assert relmax(host(out), want_H) < tol, (E, pick)
                ctx.precond(ph_d, f_d, 1.3, out)
                assert relmax(host(out), want_P) < tol, (E, pick)


def test_set_plan_rejects_what_the_kernels_cannot_run(G):
    n, L = (16, 64), (4.0, 8.0)
    with G.Context(n, L, 10.0, 0.3, I.harmonic(n, L), prec=G.GPE_FP64) as ctx:
        for mode, axis, E, w in [(MODE_FP64, 0, 4, 1),      # E = 4 needs M >= 32 (nx = 16)
                                 (MODE_FP64, 1, 8, 3),      # width not a power of two
                                 (MODE_FP64, 1, 8, 64),     # 8 * 64 threads > 256
                                 (MODE_FP64, 2, 8, 1),      # no z axis in 2D
                                 (MODE_FP64, 0, 6, 1),      # E not 4 or 8
                                 (MODE_C64, 0, 8, 1)]:      # no complex64 buffers in an FP64 context
            with pytest.raises(G.GpeError):
                ctx.set_plan(mode, axis, E, w)
        ctx.set_plan(MODE_FP64, 1, 4, 8)
        assert ctx.get_plan(MODE_FP64, 1) == (4, 8)


def test_fp64_per_iterate_parity_with_E4_plans(G):
    """The FP64 solver with E = 4 on both axes (graph loop) against the oracle's
    iterates: same tolerances as the default plans."""
    w = I.workload("c64_2d")
    po = O.Problem(w["n"], w["L"], w["eta"], w["omega"], w["V"])
    K = 20
    _, orep = O.pcg_solve(po, w["phi0"], O.SolveOptions(max_iter=K), keep_iterates=(K,))
    with G.Context(w["n"], w["L"], w["eta"], w["omega"], w["V"], prec=G.GPE_FP64) as ctx:
        ctx.set_plan(MODE_FP64, 0, 4, 4)
        ctx.set_plan(MODE_FP64, 1, 4, 8)
        phi = dev(w["phi0"])
        o = G.solve_opts_default()
        o.max_iter = K
        o.use_graph = 1
        rep = ctx.pcg_solve(phi, o, log_cap=64)
    assert rep["iters"] == K and rep["loop_kind"] == 1
    assert phase_aligned_rel_l2(host(phi), orep["iterates"][K]) < 1e-9
    for n_ in range(K + 1):
        e = orep["log"][n_]
        assert abs(rep["log"][n_, 2] - e["E"]) <= 1e-12 * abs(e["E"]), n_
        if n_ < K:
            assert int(rep["log"][n_, 10]) == int(e["fallback"]) and int(rep["log"][n_, 11]) == e["backtracks"]


@pytest.mark.parametrize("name", ["c64_2d", "fast256_2d"])
def test_autotuned_mixed_solve(G, name):
    """gpe_autotune on a mixed context, then the default solve: the chosen plans
    are valid, the tuned iteration is not slower than the default one, the
    process cache returns the same plans, and the answer passes the oracle."""
    w = I.workload(name)
    po = O.Problem(w["n"], w["L"], w["eta"], w["omega"], w["V"])
    with G.Context(w["n"], w["L"], w["eta"], w["omega"], w["V"], prec=G.GPE_MIXED) as ctx:
        rep_t = ctx.autotune(iters=10, use_cache=False)
        assert not rep_t["cached"] and rep_t["candidates"] > 0
        assert set(rep_t["plans"]) == {"complex64", "fp64", "refinement"}
        for m in range(3):
            assert 0 < rep_t["us_after"][m] <= rep_t["us_before"][m]
        again = ctx.autotune(iters=10, use_cache=True)
        assert again["cached"] and again["plans"] == rep_t["plans"]
        for m, name_m in enumerate(("complex64", "fp64", "refinement")):
            for ax, (E, wd) in enumerate(rep_t["plans"][name_m]):
                assert ctx.get_plan(m, ax) == (E, wd)
        phi = dev(w["phi0"])
        rep = ctx.pcg_solve(phi, check=True)
    assert rep["status"] == G.GPE_OK and rep["res_inf"] < 1e-8
    ph = host(phi)
    lam = O.chemical_potential(po, ph)
    assert np.max(np.abs(O.apply_H(po, ph, ph) - lam * ph)) < 1e-8
    assert abs(O.energy(po, ph) - rep["E"]) <= 1e-12 * abs(rep["E"])
    if name == "c64_2d":
        _, orep = O.pcg_solve(po, w["phi0"], O.SolveOptions())
        assert abs(rep["E"] - orep["E"]) <= 1e-7 * abs(orep["E"])


def test_autotuned_batch_matches_its_single_solves(G):
    """A batch tuned with gpe_batch_autotune reproduces single-instance solves
    whose contexts were tuned through the same process cache."""
    specs = [((64, 64), (8.0, 8.0), 100.0, 0.5, 1), ((32, 128), (6.0, 10.0), 60.0, 0.3, 2)]
    ws = []
    for n, L, eta, om, seed in specs:
        ws.append(dict(n=n, L=L, eta=eta, omega=om, V=I.harmonic(n, L), prec=G.GPE_MIXED,
                       phi0=I.perturbed(I.phi_d(n, L, om), seed, n, L)))
    opts = G.solve_opts_default()
    with G.Batch(ws) as B:
        B.autotune(iters=5)
        phis = [dev(w["phi0"]) for w in ws]
        s, reps = B.solve(phis, opts)
    assert s == G.GPE_OK
    for i, w in enumerate(ws):
        with G.Context(w["n"], w["L"], w["eta"], w["omega"], w["V"], prec=w["prec"]) as ctx:
            assert ctx.autotune(iters=5)["cached"]
            phi = dev(w["phi0"])
            r1 = ctx.pcg_solve(phi, opts)
        assert reps[i]["iters"] == r1["iters"] and reps[i]["E"] == r1["E"], (i, reps[i], r1)
        assert np.array_equal(host(phis[i]), host(phi))


@pytest.mark.parametrize("M", [64, 128, 256])
@pytest.mark.parametrize("E", [8, 16])
def test_batched_H_kernel_plans_match_oracle(G, M, E):
    """gpe_apply_H_batch's cluster kernel with E = 8 and E = 16 values per thread
    (plan mode 3) on a batch of complex64 fields against the oracle."""
    n, L = (M, M), (8.0, 8.0)
    V = I.harmonic(n, L)
    eta, om = 37.0, 0.7
    po = O.Problem(n, L, eta, om, V)
    nb = 5
    phis = np.stack([I.random_field(10 + b, n, L) for b in range(nb)])
    fs = np.stack([I.random_field(20 + b, n, L) for b in range(nb)])
    ph_d, f_d = dev(phis, torch.complex64), dev(fs, torch.complex64)
    out = torch.empty_like(f_d)
    with G.Context(n, L, eta, om, V, prec=G.GPE_MIXED) as ctx:
        ctx.set_plan(3, 0, E, 16)
        assert ctx.get_plan(3, 0) == (E, 16)
        ctx.apply_H_batch(nb, ph_d, f_d, out)
        got = host(out)
    phh, fh = host(ph_d), host(f_d)
    for b in range(nb):
        assert relmax(got[b], O.apply_H(po, phh[b], fh[b])) < 2e-5, b


@pytest.mark.parametrize("rows", [16, 32])
@pytest.mark.parametrize("M,nb", [(64, 150), (256, 37)])
def test_streaming_batched_H_kernel_loops_over_fields(G, M, nb, rows):
    """With E = 16 and 16-byte aligned fields the batched H kernel runs as
    resident clusters looping over the fields (rows of the next field copied
    while the current one's columns are transformed): more fields than
    resident clusters, every field against the oracle; phi != f."""
    n, L = (M, M), (8.0, 8.0)
    V = I.harmonic(n, L) + 0.2 * I.smooth_bumps(n, L, 3)
    eta, om = 41.0, 0.6
    po = O.Problem(n, L, eta, om, V)
    phis = np.stack([I.random_field(100 + b, n, L) for b in range(nb)])
    fs = np.stack([I.random_field(300 + b, n, L) for b in range(nb)])
    ph_d, f_d = dev(phis, torch.complex64), dev(fs, torch.complex64)
    out = torch.empty_like(f_d)
    with G.Context(n, L, eta, om, V, prec=G.GPE_MIXED) as ctx:
        ctx.set_plan(3, 0, 16, rows)
        assert ctx.get_plan(3, 0) == (16, rows)
        for rep in range(2):  # twice: the second launch starts from the first one's buffers
            out.fill_(float("nan"))
            ctx.apply_H_batch(nb, ph_d, f_d, out)
            got = host(out)
            assert np.isfinite(got).all()
    phh, fh = host(ph_d), host(f_d)
    for b in range(nb):
        assert relmax(got[b], O.apply_H(po, phh[b], fh[b])) < 2e-5, b


def test_batched_H_kernel_falls_back_for_misaligned_fields(G):
    """Fields that do not start on a 16-byte boundary cannot be copied by the
    streaming form's 16-byte asynchronous copies: the one-field-per-cluster
    form runs instead, with the same results."""
    M, nb = 128, 20
    n, L = (M, M), (8.0, 8.0)
    V = I.harmonic(n, L)
    po = O.Problem(n, L, 30.0, 0.5, V)
    fs = np.stack([I.random_field(500 + b, n, L) for b in range(nb)])
    buf = torch.empty(nb * M * M + 1, dtype=torch.complex64, device="cuda")
    f_d = buf[1:]  # 8 bytes past a 256-byte boundary
    f_d.copy_(torch.from_numpy(fs.reshape(-1).astype(np.complex64)))
    assert f_d.data_ptr() % 16 == 8
    out = torch.empty_like(f_d)
    with G.Context(n, L, 30.0, 0.5, V, prec=G.GPE_MIXED) as ctx:
        assert ctx.get_plan(3, 0) == (16, 16)  # the default in single precision
        ctx.apply_H_batch(nb, f_d, f_d, out)
        got = host(out).reshape(nb, M, M)
    fh = host(f_d).reshape(nb, M, M)
    for b in range(nb):
        assert relmax(got[b], O.apply_H(po, fh[b], fh[b])) < 2e-5, b


def _flow_fields(nb, seed0, n, L):
    return np.stack([I.random_field(seed0 + b, n, L) for b in range(nb)])


def test_dataflow_batched_H_matches_oracle_ragged_batches(G):
    """The dataflow form of gpe_apply_H_batch (256 x 256 complex64, f == phi:
    row and column units from one ticket queue, column units waiting on the
    field's row-unit counter, TMA-fed stages, TMA reduce-add of the column
    part) against the oracle, field by field, on batches below, at and above
    the 32-field lag between a field's row and column units (1, 5, 32, 33, 70
    fields), each batch twice and in an order that grows and shrinks the batch
    (the kernel leaves its counters zero for the next launch)."""
    M = 256
    n, L = (M, M), (16.0, 16.0)
    V = I.harmonic(n, L) + 0.3 * I.smooth_bumps(n, L, 4)
    eta, om = 900.0, 0.85
    po = O.Problem(n, L, eta, om, V)
    fields = _flow_fields(70, 700, n, L)
    with G.Context(n, L, eta, om, V, prec=G.GPE_MIXED) as ctx:
        assert ctx.get_plan(3, 0) == (16, 16)
        for nb in (5, 70, 1, 33, 32, 70):
            f_d = dev(fields[:nb], torch.complex64)
            out = torch.full_like(f_d, float("nan"))
            for rep in range(2):
                if rep:
                    out.fill_(float("nan"))
                ctx.apply_H_batch(nb, f_d, f_d, out)
                got = host(out)
                assert np.isfinite(got).all(), (nb, rep)
            fh = host(f_d)
            for b in range(nb):
                assert relmax(got[b], O.apply_H(po, fh[b], fh[b])) < 2e-5, (nb, b)


def test_dataflow_batched_H_full_size_sampled(G):
    """The roofline launch of the benchmark: 512 fields of 256 x 256 complex64
    (268 MB in, 268 MB out, above the 129 MB L2), f == phi, random normal
    fields; sampled fields (first, around the lag, middle, last) against the
    oracle, and every field finite."""
    M, nb = 256, 512
    n, L = (M, M), (16.0, 16.0)
    V = I.harmonic(n, L)
    eta, om = 1000.0, 0.9
    po = O.Problem(n, L, eta, om, V)
    g = torch.Generator(device="cuda").manual_seed(1)
    x = torch.randn(nb * M * M, dtype=torch.complex64, device="cuda", generator=g)
    out = torch.empty_like(x)
    with G.Context(n, L, eta, om, V, prec=G.GPE_MIXED) as ctx:
        ctx.apply_H_batch(nb, x, x, out)
        torch.cuda.synchronize()
        assert bool(torch.isfinite(torch.view_as_real(out)).all())
        xs, os_ = x.view(nb, M, M), out.view(nb, M, M)
        for b in (0, 31, 32, 33, 255, 480, 511):
            fh = xs[b].cpu().numpy()
            assert relmax(os_[b].cpu().numpy(), O.apply_H(po, fh, fh)) < 2e-5, b


def test_dataflow_batched_H_falls_back_for_misaligned_fields(G):
    """256 x 256 fields 8 bytes off a 16-byte boundary cannot be fed to the
    TMA: the cluster form runs instead, with the same results."""
    M, nb = 256, 4
    n, L = (M, M), (16.0, 16.0)
    V = I.harmonic(n, L)
    po = O.Problem(n, L, 500.0, 0.5, V)
    fs = _flow_fields(nb, 900, n, L)
    buf = torch.empty(nb * M * M + 1, dtype=torch.complex64, device="cuda")
    f_d = buf[1:]
    f_d.copy_(torch.from_numpy(fs.reshape(-1).astype(np.complex64)))
    assert f_d.data_ptr() % 16 == 8
    out = torch.empty_like(f_d)
    with G.Context(n, L, 500.0, 0.5, V, prec=G.GPE_MIXED) as ctx:
        ctx.apply_H_batch(nb, f_d, f_d, out)
        got = host(out).reshape(nb, M, M)
    fh = host(f_d).reshape(nb, M, M)
    for b in range(nb):
        assert relmax(got[b], O.apply_H(po, fh[b], fh[b])) < 2e-5, b
