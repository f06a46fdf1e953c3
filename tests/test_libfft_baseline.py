"""The library-FFT baseline (plain PyTorch + torch.fft PCG_C, complex128) runs
the same algorithm as the oracle: per-iterate energies and steps agree to
rounding, and the converged energy to rel 1e-12.  Runs on the CPU (torch.fft
without cuFFT); the bench times the same code on the GPU."""
import numpy as np
import pytest

from oracle import gpe_oracle as O
from paper_1611_02045_gb300 import inputs as I

torch = pytest.importorskip("torch")
from baseline.libfft_pcg import LibFFTPCG  # noqa: E402


def test_per_iterate_and_converged_against_oracle_2d():
    w = I.workload("c64_2d")
    po = O.Problem(w["n"], w["L"], w["eta"], w["omega"], w["V"])
    K = 20
    _, orep = O.pcg_solve(po, w["phi0"], O.SolveOptions(max_iter=K))
    b = LibFFTPCG(w["n"], w["L"], w["eta"], w["omega"], w["V"], device="cpu")
    log = []
    rep = b.solve(w["phi0"], max_iter=K, log=log)
    assert rep["iters"] == K and len(log) == K
    for n_ in range(K):
        e = orep["log"][n_]
        assert abs(log[n_][0] - e["E"]) <= 1e-12 * abs(e["E"]), n_
        assert abs(log[n_][3] - e["theta"]) <= 1e-9 * max(abs(e["theta"]), 1e-3), n_
    _, ofull = O.pcg_solve(po, w["phi0"], O.SolveOptions())
    full = b.solve(w["phi0"])
    assert full["status"] == "converged" and ofull["status"] == "converged"
    assert abs(full["E"] - ofull["E"]) <= 1e-12 * abs(ofull["E"])
    phi = full["phi"].numpy().reshape(po.n[::-1])
    lam = O.chemical_potential(po, phi)
    assert np.max(np.abs(O.apply_H(po, phi, phi) - lam * phi)) < 1e-8


def test_per_iterate_against_oracle_3d():
    n, L = (16, 16, 16), (6.0, 6.0, 6.0)
    V = I.harmonic(n, L, [1.0, 1.0, 2.0])
    phi0 = I.perturbed(I.phi_a(n, L), 3, n, L)
    po = O.Problem(n, L, 50.0, 0.4, V)
    K = 10
    _, orep = O.pcg_solve(po, phi0, O.SolveOptions(max_iter=K))
    log = []
    LibFFTPCG(n, L, 50.0, 0.4, V, device="cpu").solve(phi0, max_iter=K, log=log)
    for n_ in range(K):
        assert abs(log[n_][0] - orep["log"][n_]["E"]) <= 1e-12 * abs(orep["log"][n_]["E"]), n_
