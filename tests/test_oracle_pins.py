"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(not by the oracle itself).  Each test names the pin it implements:

P0 transforms = brute-force DFT sums; P1 harmonic ground state (closed form);
P2 sign/scale of L_z via phi_b; P3 Hermiticity; P4 gradient = 2 H phi (FD);
P5 exact energy change along the geodesic and its curvature (FD);
P6 preconditioner symmetry/positivity and exact inversion of P_Delta;
P7 converged energies printed in the paper's Table 2;
P8 method invariants (monotone energy, unit norm); P9 stationarity;
P10-P12 derivatives (differences of energies and of re-solved ground states);
P13 Thomas-Fermi mu (continuum closed forms); P14 spectral interpolation
(band-limited exactness, brute-force trigonometric sums);
P15 the shift lambda~ of eq. Opt_Alpha (closed forms of the harmonic states);
P16 the scalar logic of Algorithm 2: every step descends and beta+ >= 0,
restarts take the preconditioned gradient, Polak-Ribiere directions are
secant-conjugate (Hestenes-Stiefel), theta_0 is the Newton step of the energy
along the geodesic, and CG needs fewer iterations than the gradient method.
"""
import json
import os

import numpy as np
import pytest

from oracle import gpe_oracle as O
from paper_1611_02045_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_table_energies.json")


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def prob2(M=16, L=4.0, eta=3.0, omega=0.4, backend="fft", V=None, n=None):
    n = n or (M, M)
    L_ = (L,) * len(n)
    if V is None:
        V = I.harmonic(n, L_)
    return O.Problem(n, L_, eta, omega, V, backend=backend)


# ---------------------------------------------------------------- P0
@pytest.mark.parametrize("n", [(8, 8), (4, 8), (4, 4, 4), (8, 4, 2)])
def test_P0_separable_dft_equals_bruteforce(n):
    """Naive separable DFT == the d-dimensional DFT sum written out over all
    (p, k) pairs (Section 3 convention)."""
    f = I.random_field(11, n, (1.0,) * len(n))
    p = O.Problem(n, (1.0,) * len(n), 0.0, 0.0, np.zeros(f.shape), backend="naive")
    shape = f.shape  # [z][y][x]
    idx = np.array(np.unravel_index(np.arange(f.size), shape)).T  # (N, d) numpy axes
    Ms = np.array(shape)
    phase = -2j * np.pi * (idx[:, None, :] * idx[None, :, :] / Ms).sum(-1)
    brute = (np.exp(phase) @ f.ravel()).reshape(shape)
    assert rel(O.dftn(p, f), brute) < 1e-13
    back = (np.exp(-phase) @ brute.ravel()).reshape(shape) / f.size
    assert rel(O.dftn(p, brute, inverse=True), back) < 1e-13
    assert rel(back, f) < 1e-13


def test_P0_fft_backend_equals_naive_backend():
    n = (16, 8)
    V = I.harmonic(n, (3.0, 3.0))
    pf = O.Problem(n, (3.0, 3.0), 2.0, 0.7, V, backend="fft")
    pn = O.Problem(n, (3.0, 3.0), 2.0, 0.7, V, backend="naive")
    phi = I.random_field(1, n, (3.0, 3.0))
    f = I.random_field(2, n, (3.0, 3.0))
    assert rel(O.apply_H(pf, phi, f), O.apply_H(pn, phi, f)) < 1e-13
    assert rel(O.precond_C(pf, phi, f, 2.5), O.precond_C(pn, phi, f, 2.5)) < 1e-13


@pytest.mark.parametrize("axis", [0, 1])
def test_P0_spectral_derivative_of_single_mode(axis):
    """A single Fourier mode e^{i xi_p (x+L)} has d/dx = i xi_p, d2/dx2 = -xi_p^2,
    with xi_p = p pi / L (Section 3), including the kept Nyquist mode p = -M/2."""
    n, L = (16, 16), (2.5, 2.5)
    p = O.Problem(n, L, 0.0, 0.0, np.zeros((16, 16)))
    x = p.coord(axis) + L[axis]
    for q in (1, 3, -5, -8):
        xi = q * np.pi / L[axis]
        f = np.exp(1j * xi * x) * np.ones((16, 16))
        assert rel(O.d1_axis(p, f, axis), 1j * xi * f) < 1e-12
        assert rel(O.d2_axis(p, f, axis), -xi * xi * f) < 1e-12


# ---------------------------------------------------------------- P1
def test_P1_harmonic_gaussian_2d():
    n, L = (64, 64), (8.0, 8.0)
    p = O.Problem(n, L, 0.0, 0.0, I.harmonic(n, L))
    g = I.phi_a(n, L)
    assert abs(O.norm(p, g) - 1.0) < 1e-13
    e = O.energy_parts(p, g)
    assert abs(e["total"] - 1.0) < 1e-12
    assert abs(e["kin"] - 0.5) < 1e-12 and abs(e["pot"] - 0.5) < 1e-12  # virial split
    assert np.max(np.abs(O.apply_H(p, g, g) - g)) < 1e-12


def test_P1_harmonic_gaussian_3d_anisotropic():
    n, L = (64, 64, 64), (8.0, 8.0, 8.0)  # h = 1/4: aliasing of the Gaussians below 1e-15
    p = O.Problem(n, L, 0.0, 0.0, I.harmonic(n, L, [1.0, 1.0, 2.0]))
    g = I.anisotropic_gaussian(n, L, [1.0, 1.0, 2.0])
    assert abs(O.energy(p, g) - 2.0) < 1e-12
    assert abs(O.chemical_potential(p, g) - 2.0) < 1e-12


def test_P1_pcg_converges_to_harmonic_ground_state():
    n, L = (32, 32), (8.0, 8.0)
    p = O.Problem(n, L, 0.0, 0.0, I.harmonic(n, L))
    phi0 = I.perturbed(I.phi_a(n, L), 7, n, L, amp=0.2)
    phi, rep = O.pcg_solve(p, phi0, O.SolveOptions(tol_res_inf=1e-10, max_iter=500))
    assert rep["status"] == "converged"
    assert abs(rep["E"] - 1.0) < 1e-12
    assert abs(rep["lam"] - 1.0) < 1e-9


# ---------------------------------------------------------------- P2
def test_P2_angular_momentum_sign_and_scale():
    """L_z phi_a = 0 (radial), L_z phi_b = +phi_b for phi_b = (x+iy) phi_a; at eta = 0
    H phi_b = (2 - omega) phi_b and E(phi_b) = 2 - omega (Section 2, initial data (b))."""
    n, L = (64, 64), (8.0, 8.0)
    om = 0.3
    p = O.Problem(n, L, 0.0, om, I.harmonic(n, L))
    a = I.phi_a(n, L)
    b = I.normalise(I.phi_b(n, L), n, L)
    assert np.max(np.abs(O.Lz(p, a))) < 1e-12
    assert np.max(np.abs(O.Lz(p, b) - b)) < 1e-11
    assert np.max(np.abs(O.apply_H(p, b, b) - (2.0 - om) * b)) < 1e-11
    assert abs(O.energy(p, b) - (2.0 - om)) < 1e-12
    assert abs(O.energy(p, np.conj(b)) - (2.0 + om)) < 1e-12


# ---------------------------------------------------------------- P3
@pytest.mark.parametrize("n", [(16, 16), (8, 16, 8)])
def test_P3_hamiltonian_hermitian(n):
    L = (3.0,) * len(n)
    p = O.Problem(n, L, 5.0, 0.8, I.harmonic(n, L))
    phi, f, g = (I.random_field(s, n, L) for s in (1, 2, 3))
    lhs = O.inner(p, g, O.apply_H(p, phi, f))
    rhs = np.conj(O.inner(p, f, O.apply_H(p, phi, g)))
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


# ---------------------------------------------------------------- P4
def test_P4_gradient_is_two_H_phi():
    n, L = (16, 16), (4.0, 4.0)
    p = O.Problem(n, L, 7.0, 0.6, I.harmonic(n, L))
    phi = I.normalise(I.phi_d(n, L, 0.6) * (1 + 0.1 * I.random_field(4, n, L)), n, L)
    d = I.random_field(5, n, L) * 0.1
    eps = 1e-5
    fd = (O.energy(p, phi + eps * d) - O.energy(p, phi - eps * d)) / (2 * eps)
    an = 2.0 * O.inner(p, O.apply_H(p, phi, phi), d).real
    assert abs(fd - an) < 1e-8 * abs(an)


# ---------------------------------------------------------------- P5
def _tangent_unit(p, phi, seed):
    q = I.random_field(seed, p.n, p.L)
    q = q - O.inner(p, q, phi).real * phi
    return q / O.norm(p, q)


def test_P5_exact_energy_change_along_geodesic():
    n, L = (16, 16), (4.0, 4.0)
    p = O.Problem(n, L, 40.0, 0.7, I.harmonic(n, L))
    phi = I.normalise(I.phi_d(n, L, 0.7), n, L)
    q = _tangent_unit(p, phi, 9)
    Hphi = O.apply_H(p, phi, phi)
    lam = O.inner(p, phi, Hphi).real
    m = O.step_moments(p, phi, Hphi, lam, q)
    E0 = O.energy(p, phi)
    for th in (1e-3, 1e-2, 0.1, 0.5, 1.3, -0.4):
        direct = O.energy(p, np.cos(th) * phi + np.sin(th) * q) - E0
        model = O.delta_energy(m, p.eta, th)
        assert abs(direct - model) < 1e-12 * abs(E0) + 1e-11 * abs(direct)


def test_P5_curvature_matches_second_difference():
    n, L = (16, 16), (4.0, 4.0)
    p = O.Problem(n, L, 40.0, 0.7, I.harmonic(n, L))
    phi = I.normalise(I.phi_d(n, L, 0.7), n, L)
    q = _tangent_unit(p, phi, 10)
    lam = O.chemical_potential(p, phi)
    Eh = lambda t: O.energy(p, np.cos(t) * phi + np.sin(t) * q)  # noqa: E731
    h = 1e-3
    fd2 = (Eh(h) - 2 * Eh(0.0) + Eh(-h)) / (h * h)
    assert abs(fd2 - 2.0 * O.model_curvature(p, phi, lam, q)) < 1e-5 * abs(fd2)
    fd1 = (Eh(h) - Eh(-h)) / (2 * h)
    R = O.inner(p, O.apply_H(p, phi, phi), q).real
    assert abs(fd1 - 2.0 * R) < 1e-5 * abs(fd1)


# ---------------------------------------------------------------- P6
@pytest.mark.parametrize("n", [(16, 16), (8, 8, 16)])
def test_P6_preconditioner_hermitian_positive(n):
    L = (3.0,) * len(n)
    p = O.Problem(n, L, 5.0, 0.8, I.harmonic(n, L))
    phi, f, g = (I.random_field(s, n, L) for s in (21, 22, 23))
    alpha = 1.7
    a = O.inner(p, g, O.precond_C(p, phi, f, alpha))
    b = np.conj(O.inner(p, f, O.precond_C(p, phi, g, alpha)))
    assert abs(a - b) < 1e-13 * abs(a)
    for s in range(5):
        h = I.random_field(30 + s, n, L)
        assert O.inner(p, h, O.precond_C(p, phi, h, alpha)).real > 0


def test_P6_kinetic_preconditioner_inverts_shifted_laplacian():
    n, L = (16, 8), (3.0, 2.0)
    p = O.Problem(n, L, 0.0, 0.0, np.zeros((8, 16)))
    f = I.random_field(3, n, L)
    alpha = 0.9
    g = O.precond_delta(p, f, alpha)
    assert rel(alpha * g - 0.5 * O.laplacian(p, g), f) < 1e-13
    # P_C with V = 0 and eta = 0 is P_Delta / alpha (P_V = 1/alpha)
    assert rel(O.precond_C(p, np.zeros_like(f), f, alpha), g / alpha) < 1e-13


# ---------------------------------------------------------------- P7
def _paper():
    with open(GOLDEN) as fh:
        return json.load(fh)


@pytest.mark.parametrize("omega", [0.0, 0.5])
def test_P7_radial_state_energy_matches_paper(omega):
    n, L = (256, 256), (16.0, 16.0)
    p = O.Problem(n, L, 500.0, omega, I.harmonic(n, L))
    phi, rep = O.pcg_solve(p, I.phi_a(n, L), O.SolveOptions(tol_res_inf=1e-8, max_iter=300))
    assert rep["status"] == "converged"
    assert abs(rep["E"] - _paper()["radial_state_from_phi_a"]["any_omega"]) < 1e-4


@pytest.mark.parametrize("omega", ["0.5", "0.6"])
def test_P7_vortex_state_energy_matches_paper(omega):
    n, L = (256, 256), (16.0, 16.0)
    p = O.Problem(n, L, 500.0, float(omega), I.harmonic(n, L))
    phi, rep = O.pcg_solve(p, I.phi_b(n, L), O.SolveOptions(tol_res_inf=1e-8, max_iter=300))
    assert rep["status"] == "converged"
    assert abs(rep["E"] - _paper()["vortex_state_from_phi_b"][omega]) < 1e-4


def test_P7_fast_rotation_lowest_energy_matches_paper():
    """omega = 0.9 from phi_d: the lowest energy 4.7777 of Table 2."""
    n, L = (256, 256), (16.0, 16.0)
    p = O.Problem(n, L, 500.0, 0.9, I.harmonic(n, L))
    phi, rep = O.pcg_solve(p, I.phi_d(n, L, 0.9), O.SolveOptions(tol_res_inf=3e-5, max_iter=4000))
    assert rep["status"] == "converged"
    assert abs(rep["E"] - _paper()["lowest_energy"]["0.9"]) < 1e-4


# ---------------------------------------------------------------- P8 / P9
def test_P8_P9_invariants_and_stationarity():
    w = I.workload("c64_2d")
    p = O.Problem(w["n"], w["L"], w["eta"], w["omega"], w["V"])
    keep = tuple(range(0, 400, 7))
    phi, rep = O.pcg_solve(p, w["phi0"], O.SolveOptions(tol_res_inf=1e-8, max_iter=2000), keep_iterates=keep)
    assert rep["status"] == "converged"
    E = np.array([e["E"] for e in rep["log"]])
    assert np.all(np.diff(E) <= 1e-12 * abs(E[0]))  # every accepted step lowers E
    for ph in rep["iterates"].values():
        assert abs(O.norm(p, ph) - 1.0) < 1e-13
    Hphi = O.apply_H(p, phi, phi)
    lam = O.inner(p, phi, Hphi).real
    assert np.max(np.abs(Hphi - lam * phi)) < 1e-8
    # energy error is quadratic in the residual near the minimum
    assert abs(E[-1] - rep["E"]) == 0.0


# ---------------------------------------------------------------- P10-P12: derivatives
def _grad_problem(omega=0.3):
    n, L = (16, 16), (4.0, 4.0)
    V = I.harmonic(n, L) + 0.3 * I.smooth_bumps(n, L, 11)
    return O.Problem(n, L, 10.0, omega, V)


def test_P10_energy_gradient_matches_central_differences():
    """energy_gradient is dE/dRe phi + i dE/dIm phi: central differences of the
    energy along a real and an imaginary direction reproduce Re<g, d> (unweighted)."""
    p = _grad_problem()
    n, L = p.n, p.L
    phi = I.normalise(I.phi_d(n, L, 0.5) * (1 + 0.2 * I.random_field(21, n, L)), n, L)
    g = O.energy_gradient(p, phi)
    eps = 1e-6
    for d in (I.random_field(22, n, L).real + 0j, 1j * I.random_field(23, n, L).real):
        fd = (O.energy(p, phi + eps * d) - O.energy(p, phi - eps * d)) / (2 * eps)
        an = np.sum((np.conj(g) * d).real)
        assert abs(fd - an) < 1e-7 * abs(an)


@pytest.mark.parametrize("omega", [0.3, 0.0])
def test_P10_parameter_derivatives_match_central_differences(omega):
    """dE/dV, dE/deta, dE/domega at fixed phi against differences of the energy
    in each parameter (omega = 0 included: the derivative is -<phi, L_z phi>)."""
    p = _grad_problem(omega)
    n, L = p.n, p.L
    phi = I.normalise(I.phi_d(n, L, 0.5) * (1 + 0.2 * I.random_field(24, n, L)), n, L)
    d = O.energy_parameter_derivatives(p, phi)
    h = 1e-6

    def E(eta=p.eta, om=p.omega, V=p.V):
        return O.energy(O.Problem(n, L, eta, om, V), phi)

    assert abs((E(eta=p.eta + h) - E(eta=p.eta - h)) / (2 * h) - d["deta"]) < 1e-7 * abs(d["deta"])
    fd_om = (E(om=omega + h) - E(om=omega - h)) / (2 * h)
    assert abs(d["domega"]) > 1e-3 and abs(fd_om - d["domega"]) < 1e-7 * abs(d["domega"])
    S = I.smooth_bumps(n, L, 13)
    fd_V = (E(V=p.V + h * S) - E(V=p.V - h * S)) / (2 * h)
    assert abs(fd_V - np.sum(d["dV"] * S)) < 1e-7 * abs(fd_V)


def solve_ground_state_16():
    p = _grad_problem()
    phi0 = I.perturbed(I.phi_a(p.n, p.L), 12, p.n, p.L, amp=1e-2)
    phi, rep = O.pcg_solve(p, phi0, O.SolveOptions(tol_res_inf=1e-12))
    assert rep["status"] == "converged"
    return p, phi


@pytest.fixture(scope="module")
def ground_state_16():
    return solve_ground_state_16()


def _resolve(p, phi_start, eta=None, omega=None, dV=0.0):
    q = O.Problem(p.n, p.L, p.eta if eta is None else eta, p.omega if omega is None else omega, p.V + dV)
    f, rep = O.pcg_solve(q, phi_start, O.SolveOptions(tol_res_inf=1e-12))
    assert rep["status"] == "converged"
    return f, rep["E"]


def test_P11_hellmann_feynman_matches_differences_of_solves(ground_state_16):
    """At a ground state, the fixed-phi derivatives equal the derivatives of the
    ground-state energy E*(eta, omega, V), obtained here by re-solving the
    perturbed problems (warm start at phi*) and central differences."""
    p, phi = ground_state_16
    d = O.energy_parameter_derivatives(p, phi)
    h = 1e-5
    fd = (_resolve(p, phi, eta=p.eta + h)[1] - _resolve(p, phi, eta=p.eta - h)[1]) / (2 * h)
    assert abs(fd - d["deta"]) < 1e-7 * abs(d["deta"])
    fd = (_resolve(p, phi, omega=p.omega + h)[1] - _resolve(p, phi, omega=p.omega - h)[1]) / (2 * h)
    assert abs(fd - d["domega"]) < 1e-5 * abs(d["domega"])
    S = I.smooth_bumps(p.n, p.L, 13)
    fd = (_resolve(p, phi, dV=h * S)[1] - _resolve(p, phi, dV=-h * S)[1]) / (2 * h)
    assert abs(fd - np.sum(d["dV"] * S)) < 1e-7 * abs(fd)


def test_P12_hessian_operator_is_the_second_order_form(ground_state_16):
    """Re<f, K f> = 1/2 grad^2 E[f, f] - lam ||f||^2 (Section 2), and the phase
    direction i phi is in the kernel of K at a critical point."""
    p, phi = ground_state_16
    lam = O.chemical_potential(p, phi)
    f = I.random_field(31, p.n, p.L)
    lhs = O.inner(p, f, O.hessian_apply(p, phi, lam, f)).real
    rhs = O.hessian_form(p, phi, f) - lam * O.inner(p, f, f).real
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)
    k = O.hessian_apply(p, phi, lam, 1j * phi)
    assert O.norm(p, k) < 1e-10


def test_P12_density_loss_gradient_matches_differences_of_solves(ground_state_16):
    """The tangent-space adjoint gradient of L = int (|phi*|^2 - rho)^2 with
    respect to V against central differences of L over re-solved ground states."""
    p, phi = ground_state_16
    rho = np.abs(I.normalise(I.anisotropic_gaussian(p.n, p.L, [1.3, 0.8]), p.n, p.L)) ** 2
    gV, it, res = O.density_loss_gradient_V(p, phi, rho)
    assert res < 1e-12 and it < 200
    h = 1e-5
    for seed in (13, 14):
        S = I.smooth_bumps(p.n, p.L, seed)
        fp, _ = _resolve(p, phi, dV=h * S)
        fm, _ = _resolve(p, phi, dV=-h * S)
        fd = (O.density_loss(p, fp, rho) - O.density_loss(p, fm, rho)) / (2 * h)
        an = np.sum(gV * S)
        assert abs(fd - an) < 1e-5 * abs(an)


# ---------------------------------------------------------------- P6b / P8b: preconditioner variants
def test_P6_preconditioner_variants_adjointness():
    """P_V and P_Delta are self-adjoint, so P_C, P_Delta, P_V are self-adjoint and
    P_C1 = P_V P_Delta and P_C2 = P_Delta P_V (eq. combinedP) are each other's
    adjoints, <f, P_C1 g> = <P_C2 f, g>, while P_C1 itself is not self-adjoint."""
    p = prob2(M=16, eta=5.0)
    n, L = p.n, p.L
    phi = I.normalise(I.phi_d(n, L, 0.4) * (1 + 0.3 * I.random_field(41, n, L)), n, L)
    f, g = I.random_field(42, n, L), I.random_field(43, n, L)
    a = 2.3

    def P(x, kind):
        return O.apply_preconditioner(p, phi, x, a, kind)

    for kind in ("C", "Delta", "V", "none"):
        lhs, rhs = O.inner(p, f, P(g, kind)), O.inner(p, P(f, kind), g)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs), kind
    lhs, rhs = O.inner(p, f, P(g, "C1")), O.inner(p, P(f, "C2"), g)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    asym = O.inner(p, f, P(g, "C1")) - O.inner(p, P(f, "C1"), g)
    assert abs(asym) > 1e-3 * abs(lhs)
    # P_V is the inverse of multiplication by alpha + V + eta |phi|^2
    m = a + p.V + p.eta * np.abs(phi) ** 2
    assert np.max(np.abs(m * P(g, "V") - g)) < 1e-13 * np.max(np.abs(g))


@pytest.mark.parametrize("precond,beta", [("C", "PR"), ("Delta", "PR"), ("V", "PR"), ("C1", "PR"),
                                          ("C2", "PR"), ("none", "PR"), ("C", "FR")])
def test_P8_every_preconditioner_reaches_the_same_ground_state(precond, beta):
    """The ground state does not depend on the preconditioner or on the
    conjugation rule: each variant converges (||r||_inf < 1e-9) to the energy of
    the default (P_C, Polak-Ribiere) solve, with monotone energy decrease."""
    n, L = (64, 64), (8.0, 8.0)
    p = O.Problem(n, L, 100.0, 0.2, I.harmonic(n, L))
    phi0 = I.perturbed(I.phi_a(n, L), 7, n, L)
    ref = _P8_reference(p, phi0)
    _, rep = O.pcg_solve(p, phi0, O.SolveOptions(tol_res_inf=1e-9, max_iter=5000, precond=precond, beta=beta))
    assert rep["status"] == "converged", (precond, beta, rep["iters"])
    assert abs(rep["E"] - ref) < 1e-11 * abs(ref)
    Es = [e["E"] for e in rep["log"]]
    assert all(b <= a + 1e-12 * abs(a) for a, b in zip(Es, Es[1:]))


_P8_REF = {}


def _P8_reference(p, phi0):
    if "E" not in _P8_REF:
        _, rep = O.pcg_solve(p, phi0, O.SolveOptions(tol_res_inf=1e-10))
        _P8_REF["E"] = rep["E"]
    return _P8_REF["E"]


# ---------------------------------------------------------------- P5b: exact line search
def _line_moments(seed=51):
    p = _grad_problem()
    n, L = p.n, p.L
    phi = I.normalise(I.phi_d(n, L, 0.5) * (1 + 0.2 * I.random_field(seed, n, L)), n, L)
    lam = O.chemical_potential(p, phi)
    Hphi = O.apply_H(p, phi, phi)
    r = Hphi - lam * phi
    q = -O.precond_C(p, phi, r, O.lambda_tilde(p, phi))
    q = q - O.inner(p, q, phi).real * phi
    q = q / O.norm(p, q)
    return p, O.step_moments(p, phi, Hphi, lam, q)


def test_P5_line_search_derivatives_match_differences():
    """The closed-form first and second derivatives of the step polynomial
    against central differences of delta_energy at several steps."""
    p, m = _line_moments()
    h = 1e-5
    for t in (0.01, 0.1, 0.4, 1.0):
        d1, d2 = O.delta_energy_derivatives(m, p.eta, t)
        f = lambda x: O.delta_energy(m, p.eta, x)  # noqa: E731
        fd1 = (f(t + h) - f(t - h)) / (2 * h)
        fd2 = (O.delta_energy_derivatives(m, p.eta, t + h)[0] - O.delta_energy_derivatives(m, p.eta, t - h)[0]) / (2 * h)
        assert abs(d1 - fd1) < 1e-7 * max(abs(d1), 1e-3), t
        assert abs(d2 - fd2) < 1e-6 * max(abs(d2), 1e-3), t


def test_P5_exact_step_minimises_the_energy_along_the_geodesic():
    """The Newton step is the minimiser of the energy along cos t phi + sin t q
    near the model step: no point of a dense scan of the direct energy
    difference is lower, and the derivative vanishes there."""
    p, m = _line_moments()
    curv = m["aqq"] - m["lam"]
    t0 = -m["R"] / curv
    ts = O.exact_step(m, p.eta, t0)
    assert ts != t0 and 0 < ts < 1.5
    assert abs(O.delta_energy_derivatives(m, p.eta, ts)[0]) < 1e-12 * max(abs(m["R"]), 1e-12)
    grid = np.linspace(0.5 * ts, 1.5 * ts, 2001)
    vals = np.array([O.delta_energy(m, p.eta, t) for t in grid])
    assert O.delta_energy(m, p.eta, ts) <= vals.min() + 1e-14 * abs(vals.min())
    assert O.delta_energy(m, p.eta, ts) <= O.delta_energy(m, p.eta, t0)


# ---------------------------------------------------------------- P13: Thomas-Fermi initial data
@pytest.mark.parametrize("gammas", [(1.0, 1.0), (1.0, 1.5)])
def test_P13_thomas_fermi_mu_matches_the_continuum_closed_form_2d(gammas):
    """For V = sum gamma_i^2 x_i^2 / 2 the region V < mu is an ellipse and
    int max(mu - V, 0) / eta = pi mu^2 / (eta gamma_x gamma_y) = 1 gives
    mu = sqrt(eta gamma_x gamma_y / pi); the grid sum converges to it."""
    n, L = (512, 512), (16.0, 16.0)
    eta = 1000.0
    p = O.Problem(n, L, eta, 0.0, I.harmonic(n, L, list(gammas)))
    mu = O.thomas_fermi_mu(p)
    want = np.sqrt(eta * gammas[0] * gammas[1] / np.pi)
    assert abs(mu - want) < 2e-4 * want
    phi, mu2 = O.thomas_fermi_state(p)
    assert mu2 == mu and abs(O.norm(p, phi) - 1.0) < 1e-14
    # the unnormalised state already has unit norm (the defining condition)
    raw = np.sqrt(np.maximum(mu - p.V, 0.0) / eta)
    assert abs(p.weight * np.sum(raw ** 2) - 1.0) < 1e-12


def test_P13_thomas_fermi_mu_matches_the_continuum_closed_form_3d():
    """3D: with y_i = g_i x_i / sqrt(2 mu) the region is the unit ball and
    int max(mu - V, 0) = (2 mu)^{3/2} mu (4 pi/3 - 4 pi/5) / (g_x g_y g_z)
    = 16 sqrt(2) pi mu^{5/2} / (15 g_x g_y g_z), so
    mu = (15 eta g_x g_y g_z / (16 sqrt(2) pi))^{2/5}."""
    n, L = (128, 128, 128), (8.0, 8.0, 8.0)
    g = (1.0, 1.0, 2.0)
    eta = 5000.0
    p = O.Problem(n, L, eta, 0.0, I.harmonic(n, L, list(g)))
    mu = O.thomas_fermi_mu(p)
    want = (15.0 * eta * g[0] * g[1] * g[2] / (16.0 * np.sqrt(2.0) * np.pi)) ** 0.4
    assert abs(mu - want) < 2e-3 * want


# ---------------------------------------------------------------- P14: spectral interpolation
def _band_limited(n, L, modes):
    m = I.mesh(n, L)
    f = np.zeros(m[0].shape, dtype=complex)
    for k, (coef, ks) in enumerate(modes):
        phase = sum(kk * np.pi / Li * (xi + Li) for kk, xi, Li in zip(ks, m, L))
        f = f + coef * np.exp(1j * phase)
    return f


@pytest.mark.parametrize("nc,nf", [((16, 8), (32, 16)), ((8, 8, 8), (16, 16, 16)), ((16, 16), (64, 64))])
def test_P14_interpolation_is_exact_for_band_limited_fields(nc, nf):
    """A field made of Fourier modes |p| < Mc/2 (and a cosine at the coarse
    Nyquist frequency, which the symmetric split reproduces) is interpolated
    exactly: the result equals the same analytic field sampled on the fine grid."""
    L = tuple([4.0, 5.0, 3.0][: len(nc)])
    modes = [(1.0 + 0.5j, [1] * len(nc)), (0.3, [-(nc[0] // 2) + 1] + [2] * (len(nc) - 1)),
             (-0.7j, [3] + [-1] * (len(nc) - 1))]
    pc = O.Problem(nc, L, 1.0, 0.0, np.zeros(I.shape_of(nc)))
    pf = O.Problem(nf, L, 1.0, 0.0, np.zeros(I.shape_of(nf)))
    fc = _band_limited(nc, L, modes)
    # a cosine at the coarse Nyquist frequency along x (cos(Mc/2 * pi/L * (x + L)))
    mc = I.mesh(nc, L)
    mf = I.mesh(nf, L)
    fc = fc + 0.4 * np.cos(nc[0] // 2 * np.pi / L[0] * (mc[0] + L[0]))
    want = _band_limited(nf, L, modes) + 0.4 * np.cos(nc[0] // 2 * np.pi / L[0] * (mf[0] + L[0]))
    got = O.interpolate(pc, fc, pf)
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))


def test_P14_interpolation_keeps_coarse_values_and_matches_the_trigonometric_sum():
    """On a tiny grid: the fine values at the coarse points are the coarse
    values, and every fine value equals the brute-force trigonometric sum."""
    nc, nf, L = (8, 4), (16, 8), (2.0, 3.0)
    pc = O.Problem(nc, L, 1.0, 0.0, np.zeros(I.shape_of(nc)))
    pf = O.Problem(nf, L, 1.0, 0.0, np.zeros(I.shape_of(nf)))
    fc = I.random_field(61, nc, L)
    got = O.interpolate(pc, fc, pf)
    assert np.max(np.abs(got[::2, ::2] - fc)) < 1e-13
    xc, yc = pc.coord(0), pc.coord(1)
    xs, ys = pf.coord(0).ravel(), pf.coord(1).ravel()

    def weight(p, M):  # Nyquist shared by -M/2 and +M/2
        return 0.5 if abs(p) == M // 2 else 1.0

    for j, y in enumerate(ys):
        for i, x in enumerate(xs):
            tot = 0.0
            for py in range(-nc[1] // 2, nc[1] // 2 + 1):
                for px in range(-nc[0] // 2, nc[0] // 2 + 1):
                    w = weight(px, nc[0]) * weight(py, nc[1])
                    # coefficient F_p of the coarse DFT (index p mod M)
                    e = np.exp(-1j * (px * np.pi / L[0] * (xc + L[0]) + py * np.pi / L[1] * (yc + L[1])))
                    Fp = np.sum(fc * e)
                    tot += w * Fp * np.exp(1j * (px * np.pi / L[0] * (x + L[0]) + py * np.pi / L[1] * (y + L[1])))
            tot /= nc[0] * nc[1]
            assert abs(tot - got[j, i]) < 1e-12, (i, j)


# ---------------------------------------------------------------- P15: the shift alpha = lambda~
@pytest.mark.parametrize("eta,omega", [(0.0, 0.0), (0.0, 0.7), (100.0, 0.0), (100.0, 0.7)])
def test_P15_lambda_tilde_closed_forms(eta, omega):
    """lambda~(phi) = int 1/2|grad phi|^2 + V|phi|^2 + eta|phi|^4 (eq. Opt_Alpha) for
    V = r^2/2 and the two lowest harmonic states (Section 6, initial data (a), (b)):
    phi_a = pi^{-1/2} e^{-r^2/2} has kinetic + potential energy 1 and int |phi_a|^4 = 1/(2 pi);
    phi_b = (x+iy) phi_a has 2 and int |phi_b|^4 = 1/(4 pi).  lambda~ carries no
    rotation term, so it is independent of omega, and lambda~ - lambda = omega <phi, L_z phi>,
    which is omega for phi_b (L_z phi_b = phi_b) and 0 for the radial phi_a."""
    n, L = (64, 64), (8.0, 8.0)
    p = O.Problem(n, L, eta, omega, I.harmonic(n, L))
    a, b = I.phi_a(n, L), I.phi_b(n, L)
    assert abs(O.norm(p, b) - 1.0) < 1e-13
    assert abs(O.lambda_tilde(p, a) - (1.0 + eta / (2.0 * np.pi))) < 1e-12
    assert abs(O.lambda_tilde(p, b) - (2.0 + eta / (4.0 * np.pi))) < 1e-12
    assert abs(O.lambda_tilde(p, b) - O.chemical_potential(p, b) - omega) < 1e-12
    assert abs(O.lambda_tilde(p, a) - O.chemical_potential(p, a)) < 1e-12


# ---------------------------------------------------------------- P16: the scalar logic of Algorithm 2
def _solve_with_iterates(p, phi0, n_iter, **kw):
    opts = O.SolveOptions(tol_res_inf=1e-8, max_iter=n_iter, **kw)
    _, rep = O.pcg_solve(p, phi0, opts, keep_iterates=tuple(range(n_iter + 1)))
    return rep


def _directions(p, rep):
    """Per accepted iteration n: phi_n, the residual r_n = H phi_n - lambda_n phi_n from
    the Hamiltonian (pinned by P1-P4), and the unit search direction q_n recovered from the
    retraction phi_{n+1} = cos(theta_n) phi_n + sin(theta_n) q_n (which has unit norm
    because Re<phi_n, q_n> = 0): nothing here repeats the solver's scalar formulas."""
    out = []
    its, log = rep["iterates"], rep["log"]
    for n in range(rep["iters"]):
        if n + 1 not in its:
            break
        phi, th = its[n], log[n]["theta"]
        Hphi = O.apply_H(p, phi, phi)
        r = Hphi - O.inner(p, phi, Hphi).real * phi
        q = (its[n + 1] - np.cos(th) * phi) / np.sin(th)
        out.append(dict(n=n, phi=phi, r=r, q=q, **{k: log[n][k] for k in ("theta", "beta", "fallback", "backtracks")}))
    return out


def _fast_rotation_32():
    """A small fast-rotation problem whose first 40 iterations include a Polak-Ribiere
    restart (beta_PR < 0, iteration 6) and a descent-check fallback (iteration 16)."""
    n, L = (32, 32), (6.0, 6.0)
    p = O.Problem(n, L, 200.0, 0.95, I.harmonic(n, L))
    return p, I.perturbed(I.phi_d(n, L, 0.95), 3, n, L)


def _cosine(p, f, g):
    return O.inner(p, f, g).real / (O.norm(p, f) * O.norm(p, g))


def test_P16_every_step_descends_and_beta_is_nonnegative():
    """Section 5.2 enforces a descent direction at every step (reverting to the
    gradient step otherwise), so Re<grad E(phi_n), q_n> = 2 Re<r_n, q_n> < 0 for
    every accepted q_n; the energy decreases at every step; beta+ = max(beta_PR, 0)
    of eq. CG:PR is never negative."""
    p, phi0 = _fast_rotation_32()
    rep = _solve_with_iterates(p, phi0, 40)
    dirs = _directions(p, rep)
    assert len(dirs) == 40
    assert sum(d["fallback"] for d in dirs) >= 1
    assert any(d["n"] > 0 and d["beta"] == 0.0 and not d["fallback"] for d in dirs)  # a PR restart happened
    for d in dirs:
        assert O.inner(p, d["r"], d["q"]).real < 0.0, d["n"]
        assert d["beta"] >= 0.0, d["n"]
    E = [e["E"] for e in rep["log"]]
    assert all(b < a for a, b in zip(E, E[1:]))


def test_P16_restart_and_fallback_take_the_preconditioned_gradient():
    """When beta = 0 (first step, PR restart, or the descent-check fallback) the step is
    the projected preconditioned gradient, p = -(P r - Re<P r, phi> phi) with P = P_C and
    alpha = lambda~ (pinned by P6, P15); with beta > 0 the direction differs from it."""
    p, phi0 = _fast_rotation_32()
    rep = _solve_with_iterates(p, phi0, 40)
    n_gradient = 0
    for d in _directions(p, rep):
        phi = d["phi"]
        Pr = O.precond_C(p, phi, d["r"], O.lambda_tilde(p, phi))
        g = -(Pr - O.inner(p, Pr, phi).real * phi)
        c = _cosine(p, g, d["q"])
        if d["beta"] == 0.0:
            n_gradient += 1
            assert c > 1.0 - 1e-10, (d["n"], c)
        else:
            assert c < 1.0 - 1e-6, (d["n"], c)
    assert n_gradient >= 3


@pytest.mark.parametrize("line_search", ["model", "exact"])
def test_P16_polak_ribiere_directions_are_secant_conjugate(line_search):
    """With (near-)exact line searches the Polak-Ribiere coefficient equals the
    Hestenes-Stiefel one, whose defining property is that the new direction is
    orthogonal to the change of gradient, Re<r_n - r_{n-1}, d_n> = 0 (the linear-case
    equivalence the paper states under eq. CG:FR).  On the sphere this holds up to
    O(theta) terms, so once the steps are small |cos(r_n - r_{n-1}, q_n)| is small,
    whereas for example the Fletcher-Reeves rule leaves it of order 0.1-0.5 here."""
    w = I.workload("c64_2d")
    p = O.Problem(w["n"], w["L"], w["eta"], w["omega"], w["V"])
    rep = _solve_with_iterates(p, w["phi0"], 60, line_search=line_search)
    assert rep["status"] == "converged"
    dirs = _directions(p, rep)
    checked = 0
    for prev, d in zip(dirs, dirs[1:]):
        if prev["theta"] < 1e-3 and d["beta"] > 0.0 and not d["fallback"]:
            y = d["r"] - prev["r"]
            assert abs(_cosine(p, y, d["q"])) < 1e-2, (d["n"], _cosine(p, y, d["q"]))
            checked += 1
    assert checked >= 15


def test_P16_trial_step_is_the_newton_step_of_the_energy_along_the_geodesic():
    """eq. theta_opt: theta_0 minimises the second-order expansion of
    t -> E(cos t phi_n + sin t q_n), i.e. theta_0 = -E'(0) / E''(0), taken here by
    central differences of the energy (P5 pins the expansion).  Section 5.2 reports
    that near a minimum this step always decreases the energy, so no backtracking
    happens once the residual is small."""
    w = I.workload("c64_2d")
    p = O.Problem(w["n"], w["L"], w["eta"], w["omega"], w["V"])
    rep = _solve_with_iterates(p, w["phi0"], 60)
    assert rep["status"] == "converged"
    checked = 0
    for d in _directions(p, rep):
        res = rep["log"][d["n"]]["res_inf"]
        if res < 1e-3:
            assert d["backtracks"] == 0, d["n"]
        if d["backtracks"] or not (1e-5 < d["theta"] < 0.3):
            continue
        phi, q = d["phi"], d["q"]
        Et = lambda t: O.energy(p, np.cos(t) * phi + np.sin(t) * q)  # noqa: E731
        # central differences with one Richardson step (errors O(h^4)); h = 1e-3 keeps
        # the cancellation in E(h) - 2E(0) + E(-h) below 1e-9 relative
        E0, h = Et(0.0), 1e-3
        Ep = {k: Et(k * h) for k in (-2, -1, 1, 2)}
        e1 = (8 * (Ep[1] - Ep[-1]) - (Ep[2] - Ep[-2])) / (12 * h)
        e2 = (16 * (Ep[1] + Ep[-1]) - (Ep[2] + Ep[-2]) - 30 * E0) / (12 * h * h)
        assert e2 > 0
        assert abs(d["theta"] + e1 / e2) < 1e-5 * d["theta"], (d["n"], d["theta"], -e1 / e2)
        checked += 1
    assert checked >= 5


def test_P16_conjugate_gradient_beats_the_gradient_method():
    """Section 6 reports that PCG_C needs far fewer iterations than PG_C (the projected
    gradient method of Algorithm 1 with the same preconditioner and step rule) on the
    2D rotating problems; both reach the same ground state."""
    w = I.workload("c64_2d")
    p = O.Problem(w["n"], w["L"], w["eta"], w["omega"], w["V"])
    _, cg = O.pcg_solve(p, w["phi0"], O.SolveOptions(tol_res_inf=1e-8, max_iter=1000))
    _, pg = O.pcg_solve(p, w["phi0"], O.SolveOptions(tol_res_inf=1e-8, max_iter=1000, cg=False))
    assert cg["status"] == "converged" and pg["status"] == "converged"
    assert abs(cg["E"] - pg["E"]) < 1e-10 * abs(cg["E"])
    assert 2 * cg["iters"] < pg["iters"]
