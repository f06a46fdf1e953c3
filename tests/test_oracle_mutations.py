"""Planted mistakes in the oracle must each break at least one pin.

Each case patches one plausible error into oracle.gpe_oracle (on the CPU) and
re-runs the quick pins from test_oracle_pins; the test passes only if some pin
now fails.  This checks that the pins constrain every part of the oracle.
"""
import contextlib

import numpy as np
import pytest

from oracle import gpe_oracle as O

import test_oracle_pins as P

QUICK_PINS = [
    lambda: P.test_P0_spectral_derivative_of_single_mode(0),
    P.test_P1_harmonic_gaussian_2d,
    P.test_P2_angular_momentum_sign_and_scale,
    lambda: P.test_P3_hamiltonian_hermitian((16, 16)),
    P.test_P4_gradient_is_two_H_phi,
    P.test_P5_exact_energy_change_along_geodesic,
    P.test_P5_curvature_matches_second_difference,
    lambda: P.test_P6_preconditioner_hermitian_positive((16, 16)),
    P.test_P6_kinetic_preconditioner_inverts_shifted_laplacian,
    P.test_P10_energy_gradient_matches_central_differences,
    lambda: P.test_P10_parameter_derivatives_match_central_differences(0.0),
    lambda: P.test_P11_hellmann_feynman_matches_differences_of_solves(P.solve_ground_state_16()),
    lambda: P.test_P12_hessian_operator_is_the_second_order_form(P.solve_ground_state_16()),
    lambda: P.test_P12_density_loss_gradient_matches_differences_of_solves(P.solve_ground_state_16()),
    P.test_P6_preconditioner_variants_adjointness,
    P.test_P5_line_search_derivatives_match_differences,
    P.test_P5_exact_step_minimises_the_energy_along_the_geodesic,
    lambda: P.test_P14_interpolation_is_exact_for_band_limited_fields((16, 8), (32, 16)),
]


def pins_all_pass():
    for pin in QUICK_PINS:
        try:
            pin()
        except AssertionError:
            return False
    return True


@contextlib.contextmanager
def patched(name, fn):
    old = getattr(O, name)
    setattr(O, name, fn)
    try:
        yield
    finally:
        setattr(O, name, old)


def _lz_wrong_sign(prob, f):
    x, y = prob.coord(0), prob.coord(1)
    return 1j * (x * O.d1_axis(prob, f, 1) - y * O.d1_axis(prob, f, 0))


def _lz_swapped_axes(prob, f):
    x, y = prob.coord(0), prob.coord(1)
    return -1j * (x * O.d1_axis(prob, f, 0) - y * O.d1_axis(prob, f, 1))


def _inner_unweighted(prob, f, g):
    return np.vdot(f, g)


_orig_apply_H = O.apply_H
_orig_freq = O.Problem.freq


def _H_without_nonlinearity(prob, phi, f):
    return O.apply_A(prob, f)


def _H_with_half_nonlinearity(prob, phi, f):
    return O.apply_A(prob, f) + 0.5 * prob.eta * np.abs(phi) ** 2 * f


def _hessian_as_printed(prob, phi, f):
    # the formula exactly as printed: <f, H f> + eta Re <phi^2, f^2>
    w = prob.weight
    return (O.inner(prob, f, _orig_apply_H(prob, phi, f)).real
            + prob.eta * w * np.sum(np.conj(phi) ** 2 * f ** 2).real)


_orig_delta = O.delta_energy


def _delta_wrong_coefficient(m, eta, theta):
    c, s = np.cos(theta), np.sin(theta)
    return _orig_delta(m, eta, theta) - 0.5 * eta * 2.0 * c * s ** 3 * (m["VW"] - m["U1"])


def _precond_nonsymmetric(prob, phi, r, alpha):
    return O.precond_V(prob, phi, alpha) * O.precond_delta(prob, r, alpha)


def _delta_shift_wrong(prob, f, alpha):
    return O.dftn(prob, O.dftn(prob, f) / (alpha + 2.0 * O.kinetic_symbol(prob)), inverse=True)


def _freq_twice(self, i):
    return 2.0 * _orig_freq(self, i)


_orig_grad = O.energy_gradient
_orig_pderiv = O.energy_parameter_derivatives
_orig_hess = O.hessian_apply
_orig_dloss = O.density_loss_gradient_V


def _grad_unweighted(prob, phi):
    return _orig_grad(prob, phi) / prob.weight


def _domega_wrong_sign(prob, phi):
    d = _orig_pderiv(prob, phi)
    d["domega"] = -d["domega"]
    return d


def _deta_without_half(prob, phi):
    d = _orig_pderiv(prob, phi)
    d["deta"] = 2.0 * d["deta"]
    return d


def _hessian_without_conjugate_term(prob, phi, lam, f):
    return _orig_hess(prob, phi, lam, f) - prob.eta * phi ** 2 * np.conj(f)


def _dloss_wrong_sign(prob, phi, rho, tol=1e-12, max_iter=5000):
    g, it, res = _orig_dloss(prob, phi, rho, tol, max_iter)
    return -g, it, res


_orig_apply_pc = O.apply_preconditioner


def _c2_as_c1(prob, phi, r, alpha, kind):
    return _orig_apply_pc(prob, phi, r, alpha, "C1" if kind == "C2" else kind)


def _pv_sqrt(prob, phi, r, alpha, kind):
    if kind == "V":
        return np.sqrt(O.precond_V(prob, phi, alpha)) * r
    return _orig_apply_pc(prob, phi, r, alpha, kind)


_orig_dderiv = O.delta_energy_derivatives


def _dderiv_wrong_quartic(m, eta, theta):
    d1, d2 = _orig_dderiv(m, eta, theta)
    c, s_ = np.cos(theta), np.sin(theta)
    B = 0.5 * eta * (m["U0"] + m["W2"])
    return d1 - 2.0 * B * s_ ** 3 * c, d2


def _interp_nyquist_unsplit(f, axis, Mf):
    Mc = f.shape[axis]
    if Mf == Mc:
        return f.copy()
    F = np.fft.fft(f, axis=axis)
    shape = list(f.shape)
    shape[axis] = Mf
    G = np.zeros(shape, dtype=complex)
    h = Mc // 2
    idx = lambda a, b: tuple(slice(a, b) if k == axis else slice(None) for k in range(f.ndim))  # noqa: E731
    G[idx(0, h)] = F[idx(0, h)]
    G[idx(Mf - h, Mf)] = F[idx(h, Mc)]  # Nyquist kept at -Mc/2 only
    return np.fft.ifft(G, axis=axis) * (Mf / Mc)


MUTATIONS = {
    "Lz_sign": ("Lz", _lz_wrong_sign),
    "Lz_axes": ("Lz", _lz_swapped_axes),
    "no_weight": ("inner", _inner_unweighted),
    "H_no_eta": ("apply_H", _H_without_nonlinearity),
    "H_half_eta": ("apply_H", _H_with_half_nonlinearity),
    "hessian_as_printed": ("hessian_form", _hessian_as_printed),
    "deltaE_coeff": ("delta_energy", _delta_wrong_coefficient),
    "P_nonsymmetric": ("precond_C", _precond_nonsymmetric),
    "P_delta_shift": ("precond_delta", _delta_shift_wrong),
    "grad_unweighted": ("energy_gradient", _grad_unweighted),
    "domega_sign": ("energy_parameter_derivatives", _domega_wrong_sign),
    "deta_no_half": ("energy_parameter_derivatives", _deta_without_half),
    "hessian_no_conj": ("hessian_apply", _hessian_without_conjugate_term),
    "dloss_sign": ("density_loss_gradient_V", _dloss_wrong_sign),
    "pc_c2_as_c1": ("apply_preconditioner", _c2_as_c1),
    "pc_v_sqrt": ("apply_preconditioner", _pv_sqrt),
    "line_deriv_quartic": ("delta_energy_derivatives", _dderiv_wrong_quartic),
    "interp_nyquist": ("interpolate_axis", _interp_nyquist_unsplit),
}


def test_unmutated_oracle_passes_quick_pins():
    assert pins_all_pass()


@pytest.mark.parametrize("case", sorted(MUTATIONS))
def test_mutation_is_caught(case):
    name, fn = MUTATIONS[case]
    with patched(name, fn):
        assert not pins_all_pass(), f"planted mistake {case} passed every pin"


def test_frequency_scale_mutation_is_caught():
    O.Problem.freq = _freq_twice
    try:
        assert not pins_all_pass()
    finally:
        O.Problem.freq = _orig_freq
