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
    lambda: P.test_P13_thomas_fermi_mu_matches_the_continuum_closed_form_2d((1.0, 1.5)),
    lambda: P.test_P15_lambda_tilde_closed_forms(100.0, 0.7),
    P.test_P16_every_step_descends_and_beta_is_nonnegative,
    P.test_P16_restart_and_fallback_take_the_preconditioned_gradient,
    lambda: P.test_P16_polak_ribiere_directions_are_secant_conjugate("model"),
    P.test_P16_trial_step_is_the_newton_step_of_the_energy_along_the_geodesic,
    P.test_P16_conjugate_gradient_beats_the_gradient_method,
]


def pins_all_pass():
    for pin in QUICK_PINS:
        try:
            pin()
        except (AssertionError, ValueError, FloatingPointError, ZeroDivisionError):
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


# --- the shift lambda~ (eq. Opt_Alpha) and the scalar logic of Algorithm 2
def _lt_half_eta(prob, phi):
    kin = O.inner(prob, phi, -0.5 * O.laplacian(prob, phi)).real
    pot = O.inner(prob, phi, prob.V * phi).real
    return kin + pot + 0.5 * prob.eta * prob.weight * np.sum(np.abs(phi) ** 4)


def _lt_with_rotation(prob, phi):
    return O.chemical_potential(prob, phi)


def _beta_without_max(prob, r, r_prev, Pr, rPr_prev, rule):
    return O.inner(prob, r - r_prev, Pr).real / rPr_prev


def _beta_r_n_numerator(prob, r, r_prev, Pr, rPr_prev, rule):
    return max(O.inner(prob, r, Pr).real / rPr_prev, 0.0)


def _theta_half_curvature(m, curv, theta_default):
    return -m["R"] / (0.5 * curv) if curv > 0.0 else theta_default


def _never_fallback(prob, Hphi, p):
    return True


def _fallback_inverted(prob, Hphi, p):
    return 2.0 * O.inner(prob, Hphi, p).real >= 0.0


# --- further single-function mistakes, one per remaining oracle function
_orig_dft = O.dft_axis
_orig_coord = O.Problem.coord


def _dft_inverse_unscaled(prob, f, i, inverse=False):
    g = _orig_dft(prob, f, i, inverse)
    return g * f.shape[prob.axis(i)] if inverse else g


def _coord_shifted(self, i):
    return _orig_coord(self, i) + self.h[i]


def _laplacian_one_axis(prob, f):
    return O.d2_axis(prob, f, 0)


def _A_without_V(prob, f):
    return -0.5 * O.laplacian(prob, f) - prob.omega * O.Lz(prob, f)


def _energy_full_interaction(prob, phi):
    kin = O.inner(prob, phi, -0.5 * O.laplacian(prob, phi)).real
    pot = O.inner(prob, phi, prob.V * phi).real
    inter = prob.eta * prob.weight * np.sum(np.abs(phi) ** 4)
    rot = O.inner(prob, phi, -prob.omega * O.Lz(prob, phi)).real
    return dict(kin=kin, pot=pot, int=inter, rot=rot, total=kin + pot + inter + rot)


def _lambda_linear_part(prob, phi):
    return O.inner(prob, phi, O.apply_A(prob, phi)).real


def _kinetic_symbol_no_half(prob):
    return sum(prob.freq(i) ** 2 for i in range(prob.dim))


def _pv_without_eta(prob, phi, alpha):
    return 1.0 / (alpha + prob.V)


_orig_moments = O.step_moments


def _moments_R_sign(prob, phi, Hphi, lam, q):
    m = _orig_moments(prob, phi, Hphi, lam, q)
    m["R"] = -m["R"]
    return m


def _exact_step_is_model_step(m, eta, theta0, iters=30):
    return theta0


def _tf_mu_half_eta(prob, iters=200):
    V, w, eta = prob.V, prob.weight, 0.5 * prob.eta
    lo, hi = float(V.min()), float(V.max()) + eta / (w * V.size)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if w * np.sum(np.maximum(mid - V, 0.0)) / eta < 1.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _interpolate_axes_swapped(prob_c, phi_c, prob_f):
    g = phi_c
    for i in range(prob_c.dim):
        g = O.interpolate_axis(g, i, prob_f.n[i])
    return g


def _project_nothing(prob, phi, h):
    return h.copy()


_orig_tsolve = O.tangent_solve


def _tangent_solve_half(prob, phi, lam, rhs, tol=1e-12, max_iter=5000, alpha=None):
    z, it, res = _orig_tsolve(prob, phi, lam, rhs, tol, max_iter, alpha)
    return 0.5 * z, it, res


def _density_loss_unweighted(prob, phi, rho):
    return np.sum((np.abs(phi) ** 2 - rho) ** 2)


MUTATIONS = {
    "lt_half_eta": ("lambda_tilde", _lt_half_eta),
    "lt_with_rotation": ("lambda_tilde", _lt_with_rotation),
    "beta_without_max": ("conjugation_coefficient", _beta_without_max),
    "beta_r_n_numerator": ("conjugation_coefficient", _beta_r_n_numerator),
    "theta_half_curvature": ("trial_step", _theta_half_curvature),
    "never_fallback": ("is_descent_direction", _never_fallback),
    "fallback_inverted": ("is_descent_direction", _fallback_inverted),
    "dft_inverse_unscaled": ("dft_axis", _dft_inverse_unscaled),
    "laplacian_one_axis": ("laplacian", _laplacian_one_axis),
    "A_without_V": ("apply_A", _A_without_V),
    "energy_full_interaction": ("energy_parts", _energy_full_interaction),
    "lambda_linear_part": ("chemical_potential", _lambda_linear_part),
    "kinetic_symbol_no_half": ("kinetic_symbol", _kinetic_symbol_no_half),
    "pv_without_eta": ("precond_V", _pv_without_eta),
    "moments_R_sign": ("step_moments", _moments_R_sign),
    "exact_step_is_model_step": ("exact_step", _exact_step_is_model_step),
    "tf_mu_half_eta": ("thomas_fermi_mu", _tf_mu_half_eta),
    "interpolate_axes_swapped": ("interpolate", _interpolate_axes_swapped),
    "project_nothing": ("tangent_project", _project_nothing),
    "tangent_solve_half": ("tangent_solve", _tangent_solve_half),
    "density_loss_unweighted": ("density_loss", _density_loss_unweighted),
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


@pytest.mark.parametrize("attr,fn", [("freq", _freq_twice), ("coord", _coord_shifted)])
def test_problem_method_mutation_is_caught(attr, fn):
    orig = getattr(O.Problem, attr)
    setattr(O.Problem, attr, fn)
    try:
        assert not pins_all_pass()
    finally:
        setattr(O.Problem, attr, orig)
