"""Plain FP64 CPU oracle for the PCG_C ground-state method of Antoine, Levitt
and Tang (arXiv:1611.02045).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
module: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
reference legs use it.  It shares no code with the CUDA library; it is slow and
written so that each step can be checked against the paper by eye.

Conventions (paper Section 3):
  * grid x_k = -L + k h, h = 2L/M, arrays [z][y][x] (x = last numpy axis);
  * frequencies xi_p = p pi / L for p = -M/2 .. M/2-1, stored in DFT order
    (index p and p - M name the same mode), Nyquist kept as -M pi / (2L);
  * forward DFT unnormalised with e^{-2 pi i p k / M}, inverse with 1/M.
Readings of the paper that this file relies on (all listed in the design
notes): inner products carry the weight h^d (R1); the Hessian form includes
eta int |phi|^2 |f|^2 (R3); the step-size model and its default/backtracking
constants (R4, R5); the energy-decrease test is evaluated in exact
trigonometric-polynomial form from moments (R6); beta uses the stored
<r_{n-1}, P_{n-1} r_{n-1}> (R7).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# Discretisation (Section 3)
# --------------------------------------------------------------------------


@dataclass
class Problem:
    """Discrete rotating GP problem: grid sizes n = (nx, ny[, nz]), half-widths
    L, nonlinearity eta, rotation omega about z, real potential V on the grid."""

    n: tuple
    L: tuple
    eta: float
    omega: float
    V: np.ndarray
    backend: str = "fft"  # "fft" (numpy pocketfft) or "naive" (explicit DFT sums)
    _cache: dict = field(default_factory=dict, repr=False)

    @property
    def dim(self):
        return len(self.n)

    @property
    def h(self):
        return tuple(2.0 * L / n for n, L in zip(self.n, self.L))

    @property
    def weight(self):
        """h^d: the quadrature weight of the discrete inner product (R1)."""
        return float(np.prod(self.h))

    def axis(self, i):
        """numpy axis holding physical axis i (0 = x, 1 = y, 2 = z)."""
        return self.dim - 1 - i

    def coord(self, i):
        """x_k = -L + k h for axis i, broadcast along numpy axis `axis(i)`."""
        x = -self.L[i] + np.arange(self.n[i]) * self.h[i]
        shape = [1] * self.dim
        shape[self.axis(i)] = self.n[i]
        return x.reshape(shape)

    def freq(self, i):
        """xi_p = p pi / L in DFT order, Nyquist mode p = -M/2 kept (R2)."""
        M = self.n[i]
        p = np.arange(M)
        p = np.where(p < M // 2, p, p - M)
        xi = p * np.pi / self.L[i]
        shape = [1] * self.dim
        shape[self.axis(i)] = M
        return xi.reshape(shape)


def _dft_matrix(M, sign):
    k = np.arange(M)
    return np.exp(sign * 2j * np.pi * np.outer(k, k) / M)


def dft_axis(prob: Problem, f, i, inverse=False):
    """1-D transform along physical axis i: forward sum_k f_k e^{-2pi i pk/M},
    inverse (1/M) sum_p g_p e^{+2pi i pk/M} (Section 3)."""
    ax = prob.axis(i)
    if prob.backend == "fft":
        return np.fft.ifft(f, axis=ax) if inverse else np.fft.fft(f, axis=ax)
    M = f.shape[ax]
    F = _dft_matrix(M, +1.0 if inverse else -1.0)
    g = np.moveaxis(np.tensordot(F, np.moveaxis(f, ax, 0), axes=(1, 0)), 0, ax)
    return g / M if inverse else g


def dftn(prob: Problem, f, inverse=False):
    """Full d-dimensional transform as successive 1-D transforms."""
    for i in range(prob.dim):
        f = dft_axis(prob, f, i, inverse)
    return f


def d2_axis(prob, f, i):
    """[[d^2/dx_i^2]] f: -(1/M) sum_p xi_p^2 fhat_p e^{i xi_p (x+L)} (eq. FFTdiscret)."""
    return dft_axis(prob, -(prob.freq(i) ** 2) * dft_axis(prob, f, i), i, inverse=True)


def d1_axis(prob, f, i):
    """[[d/dx_i]] f: (1/M) sum_p i xi_p fhat_p e^{i xi_p (x+L)} (eq. FFTdiscret)."""
    return dft_axis(prob, 1j * prob.freq(i) * dft_axis(prob, f, i), i, inverse=True)


def laplacian(prob, f):
    """[[Delta]] = sum over axes of [[d^2/dx_i^2]]."""
    return sum(d2_axis(prob, f, i) for i in range(prob.dim))


def Lz(prob, f):
    """[[L_z]] = -i (x [[d_y]] - y [[d_x]]) (Section 3; L_z = i(y d_x - x d_y), Section 2)."""
    x, y = prob.coord(0), prob.coord(1)
    return -1j * (x * d1_axis(prob, f, 1) - y * d1_axis(prob, f, 0))


# --------------------------------------------------------------------------
# Operators and functionals (Sections 2, 3 and 5.5)
# --------------------------------------------------------------------------


def inner(prob, f, g):
    """<f, g> = h^d sum conj(f) g (reading R1)."""
    return prob.weight * np.vdot(f, g)


def norm(prob, f):
    return np.sqrt(inner(prob, f, f).real)


def apply_A(prob, f):
    """Linear part A f = -1/2 Delta f + V f - omega L_z f."""
    return -0.5 * laplacian(prob, f) + prob.V * f - prob.omega * Lz(prob, f)


def apply_H(prob, phi, f):
    """Mean-field Hamiltonian H_phi f = A f + eta |phi|^2 f (Section 2)."""
    return apply_A(prob, f) + prob.eta * np.abs(phi) ** 2 * f


def energy_parts(prob, phi):
    """E(phi) = int 1/2|grad phi|^2 + V|phi|^2 + eta/2 |phi|^4 - omega phi* L_z phi
    (Section 2), each integral as its discrete inner product."""
    kin = inner(prob, phi, -0.5 * laplacian(prob, phi)).real
    pot = inner(prob, phi, prob.V * phi).real
    inter = 0.5 * prob.eta * prob.weight * np.sum(np.abs(phi) ** 4)
    rot = inner(prob, phi, -prob.omega * Lz(prob, phi)).real
    return dict(kin=kin, pot=pot, int=inter, rot=rot, total=kin + pot + inter + rot)


def energy(prob, phi):
    return energy_parts(prob, phi)["total"]


def chemical_potential(prob, phi):
    """lambda = <H_phi phi, phi> (Section 2)."""
    return inner(prob, phi, apply_H(prob, phi, phi)).real


def lambda_tilde(prob, phi):
    """Adaptive shift int 1/2|grad phi|^2 + V|phi|^2 + eta|phi|^4 (eq. Opt_Alpha)."""
    kin = inner(prob, phi, -0.5 * laplacian(prob, phi)).real
    pot = inner(prob, phi, prob.V * phi).real
    return kin + pot + prob.eta * prob.weight * np.sum(np.abs(phi) ** 4)


def hessian_form(prob, phi, f):
    """1/2 grad^2 E(phi)[f, f] = <f, H_phi f> + eta int |phi|^2|f|^2 + eta Re int conj(phi)^2 f^2
    (Section 2 with the term the paper's formula omits, reading R3)."""
    w = prob.weight
    return (inner(prob, f, apply_H(prob, phi, f)).real
            + prob.eta * w * np.sum(np.abs(phi) ** 2 * np.abs(f) ** 2)
            + prob.eta * w * np.sum(np.conj(phi) ** 2 * f ** 2).real)


def kinetic_symbol(prob):
    """1/2 |k|^2 on the full d-dimensional frequency grid."""
    return 0.5 * sum(prob.freq(i) ** 2 for i in range(prob.dim))


def precond_delta(prob, f, alpha):
    """P_Delta f = (alpha - Delta/2)^{-1} f, diagonal in Fourier space (eq. PDelta)."""
    return dftn(prob, dftn(prob, f) / (alpha + kinetic_symbol(prob)), inverse=True)


def precond_V(prob, phi, alpha):
    """Diagonal of P_V = (alpha + V + eta |phi|^2)^{-1} (eq. PV)."""
    return 1.0 / (alpha + prob.V + prob.eta * np.abs(phi) ** 2)


def precond_C(prob, phi, r, alpha):
    """Symmetric combined preconditioner P_V^{1/2} P_Delta P_V^{1/2} (eq. combinedP_12)."""
    s = np.sqrt(precond_V(prob, phi, alpha))
    return s * precond_delta(prob, s * r, alpha)


def apply_preconditioner(prob, phi, r, alpha, kind):
    """P r for the preconditioners of Section 5.4, all with the shift alpha:
    "C" P_V^{1/2} P_Delta P_V^{1/2} (eq. combinedP_12), "Delta" P_Delta (eq. PDelta),
    "V" P_V (eq. PV), "C1" P_V P_Delta and "C2" P_Delta P_V (eq. combinedP; the
    right factor acts first), "none" the identity."""
    if kind == "C":
        return precond_C(prob, phi, r, alpha)
    if kind == "Delta":
        return precond_delta(prob, r, alpha)
    if kind == "V":
        return precond_V(prob, phi, alpha) * r
    if kind == "C1":
        return precond_V(prob, phi, alpha) * precond_delta(prob, r, alpha)
    if kind == "C2":
        return precond_delta(prob, precond_V(prob, phi, alpha) * r, alpha)
    if kind == "none":
        return r.copy()
    raise ValueError(kind)


# --------------------------------------------------------------------------
# Line search along the geodesic (Section 5.1, readings R4-R6)
# --------------------------------------------------------------------------


def step_moments(prob, phi, Hphi, lam, q):
    """Scalars that fix E(cos t phi + sin t q) as a trigonometric polynomial in t.

    R = Re<H phi, q>,  aqq = <q, A q>,  and with u = |phi|^2, v = Re(conj(phi) q),
    w = |q|^2 the integrals U0 = int u^2, U1 = int u v, V2 = int v^2,
    UW = int u w, VW = int v w, W2 = int w^2.
    """
    wgt = prob.weight
    u = np.abs(phi) ** 2
    v = (np.conj(phi) * q).real
    w = np.abs(q) ** 2
    return dict(
        R=inner(prob, Hphi, q).real,
        aqq=inner(prob, q, apply_A(prob, q)).real,
        lam=lam,
        U0=wgt * np.sum(u * u), U1=wgt * np.sum(u * v), V2=wgt * np.sum(v * v),
        UW=wgt * np.sum(u * w), VW=wgt * np.sum(v * w), W2=wgt * np.sum(w * w),
        rho=inner(prob, phi, q).real,
    )


def delta_energy(m, eta, theta):
    """E(cos t phi + sin t q) - E(phi), exact for ||q|| arbitrary (reading R6):

        2cs R + s^2 (aqq - lam)
        + eta/2 [ s^4 (U0 + W2) + c^2 s^2 (4 V2 + 2 UW) + 4 c s^3 (VW - U1) ].

    Obtained by expanding <phi_t, A phi_t> + eta/2 int |phi_t|^4 with
    Re<phi, A q> = R - eta U1 and <phi, A phi> = lam - eta U0; no term is
    dropped, so it equals the direct energy difference up to rounding while
    staying accurate when the difference is far below |E| * machine epsilon.
    """
    c, s = np.cos(theta), np.sin(theta)
    return (2.0 * c * s * m["R"] + s * s * (m["aqq"] - m["lam"])
            + 0.5 * eta * (s ** 4 * (m["U0"] + m["W2"])
                           + c * c * s * s * (4.0 * m["V2"] + 2.0 * m["UW"])
                           + 4.0 * c * s ** 3 * (m["VW"] - m["U1"])))


def delta_energy_derivatives(m, eta, theta):
    """First and second derivatives in t of delta_energy (same moments): with
    c = cos t, s = sin t, A = aqq - lam, B = eta/2 (U0 + W2), C = eta/2 (4 V2 + 2 UW),
    D = 2 eta (VW - U1), delta_energy = 2cs R + s^2 A + s^4 B + c^2 s^2 C + c s^3 D and
        d/dt   = 2R cos 2t + A sin 2t + 4B s^3 c + C/2 sin 4t + D (3 c^2 s^2 - s^4),
        d2/dt2 = -4R sin 2t + 2A cos 2t + 4B (3 s^2 c^2 - s^4) + 2C cos 4t + D (6 c s (c^2 - s^2) - 4 s^3 c)."""
    c, s = np.cos(theta), np.sin(theta)
    A = m["aqq"] - m["lam"]
    B = 0.5 * eta * (m["U0"] + m["W2"])
    C = 0.5 * eta * (4.0 * m["V2"] + 2.0 * m["UW"])
    D = 2.0 * eta * (m["VW"] - m["U1"])
    R = m["R"]
    d1 = (2.0 * R * np.cos(2 * theta) + A * np.sin(2 * theta) + 4.0 * B * s ** 3 * c + 0.5 * C * np.sin(4 * theta)
          + D * (3.0 * c * c * s * s - s ** 4))
    d2 = (-4.0 * R * np.sin(2 * theta) + 2.0 * A * np.cos(2 * theta) + 4.0 * B * (3.0 * s * s * c * c - s ** 4)
          + 2.0 * C * np.cos(4 * theta) + D * (6.0 * c * s * (c * c - s * s) - 4.0 * s ** 3 * c))
    return d1, d2


def exact_step(m, eta, theta0, iters=30):
    """The step minimising delta_energy near theta0 ("full line search" variant):
    Newton's method on d/dt delta_energy = 0 from theta0, stopping when the
    update is below 1e-15 |t|; returns theta0 when the curvature is not positive
    or the iteration leaves (0, pi/2]."""
    t = theta0
    for _ in range(iters):
        d1, d2 = delta_energy_derivatives(m, eta, t)
        if not d2 > 0.0:
            return theta0
        dt = d1 / d2
        t = t - dt
        if not (0.0 < t <= 0.5 * np.pi):
            return theta0
        if abs(dt) <= 1e-15 * abs(t):
            break
    return t


def model_curvature(prob, phi, lam, q):
    """T2(q) - lambda: the theta^2 coefficient of the energy along the geodesic
    (eq. expansion_energy read as E + 2t Re<r,q> + t^2 (T2(q) - lambda), R4)."""
    return hessian_form(prob, phi, q) - lam


# --------------------------------------------------------------------------
# PCG (Algorithm 2 with the descent check of Section 5.2)
# --------------------------------------------------------------------------


@dataclass
class SolveOptions:
    tol_res_inf: float = 1e-8      # stop when ||r_n||_inf < tol (eq. Stop_Residual)
    tol_dE: float = 0.0            # optional |E_{n+1} - E_n| <= tol (eq. Stop_Energy)
    max_iter: int = 20000
    theta_default: float = 0.1     # trial step when the model curvature is <= 0 (R5)
    max_backtracks: int = 30       # theta <- theta/2 at most this many times (R5)
    precond: str = "C"             # "C", "Delta", "V", "C1", "C2" or "none" (apply_preconditioner)
    beta: str = "PR"               # "PR": max(beta_PR, 0) (eq. CG:PR); "FR": Fletcher-Reeves (eq. CG:FR)
    line_search: str = "model"     # "model": theta_0 of R4 + backtracking; "exact": Newton from theta_0
    cg: bool = True                # False: the projected gradient method (Algorithm 1)


def conjugation_coefficient(prob, r, r_prev, Pr, rPr_prev, rule):
    """beta_n of Section 5.3 (R7): "PR" is beta+ = max(beta_PR, 0) with
    beta_PR = Re<r_n - r_{n-1}, P_n r_n> / <r_{n-1}, P_{n-1} r_{n-1}> (eq. CG:PR),
    "FR" is <r_n, P_n r_n> / <r_{n-1}, P_{n-1} r_{n-1}> (eq. CG:FR)."""
    if rule == "FR":
        return inner(prob, r, Pr).real / rPr_prev
    return max(inner(prob, r - r_prev, Pr).real / rPr_prev, 0.0)


def is_descent_direction(prob, Hphi, p):
    """Section 5.2: p is a descent direction iff Re<grad E(phi), p> = 2 Re<H_phi phi, p> < 0."""
    return 2.0 * inner(prob, Hphi, p).real < 0.0


def trial_step(m, curv, theta_default):
    """theta_0 of eq. theta_opt under reading R4: the minimiser -Re<r,q> / (T2(q) - lambda)
    of the second-order expansion when its curvature is positive (Re<r,q> = Re<H phi, q>
    since Re<phi, q> = 0), else the default step of R5."""
    return -m["R"] / curv if curv > 0.0 else theta_default


def pcg_solve(prob: Problem, phi0, opts: SolveOptions | None = None, keep_iterates=()):
    """Run PCG_C from phi0.  Returns (phi, report) where report['log'] holds one
    dict per iteration n (E_n, lambda_n, ||r_n||_inf, alpha_n, beta_n, theta_n,
    backtracks, fallback) and report['iterates'][n] = phi_n for n in keep_iterates."""
    opts = opts or SolveOptions()
    phi = phi0 / norm(prob, phi0)
    p_prev = r_prev = None
    rPr_prev = None
    log, iterates = [], {}
    status = "not_converged"
    n = 0
    while True:
        if n in keep_iterates:
            iterates[n] = phi.copy()
        Hphi = apply_H(prob, phi, phi)
        lam = inner(prob, phi, Hphi).real                  # lambda_n
        r = Hphi - lam * phi                               # r_n
        res_inf = np.max(np.abs(r))
        E = energy(prob, phi)
        entry = dict(n=n, E=E, lam=lam, res_inf=res_inf,
                     res_l2=norm(prob, r))
        log.append(entry)
        if not np.isfinite(E) or not np.isfinite(res_inf):
            status = "nonfinite"
            break
        if res_inf < opts.tol_res_inf:
            status = "converged"
            break
        if n >= opts.max_iter:
            break

        alpha = lambda_tilde(prob, phi)                    # eq. Opt_Alpha
        Pr = apply_preconditioner(prob, phi, r, alpha, opts.precond)
        rPr = inner(prob, r, Pr).real
        if not opts.cg or n == 0 or rPr_prev is None:
            beta = 0.0
        else:
            beta = conjugation_coefficient(prob, r, r_prev, Pr, rPr_prev, opts.beta)
        d = -Pr + beta * p_prev if beta != 0.0 else -Pr
        p = d - inner(prob, d, phi).real * phi             # projection M_phi d
        fallback = False
        # Section 5.2: revert to the gradient step when p is not a descent direction.
        if not is_descent_direction(prob, Hphi, p):
            fallback = True
            beta = 0.0
            d = -Pr
            p = d - inner(prob, d, phi).real * phi
        q = p / norm(prob, p)
        m = step_moments(prob, phi, Hphi, lam, q)
        theta = trial_step(m, model_curvature(prob, phi, lam, q), opts.theta_default)
        if opts.line_search == "exact":
            theta = exact_step(m, prob.eta, theta)
        dE = delta_energy(m, prob.eta, theta)
        backtracks = 0
        while not dE < 0.0 and backtracks < opts.max_backtracks:
            theta *= 0.5
            backtracks += 1
            dE = delta_energy(m, prob.eta, theta)
        phi_new = np.cos(theta) * phi + np.sin(theta) * q
        phi_new = phi_new / norm(prob, phi_new)            # renormalise (R9)
        entry.update(alpha=alpha, beta=beta, theta=theta, dE=dE,
                     backtracks=backtracks, fallback=fallback, rPr=rPr)
        phi, p_prev, r_prev, rPr_prev = phi_new, p, r, rPr
        n += 1
        if opts.tol_dE > 0.0 and abs(dE) <= opts.tol_dE:
            if n in keep_iterates:
                iterates[n] = phi.copy()
            Hphi = apply_H(prob, phi, phi)
            lam = inner(prob, phi, Hphi).real
            r = Hphi - lam * phi
            log.append(dict(n=n, E=energy(prob, phi), lam=lam,
                            res_inf=np.max(np.abs(r)), res_l2=norm(prob, r)))
            status = "converged_dE"
            break
    return phi, dict(status=status, iters=n, log=log, iterates=iterates,
                     E=log[-1]["E"], lam=log[-1]["lam"], res_inf=log[-1]["res_inf"])


# --------------------------------------------------------------------------
# Thomas-Fermi initial data (Section 6, eq. TF_App)
# --------------------------------------------------------------------------


def thomas_fermi_mu(prob, iters=200):
    """mu with h^d sum max(mu - V, 0) / eta = 1, i.e. ||phi^TF|| = 1 for
    phi^TF = sqrt(max(mu - V, 0) / eta): bisection on [min V, max V + eta / (h^d N)]."""
    V, w, eta = prob.V, prob.weight, prob.eta
    lo, hi = float(V.min()), float(V.max()) + eta / (w * V.size)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if w * np.sum(np.maximum(mid - V, 0.0)) / eta < 1.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def thomas_fermi_state(prob):
    """phi_0 = phi^TF / ||phi^TF|| of eq. TF_App (with the mu above, ||phi^TF|| = 1)."""
    mu = thomas_fermi_mu(prob)
    phi = np.sqrt(np.maximum(mu - prob.V, 0.0) / prob.eta) + 0j
    return phi / norm(prob, phi), mu


# --------------------------------------------------------------------------
# Spectral interpolation for multigrid continuation (Section 6)
# --------------------------------------------------------------------------


def interpolate_axis(f, axis, Mf):
    """Trigonometric interpolation of f along `axis` from Mc to Mf >= Mc points
    on the same periodic interval: the interpolant
        g(x) = (1/Mc) sum_p F_p e^{i xi_p (x + L)},  F = DFT_Mc(f),
    with the Nyquist term F_{-Mc/2} shared equally by the modes -Mc/2 and +Mc/2
    (so that real data interpolate to real data), sampled at the Mf points."""
    Mc = f.shape[axis]
    if Mf == Mc:
        return f.copy()
    F = np.fft.fft(f, axis=axis)
    shape = list(f.shape)
    shape[axis] = Mf
    G = np.zeros(shape, dtype=complex)
    h = Mc // 2

    def sl(a, b):
        idx = [slice(None)] * f.ndim
        idx[axis] = slice(a, b)
        return tuple(idx)

    G[sl(0, h)] = F[sl(0, h)]
    G[sl(Mf - h + 1, Mf)] = F[sl(h + 1, Mc)]
    G[sl(h, h + 1)] = 0.5 * F[sl(h, h + 1)]
    G[sl(Mf - h, Mf - h + 1)] = 0.5 * F[sl(h, h + 1)]
    return np.fft.ifft(G, axis=axis) * (Mf / Mc)


def interpolate(prob_c, phi_c, prob_f):
    """phi_c on the grid of prob_c interpolated onto the grid of prob_f (same
    domain, each size a multiple of the coarse one), axis by axis."""
    assert tuple(prob_c.L) == tuple(prob_f.L)
    g = phi_c
    for i in range(prob_c.dim):
        g = interpolate_axis(g, prob_c.dim - 1 - i, prob_f.n[i])  # numpy axis of physical axis i
    return g


# --------------------------------------------------------------------------
# Derivatives (Section 2: gradient, Hessian, tangent space of the sphere)
# --------------------------------------------------------------------------


def energy_gradient(prob, phi):
    """Gradient of the discrete energy with respect to the real and imaginary
    parts of the grid values, dE/dRe phi_k + i dE/dIm phi_k.

    Section 2 gives nabla E(phi) = 2 H_phi phi for the weighted inner product
    <f, g> = h^d sum conj(f) g; the coefficient-space gradient carries h^d."""
    return 2.0 * prob.weight * apply_H(prob, phi, phi)


def energy_parameter_derivatives(prob, phi):
    """Partial derivatives of E(phi; V, eta, omega) at fixed phi:
    dE/dV_k = h^d |phi_k|^2, dE/deta = 1/2 int |phi|^4, dE/domega = -<phi, L_z phi>.
    At a normalised critical point the constraint contributes nothing, so these
    are the derivatives of the ground-state energy (Hellmann-Feynman)."""
    w = prob.weight
    return dict(dV=w * np.abs(phi) ** 2,
                deta=0.5 * w * np.sum(np.abs(phi) ** 4),
                domega=-inner(prob, phi, Lz(prob, phi)).real)


def hessian_apply(prob, phi, lam, f):
    """K f = H_phi f + eta |phi|^2 f + eta phi^2 conj(f) - lam f: the operator of
    the form 1/2 grad^2 E(phi)[f, f] - lam ||f||^2 of Section 2 (with the term
    of reading R3), so that Re<f, K f> equals that form.  Real-linear in f."""
    return (apply_H(prob, phi, f) + prob.eta * np.abs(phi) ** 2 * f
            + prob.eta * phi ** 2 * np.conj(f) - lam * f)


def tangent_project(prob, phi, h):
    """Projection onto {h : <phi, h> = 0} for ||phi|| = 1: the tangent space
    Re<phi, h> = 0 of Section 2 (projector M_phi) with the phase direction
    i phi removed as well, since E and every density functional are invariant
    under phi -> e^{i a} phi, so K (i phi) = 0 at a critical point."""
    return h - inner(prob, phi, h) * phi


def tangent_solve(prob, phi, lam, rhs, tol=1e-12, max_iter=5000, alpha=None):
    """Solve K z = rhs for z with <phi, z> = 0 (rhs projected first), by the
    conjugate gradient method in the real inner product Re<.,.>, preconditioned
    by the projected P_C of eq. combinedP_12 (shift alpha, default lambda~ of
    eq. Opt_Alpha).  Returns (z, iterations, relative residual)."""
    if alpha is None:
        alpha = lambda_tilde(prob, phi)
    b = tangent_project(prob, phi, rhs)
    bnorm = norm(prob, b)
    z = np.zeros_like(b)
    if bnorm == 0.0:
        return z, 0, 0.0
    r = b.copy()
    y = tangent_project(prob, phi, precond_C(prob, phi, r, alpha))
    p = y.copy()
    ry = inner(prob, r, y).real
    it, rel_res = 0, 1.0
    while it < max_iter:
        q = tangent_project(prob, phi, hessian_apply(prob, phi, lam, p))
        a = ry / inner(prob, p, q).real
        z = z + a * p
        r = r - a * q
        it += 1
        rel_res = norm(prob, r) / bnorm
        if rel_res < tol:
            break
        y = tangent_project(prob, phi, precond_C(prob, phi, r, alpha))
        ry_new = inner(prob, r, y).real
        p = y + (ry_new / ry) * p
        ry = ry_new
    return z, it, rel_res


def density_loss(prob, phi, rho):
    """L = int (|phi|^2 - rho)^2 (discrete: h^d sum)."""
    return prob.weight * np.sum((np.abs(phi) ** 2 - rho) ** 2)


def density_loss_gradient_V(prob, phi, rho, tol=1e-12, max_iter=5000):
    """dL/dV_k for L(phi*(V)) with phi* a normalised ground state of V.

    Differentiating H_phi phi = lambda phi with ||phi|| = 1 gives
    K dphi = -(dV phi) on the tangent space, K as in hessian_apply.  With
    g = 4 (|phi|^2 - rho) phi, the gradient of L for the weighted inner
    product, the adjoint z = K^{-1} P g (P the projection of tangent_project)
    yields dL = -Re<z, dV phi>, i.e. dL/dV_k = -h^d Re(conj(z_k) phi_k).
    Returns (dL/dV, tangent_solve iterations, relative residual)."""
    lam = inner(prob, phi, apply_H(prob, phi, phi)).real
    g = 4.0 * (np.abs(phi) ** 2 - rho) * phi
    z, it, res = tangent_solve(prob, phi, lam, g, tol=tol, max_iter=max_iter)
    return -prob.weight * (np.conj(z) * phi).real, it, res
