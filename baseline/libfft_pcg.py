"""Library-FFT GPU baseline: PCG_C for the rotating Gross-Pitaevskii ground
state (arXiv:1611.02045, Algorithm 2 with Sections 5.1-5.2) in plain PyTorch,
complex128, with torch.fft (cuFFT on a CUDA device) for every transform.

It is the comparison the hand-written kernels are timed against, not part of
the library: nothing in the library imports it, and it shares no code with
the library or with the CPU oracle.  Discretisation and steps are those of
the library's FP64 mode:
  * Fourier pseudo-spectral operators on the grid x_k = -L + k h (Section 3):
    H_phi f = -1/2 Delta f + V f + eta |phi|^2 f - omega L_z f with
    L_z = -i (x d_y - y d_x);
  * P_C = P_V^{1/2} P_Delta P_V^{1/2} with the shift lambda~ = int 1/2|grad phi|^2
    + V|phi|^2 + eta|phi|^4 (eqs. combinedP_12, PDelta, PV, Opt_Alpha);
  * Polak-Ribiere beta+ (eq. CG:PR), the direction projected on the tangent
    space at phi, and the descent check of Section 5.2 (gradient step when
    Re<grad E, p> >= 0);
  * the step theta from the quadratic model of the energy along the geodesic
    cos t phi + sin t q (Section 5.1), halved until the exact energy change is
    negative, then renormalisation.
Field arithmetic stays on the device; the scalars of one iteration reach the
host in one transfer (one synchronisation per iteration), as a plain
library implementation does.  Arrays are [z][y][x] (x fastest).
"""
import math

import torch


class LibFFTPCG:
    def __init__(self, n, L, eta, omega, V, device="cuda"):
        self.n = tuple(int(m) for m in n)
        self.dim = len(self.n)
        dev = torch.device(device)
        f64 = torch.float64
        self.eta = float(eta)
        self.omega = float(omega)
        h = [2.0 * float(Li) / m for m, Li in zip(self.n, L)]
        self.w = math.prod(h)  # quadrature weight h^d
        self.shape = self.n[::-1]
        self.coord, self.freq = [], []
        for i, (m, Li) in enumerate(zip(self.n, L)):
            bshape = [1] * self.dim
            bshape[self.dim - 1 - i] = m  # physical axis i is array axis dim-1-i
            k = torch.arange(m, dtype=f64, device=dev)
            self.coord.append((-float(Li) + k * h[i]).reshape(bshape))
            p = torch.where(k < m // 2, k, k - m)  # DFT order, Nyquist mode kept
            self.freq.append((p * (math.pi / float(Li))).reshape(bshape))
        self.khalf = 0.5 * sum(xi * xi for xi in self.freq)  # 1/2 |xi|^2
        self.V = torch.as_tensor(V, dtype=f64, device=dev).reshape(self.shape)
        self.axes = tuple(range(self.dim))

    # ---- operators -----------------------------------------------------------
    def _d1(self, f, i):
        ax = self.dim - 1 - i
        return torch.fft.ifft(1j * self.freq[i] * torch.fft.fft(f, dim=ax), dim=ax)

    def _kin_rot(self, f):
        """(-1/2 Delta f, -omega L_z f) with -omega L_z f = i omega (x d_y f - y d_x f)."""
        kin = torch.fft.ifftn(self.khalf * torch.fft.fftn(f, dim=self.axes), dim=self.axes)
        rot = (1j * self.omega) * (self.coord[0] * self._d1(f, 1) - self.coord[1] * self._d1(f, 0))
        return kin, rot

    def _re_inner(self, f, g):
        """Re <f, g> = h^d Re sum conj(f) g."""
        return self.w * torch.sum(f.real * g.real + f.imag * g.imag)

    def _precond(self, u, r, alpha):
        """P_C r with P_V = (alpha + V + eta u)^{-1}, P_Delta = (alpha - Delta/2)^{-1}."""
        s = torch.rsqrt(alpha + self.V + self.eta * u)
        g = torch.fft.ifftn(torch.fft.fftn(s * r, dim=self.axes) / (alpha + self.khalf), dim=self.axes)
        return s * g

    # ---- solver --------------------------------------------------------------
    def solve(self, phi0, tol=1e-8, max_iter=20000, theta_default=0.1, max_backtracks=30, log=None):
        """Iterate from phi0 until ||H phi - lambda phi||_inf < tol or max_iter
        steps.  Returns dict(status, iters, E, lam, res_inf, phi); `log`, if a
        list, receives (E_n, lambda_n, ||r_n||_inf, theta_n) per iteration."""
        eta, w = self.eta, self.w
        phi = torch.as_tensor(phi0, device=self.V.device).to(torch.complex128).reshape(self.shape).clone()
        phi = phi / torch.sqrt(self._re_inner(phi, phi))
        p_prev = r_prev = rPr_prev = None
        zero = torch.zeros((), dtype=torch.float64, device=self.V.device)
        n = 0
        while True:
            u = phi.real ** 2 + phi.imag ** 2
            kin_f, rot_f = self._kin_rot(phi)
            Hphi = kin_f + (self.V + eta * u) * phi + rot_f
            kin = self._re_inner(phi, kin_f)
            pot = w * torch.sum(self.V * u)
            rot = self._re_inner(phi, rot_f)
            U0 = w * torch.sum(u * u)
            lam = kin + pot + rot + eta * U0
            E = lam - 0.5 * eta * U0
            r = Hphi - lam * phi
            res_inf = torch.max(torch.abs(r))
            alpha = kin + pot + eta * U0
            Pr = self._precond(u, r, alpha)
            rPr = self._re_inner(r, Pr)
            beta = zero if rPr_prev is None else torch.clamp(self._re_inner(r - r_prev, Pr) / rPr_prev, min=0.0)

            def tangent(d):
                return d - self._re_inner(d, phi) * phi

            p_gd = tangent(-Pr)
            p_cg = p_gd if p_prev is None else tangent(-Pr + beta * p_prev)
            fallback = 2.0 * self._re_inner(Hphi, p_cg) >= 0.0
            p = torch.where(fallback, p_gd, p_cg)
            beta = torch.where(fallback, zero, beta)
            q = p / torch.sqrt(self._re_inner(p, p))
            # moments fixing E(cos t phi + sin t q) exactly
            kq, rq = self._kin_rot(q)
            Aq = kq + self.V * q + rq
            z = phi.conj() * q
            v = z.real
            wq = q.real ** 2 + q.imag ** 2
            R = self._re_inner(Hphi, q)
            aqq = self._re_inner(q, Aq)
            U1 = w * torch.sum(u * v)
            V2 = w * torch.sum(v * v)
            UW = w * torch.sum(u * wq)
            VW = w * torch.sum(v * wq)
            W2 = w * torch.sum(wq * wq)
            Z2 = w * torch.sum(z.real * z.real - z.imag * z.imag)  # Re int conj(phi)^2 q^2
            curv = aqq + 2.0 * eta * UW + eta * Z2 - lam  # 1/2 d^2E(phi)[q,q] - lambda
            (E_, lam_, res_, R_, aqq_, U0_, U1_, V2_, UW_, VW_, W2_, curv_) = torch.stack(
                [E, lam, res_inf, R, aqq, U0, U1, V2, UW, VW, W2, curv]).tolist()
            if res_ < tol or n >= max_iter or not math.isfinite(E_) or not math.isfinite(res_):
                status = "converged" if res_ < tol else ("nonfinite" if not math.isfinite(E_ + res_) else "max_iter")
                return dict(status=status, iters=n, E=E_, lam=lam_, res_inf=res_, phi=phi)

            def dE(t):
                c, s = math.cos(t), math.sin(t)
                return (2.0 * c * s * R_ + s * s * (aqq_ - lam_)
                        + 0.5 * eta * (s ** 4 * (U0_ + W2_) + c * c * s * s * (4.0 * V2_ + 2.0 * UW_)
                                       + 4.0 * c * s ** 3 * (VW_ - U1_)))

            theta = -R_ / curv_ if curv_ > 0.0 else theta_default
            bt = 0
            while not dE(theta) < 0.0 and bt < max_backtracks:
                theta *= 0.5
                bt += 1
            if log is not None:
                log.append((E_, lam_, res_, theta))
            phi = math.cos(theta) * phi + math.sin(theta) * q
            phi = phi / torch.sqrt(self._re_inner(phi, phi))
            p_prev, r_prev, rPr_prev = p, r, rPr
            n += 1
