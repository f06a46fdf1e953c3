"""Seeded synthetic inputs: trapping potentials and initial wave functions.

This module only *generates* arrays (host, numpy, float64/complex128).  It
holds none of the solver's arithmetic: no transforms, operators or
reductions.  Both the CUDA path and the CPU oracle are fed from here, so the
two sides always see bit-identical inputs.

Grid points follow the paper's Section 3: x_k = -L + k h, h = 2L/M, k = 0..M-1,
arrays stored [z][y][x] with x fastest.

Random numbers come from splitmix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), evaluated as a pure function of
(seed, index) so that any element can be regenerated on its own.
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(seed: int, index: np.ndarray) -> np.ndarray:
    """splitmix64 output for state = seed + (index+1) * golden gamma (uint64)."""
    with np.errstate(over="ignore"):
        gamma = np.uint64(0x9E3779B97F4A7C15)
        z = np.uint64(seed) + (index.astype(np.uint64) + np.uint64(1)) * gamma
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """`count` doubles in [-1, 1) from the top 53 bits of splitmix64."""
    idx = np.arange(offset, offset + count, dtype=np.uint64)
    bits = splitmix64(seed, idx) >> np.uint64(11)
    return bits.astype(np.float64) * (2.0 / 2.0**53) - 1.0


def coords(n, L):
    """1-D coordinate vectors x_k = -L + k*2L/n for each axis (x, y[, z])."""
    return [(-Li + np.arange(ni) * (2.0 * Li / ni)) for ni, Li in zip(n, L)]


def mesh(n, L):
    """Broadcastable coordinate arrays (X, Y[, Z]) in [z][y][x] layout."""
    c = coords(n, L)
    if len(n) == 2:
        Y, X = np.meshgrid(c[1], c[0], indexing="ij")
        return X, Y
    Z, Y, X = np.meshgrid(c[2], c[1], c[0], indexing="ij")
    return X, Y, Z


def shape_of(n):
    """numpy shape [z][y][x] for per-axis sizes n = (nx, ny[, nz])."""
    return tuple(reversed(tuple(n)))


def weight(n, L):
    """Quadrature weight h^d used to normalise the initial guesses."""
    w = 1.0
    for ni, Li in zip(n, L):
        w *= 2.0 * Li / ni
    return w


def normalise(phi, n, L):
    return phi / np.sqrt(weight(n, L) * np.sum(np.abs(phi) ** 2))


# --- potentials --------------------------------------------------------------

def harmonic(n, L, gammas=None):
    """V = sum_i gamma_i^2 x_i^2 / 2 (gamma_i = 1 by default)."""
    m = mesh(n, L)
    gammas = gammas or [1.0] * len(n)
    return sum(0.5 * (g * xi) ** 2 for g, xi in zip(gammas, m))


def harmonic_quartic(n, L, kappa, gammas=None):
    """V = harmonic + kappa (x^2+y^2)^2 / 4 (the quartic trap shape)."""
    m = mesh(n, L)
    r2 = m[0] ** 2 + m[1] ** 2
    return harmonic(n, L, gammas) + 0.25 * kappa * r2 * r2


def paper_harmonic(n, L, gammas=None):
    """V_d^0 of eq. Lattice_Poten as printed for d = 2, 3: sum_nu gamma_nu nu^2
    (gamma_nu = 1 by default).  With gamma = 1 this is r^2, twice the V = r^2/2
    trap that Example eg:diff_initial_fix_grid states explicitly."""
    m = mesh(n, L)
    gammas = gammas or [1.0] * len(n)
    return sum(g * xi * xi for g, xi in zip(gammas, m))


def harmonic_plus_lattice(n, L, kappas, qs, gammas=None):
    """eq. Lattice_Poten: V = V_d^0 + sum_nu kappa_nu sin^2(q_nu nu^2), the
    argument nu^2 taken as printed (the 2D example of Section 6.2 uses
    gamma = 1, kappa = 25, q = pi/2 on [-32, 32]^2)."""
    m = mesh(n, L)
    return paper_harmonic(n, L, gammas) + sum(k * np.sin(q * xi * xi) ** 2 for k, q, xi in zip(kappas, qs, m))


def harmonic_plus_quartic(n, L, alpha, kappa, gammas=None, gamma_z=0.0):
    """eq. Quart_Poten: V = (1 - alpha) V_2^0 + kappa (x^2 + y^2)^2 / 4, plus
    gamma_z^2 z^2 in 3D, with V_2^0 = gamma_x x^2 + gamma_y y^2 as printed.
    alpha > 1 makes the harmonic part repulsive (the double-well regime of
    Section 6.2: alpha = 1.2, kappa = 0.3; 3D: alpha = 1.4, gamma_z = 3)."""
    m = mesh(n, L)
    g = gammas or [1.0, 1.0]
    V = (1.0 - alpha) * (g[0] * m[0] ** 2 + g[1] * m[1] ** 2)
    r2 = m[0] ** 2 + m[1] ** 2
    V = V + 0.25 * kappa * r2 * r2
    if len(n) == 3:
        V = V + gamma_z ** 2 * m[2] ** 2
    return V


def smooth_bumps(n, L, seed, count=8):
    """Sum of `count` seeded Gaussian bumps scaled to max |S| = 1."""
    m = mesh(n, L)
    u = uniform_pm1(seed, 4 * count)
    S = np.zeros(m[0].shape)
    for j in range(count):
        cx, cy = 6.0 * u[4 * j], 6.0 * u[4 * j + 1]
        sig = 2.0 + u[4 * j + 2]
        amp = u[4 * j + 3]
        S += amp * np.exp(-((m[0] - cx) ** 2 + (m[1] - cy) ** 2) / (2 * sig * sig))
    return S / np.max(np.abs(S))


# --- initial data (Section 6, initial data (a), (b), (d)) ---------------------

def phi_a(n, L):
    """(a): pi^{-d/4} exp(-|x|^2/2) (2D: pi^{-1/2} exp(-r^2/2))."""
    m = mesh(n, L)
    r2 = sum(xi * xi for xi in m)
    return (np.pi ** (-len(n) / 4.0)) * np.exp(-0.5 * r2) + 0j


def phi_b(n, L):
    """(b): (x + i y) phi_a."""
    m = mesh(n, L)
    return (m[0] + 1j * m[1]) * phi_a(n, L)


def phi_d(n, L, omega):
    """(d): normalised (1-omega) phi_a + omega phi_b."""
    return normalise((1.0 - omega) * phi_a(n, L) + omega * phi_b(n, L), n, L)


def anisotropic_gaussian(n, L, gammas):
    """prod_i (gamma_i/pi)^{1/4} exp(-gamma_i x_i^2 / 2)."""
    m = mesh(n, L)
    g = np.ones(m[0].shape, dtype=np.complex128)
    for gi, xi in zip(gammas, m):
        g = g * (gi / np.pi) ** 0.25 * np.exp(-0.5 * gi * xi * xi)
    return g


def perturbed(G, seed, n, L, amp=1e-3):
    """norm(G * (1 + amp (u1 + i u2))) with u1, u2 = splitmix64 uniforms in [-1,1)."""
    N = G.size
    u = uniform_pm1(seed, 2 * N).reshape(2, *G.shape)
    return normalise(G * (1.0 + amp * (u[0] + 1j * u[1])), n, L)


def random_field(seed, n, L):
    """A dense complex field with uniform(-1,1) parts (for operator tests)."""
    N = int(np.prod(n))
    u = uniform_pm1(seed, 2 * N).reshape(2, *shape_of(n))
    return u[0] + 1j * u[1]


# --- the named workloads -----------------------------------------------------

def workload(name: str, index: int = 0):
    """Return dict(n, L, eta, omega, V, phi0) for a named synthetic workload.

    c64_2d     : 64x64 on [-8,8]^2, V = r^2/2, eta = 100, omega = 0.5,
                 phi_a + seeded 1e-3 perturbation (seed 1).
    fast256_2d : 256x256 on [-16,16]^2, V = r^2/2, eta = 1000, omega = 0.9,
                 phi_d (Gaussian plus vortex) + 1e-3 perturbation (seed 2).
    rot128_3d  : 128^3 on [-8,8]^3, V = (x^2+y^2+4z^2)/2, eta = 5000,
                 omega = 0.8, anisotropic Gaussian (1,1,2) times the vortex
                 factor mix (1-omega) + omega (x+iy), perturbed (seed 4).
    grad256_2d : instance `index` (0..15) of the differentiation batch:
                 256x256 on [-16,16]^2, eta = 500, omega = 0.7,
                 V = r^2/2 + 0.1 S with S = smooth_bumps(seed 50 + index),
                 phi_d + 1e-3 perturbation (seed 70 + index).
    """
    if name == "c64_2d":
        n, L = (64, 64), (8.0, 8.0)
        V = harmonic(n, L)
        phi0 = perturbed(phi_a(n, L), 1, n, L)
        return dict(n=n, L=L, eta=100.0, omega=0.5, V=V, phi0=phi0)
    if name == "fast256_2d":
        n, L = (256, 256), (16.0, 16.0)
        V = harmonic(n, L)
        phi0 = perturbed(phi_d(n, L, 0.9), 2, n, L)
        return dict(n=n, L=L, eta=1000.0, omega=0.9, V=V, phi0=phi0)
    if name == "rot128_3d":
        n, L = (128, 128, 128), (8.0, 8.0, 8.0)
        V = harmonic(n, L, [1.0, 1.0, 2.0])
        m = mesh(n, L)
        G = anisotropic_gaussian(n, L, [1.0, 1.0, 2.0])
        G = ((1.0 - 0.8) + 0.8 * (m[0] + 1j * m[1])) * G
        phi0 = perturbed(normalise(G, n, L), 4, n, L)
        return dict(n=n, L=L, eta=5000.0, omega=0.8, V=V, phi0=phi0)
    if name == "grad256_2d":
        n, L = (256, 256), (16.0, 16.0)
        V = harmonic(n, L) + 0.1 * smooth_bumps(n, L, 50 + index)
        phi0 = perturbed(phi_d(n, L, 0.7), 70 + index, n, L)
        return dict(n=n, L=L, eta=500.0, omega=0.7, V=V, phi0=phi0)
    raise KeyError(name)


def sweep_instances(count: int = 96, seed: int = 3, grids=(128, 256, 512)):
    """The batched parameter sweep: `count` independent 2D problems on
    [-16,16]^2 (count a multiple of len(grids); equally many of each grid size,
    in a seeded order), omega ~ U[0, 0.95], eta in {100, 250, 500, 1000},
    V = r^2/2 + kappa r^4/4 with kappa in {0, 0.05}, initial guess phi_d(omega)
    with a 1e-3 perturbation (seed 100 + i).  Parameters are drawn from
    splitmix64 with `seed`: per instance i, uniforms u[4i..4i+3] give omega,
    the eta index, kappa and the grid-order key.  Returns a list of dicts
    (n, L, eta, omega, kappa, V, phi0); V and phi0 are built on demand by
    sweep_arrays()."""
    if count % len(grids):
        raise ValueError("count must be a multiple of the number of grid sizes")
    u = uniform_pm1(seed, 4 * count).reshape(count, 4)
    base = np.repeat(np.asarray(grids), count // len(grids))
    order = np.argsort(u[:, 3], kind="stable")
    sizes = base[np.argsort(order, kind="stable")]
    etas = (100.0, 250.0, 500.0, 1000.0)
    out = []
    for i in range(count):
        M = int(sizes[i])
        out.append(dict(n=(M, M), L=(16.0, 16.0), omega=0.95 * 0.5 * (u[i, 0] + 1.0),
                        eta=etas[min(int(2.0 * (u[i, 1] + 1.0)), 3)],
                        kappa=0.05 if u[i, 2] > 0.0 else 0.0, seed=100 + i))
    return out


def sweep_arrays(inst):
    """(V, phi0) of one sweep instance."""
    n, L = inst["n"], inst["L"]
    V = harmonic_quartic(n, L, inst["kappa"])
    phi0 = perturbed(phi_d(n, L, inst["omega"]), inst["seed"], n, L)
    return V, phi0
