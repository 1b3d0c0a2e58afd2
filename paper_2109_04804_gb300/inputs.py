"""Seeded synthetic inputs shared by the CUDA path's callers and the tests.

This module holds initial-condition formulas and seeded random fields only: it
contains none of the method's arithmetic (no basis, no operator, no solver).
Every function takes physical node coordinates (computed by whoever calls it)
and returns conserved variables in the canonical layout w[e][v][nodes..].

Initial conditions follow the paper's test cases where it gives them:
  sine_product      sin(2 pi x) [sin(2 pi y) [sin(2 pi z)]]  (linear advection
                    workloads; the paper's Eq. 20 uses sin(pi x) on [-1,1])
  density_wave      rho = 1 + A sin(k pi (x_1 + .. + x_d - a t)), v = a, p = 1
                    (Eq. 22, Euler in conserved variables with reference Mach eps)
  isentropic_vortex the textbook isentropic vortex (Shu 1998) of strength beta
                    in a uniform stream of Mach M along x, rho = p = T = 1 far away
  taylor_green      the Taylor-Green vortex of Sec. 5.3.3 with v_1 = sin x cos y
                    cos z (the divergence-free form of the printed cos x ...)
  burgers_fourier   sum of 8 random Fourier modes, scaled to max |u| = 1
"""
import numpy as np


def sine_product(coords, k=2.0):
    u = np.ones_like(coords[0])
    for x in coords:
        u = u * np.sin(k * np.pi * x)
    return u[:, None].copy()


def euler_from_primitive(rho, v, p, gamma=1.4, eps=1.0):
    d = len(v)
    w = np.empty((rho.shape[0], d + 2) + rho.shape[1:])
    w[:, 0] = rho
    v2 = np.zeros_like(rho)
    for k in range(d):
        w[:, 1 + k] = rho * v[k]
        v2 = v2 + v[k] * v[k]
    w[:, d + 1] = p / (gamma - 1.0) + 0.5 * eps * eps * rho * v2
    return w


def density_wave(coords, t=0.0, a=0.3, amp=0.3, k=1.0, gamma=1.4, eps=1.0):
    s = sum(coords) - len(coords) * a * t
    rho = 1.0 + amp * np.sin(k * np.pi * s)
    v = [np.full_like(rho, a) for _ in coords]
    p = np.ones_like(rho)
    return euler_from_primitive(rho, v, p, gamma, eps)


def isentropic_vortex(coords, t=0.0, beta=5.0, mach=0.5, gamma=1.4, lo=-10.0, hi=10.0,
                      center=(0.0, 0.0)):
    x, y = coords[0], coords[1]
    u_inf = mach * np.sqrt(gamma)
    L = hi - lo
    # periodic translation of the centre
    xc = lo + np.mod(center[0] + u_inf * t - lo, L)
    yc = center[1]
    dx = x - xc
    dx = dx - L * np.round(dx / L)
    dy = y - yc
    dy = dy - L * np.round(dy / L)
    r2 = dx * dx + dy * dy
    f = np.exp(0.5 * (1.0 - r2))
    du = -beta / (2.0 * np.pi) * f * dy
    dv = beta / (2.0 * np.pi) * f * dx
    T = 1.0 - (gamma - 1.0) * beta ** 2 / (8.0 * gamma * np.pi ** 2) * f * f
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho * T
    return euler_from_primitive(rho, [u_inf + du, dv], p, gamma, 1.0)


def taylor_green(coords, gamma=1.4, eps=0.1):
    x, y, z = coords
    rho = np.ones_like(x)
    v1 = np.sin(x) * np.cos(y) * np.cos(z)
    v2 = -np.cos(x) * np.sin(y) * np.cos(z)
    v3 = np.zeros_like(x)
    p = rho / gamma + rho * eps * eps / 16.0 * (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0)
    return euler_from_primitive(rho, [v1, v2, v3], p, gamma, eps)


def burgers_fourier(coords, seed, n_modes=8, kmax=4):
    """u0 = sum_m a_m sin(2 pi k_m . x + phi_m), k_m in [-kmax, kmax]^d \\ 0,
    a_m ~ U(-1, 1), phi_m ~ U(0, 2 pi); rescaled so max |u0| = 1 at the nodes."""
    rng = np.random.default_rng(seed)
    d = len(coords)
    u = np.zeros_like(coords[0])
    for _ in range(n_modes):
        while True:
            k = rng.integers(-kmax, kmax + 1, size=d)
            if np.any(k != 0):
                break
        a = rng.uniform(-1.0, 1.0)
        phi = rng.uniform(0.0, 2.0 * np.pi)
        u = u + a * np.sin(2.0 * np.pi * sum(k[m] * coords[m] for m in range(d)) + phi)
    u = u / np.abs(u).max()
    return u[:, None].copy()


def random_field(shape, seed, scale=1.0, offset=0.0):
    rng = np.random.default_rng(seed)
    return offset + scale * rng.standard_normal(shape)
