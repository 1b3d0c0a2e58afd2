"""Exact references that do not go through the matrix-free Newton-GMRES path.
Test infrastructure only (see ``oracle/__init__``).

  dense_newton      Newton on G(X) = 0 with the dense Jacobian formed by the
                    complex-step derivative (Squire & Trapp 1998) and solved by
                    LU; the matrix-based counterpart of Sec. 4.2 on tiny meshes.
  linear_matrix     the dense matrix of R1 for a linear flux.
  dense_stepper     Algorithm 1 for a linear flux with every stage solved by a
                    dense direct solve of (I - a1 dt L + a2 dt^2/2 L^2) W = b.
  fourier_*         for linear advection (with or without the BR2 viscous
                    term) on a uniform periodic Cartesian mesh
                    R1 is block circulant; per Fourier mode it is a small
                    matrix L(theta) (Kronecker sum of the 1-D symbols), so one
                    HBPC step and the time-exact semi-discrete solution
                    exp(t L(theta)) are computed mode by mode.
"""
import numpy as np
import scipy.linalg

from . import dgsem, hbpc, laws
from .basis import LOBATTO

CS_H = 1e-30


def dense_newton(R1, R2, b, a1, a2, dt, W0, tol=1e-14, maxit=50):
    """Solve G(X) = 0, X = (W, sigma), from (W0, R1(W0)).  R1 and R2 must accept
    complex arrays of W0's shape."""
    c1, c2 = a1 * dt, a2 * dt * dt / 2.0
    shp = W0.shape
    n = W0.size

    def G(X):
        W = X[:n].reshape(shp)
        S = X[n:].reshape(shp)
        r1 = R1(W)
        g1 = W - b - c1 * r1 + c2 * R2(W, S)
        g2 = S - r1
        return np.concatenate([np.ravel(g1), np.ravel(g2)])

    X = np.concatenate([W0.ravel(), np.ravel(R1(W0))]).astype(np.float64)
    for _ in range(maxit):
        Jm = np.zeros((2 * n, 2 * n))
        for k in range(2 * n):
            Xc = X.astype(np.complex128)
            Xc[k] += 1j * CS_H
            Jm[:, k] = np.imag(G(Xc)) / CS_H
        dX = np.linalg.solve(Jm, -G(X))
        X = X + dX
        if np.linalg.norm(dX) <= tol * max(1.0, np.linalg.norm(X)):
            break
    return X[:n].reshape(shp), X[n:].reshape(shp)


def linear_matrix(disc):
    """Dense matrix L with R1(w) = L w (linear flux only)."""
    n = disc.ndof
    L = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        L[:, k] = dgsem.R1(disc, e.reshape(disc.shape)).ravel()
    return L


def dense_stepper(L, dt, q, kmax):
    """w -> one HBPC step for dw/dt = L w, each stage by a dense direct solve.
    Works on a vector or on a stack of vectors in the last-but-one axis."""
    I = np.eye(L.shape[-1])

    def R1(w):
        return L @ w

    def R2(w, s):
        return L @ s

    def solve(b, a1, a2, guess):
        S = I - a1 * dt * L + (a2 * dt * dt / 2.0) * (L @ L)
        return np.linalg.solve(S, b)

    return lambda w: hbpc.step(w, dt, q, kmax, R1, R2, solve)


def _blocks_1d(N, h, a, family=LOBATTO, flux="lf", lf_scale=1.0, nu=0.0, eta_br2=2.0):
    """Neighbour blocks A_{-1}, A_0, A_{+1} of the 1-D advection(-diffusion)
    operator, (R1 w)_e = sum_d A_d w_{e+d}, read off the oracle's R1 on 3
    elements.  The BR2 viscous term acts along each direction separately, so the
    d-dimensional symbol is the Kronecker sum of these 1-D ones when eta_br2 is
    the d-dimensional value."""
    ph = laws.Physics(laws.ADVECTION, 1, a=(a,), flux=flux, lf_scale=lf_scale, nu=nu,
                      eta_br2=eta_br2)
    disc = dgsem.Disc(dgsem.Mesh(1, (3,), (0.0,), (3 * h,)), N, ph, family)
    p = N + 1
    A = {d: np.zeros((p, p)) for d in (-1, 0, 1)}
    for k in range(p):
        w = np.zeros((3, 1, p))
        w[1, 0, k] = 1.0
        r = dgsem.R1(disc, w)[:, 0, :]
        A[1][:, k] = r[0]
        A[0][:, k] = r[1]
        A[-1][:, k] = r[2]
    return A


def fourier_symbols(disc):
    """L(theta) for every Fourier mode of a periodic advection mesh; returns an
    array (n_{d-1}, .., n_0, P, P) with P = p^d in canonical node order."""
    mesh, N, ph = disc.mesh, disc.basis.N, disc.ph
    p, d = disc.p, disc.d
    sym1 = []
    for m in range(d):
        A = _blocks_1d(N, mesh.h[m], ph.a[m], disc.basis.family, ph.flux, ph.lf_scale,
                       ph.nu, ph.eta_br2)
        th = 2.0 * np.pi * np.arange(mesh.n[m]) / mesh.n[m]
        S = (A[-1][None] * np.exp(-1j * th)[:, None, None] + A[0][None]
             + A[1][None] * np.exp(1j * th)[:, None, None])
        sym1.append(S)
    P = p ** d
    out = np.zeros(tuple(reversed(mesh.n)) + (P, P), dtype=np.complex128)
    for idx in np.ndindex(*reversed(mesh.n)):
        kk = list(reversed(idx))       # kk[m] = mode index in direction m
        Lt = np.zeros((P, P), dtype=np.complex128)
        for m in range(d):
            # node order: axis m is the (d-1-m)-th of the d node axes
            mats = [np.eye(p)] * d
            mats = list(mats)
            mats[d - 1 - m] = sym1[m][kk[m]]
            K = mats[0]
            for M in mats[1:]:
                K = np.kron(K, M)
            Lt = Lt + K
        out[idx] = Lt
    return out


def _to_modes(disc, w):
    d = disc.d
    g = w.reshape(tuple(reversed(disc.mesh.n)) + (disc.p ** d,))
    return np.fft.fftn(g, axes=tuple(range(d)))


def _from_modes(disc, gh):
    d = disc.d
    g = np.fft.ifftn(gh, axes=tuple(range(d)))
    return np.real(g).reshape(disc.shape)


def fourier_hbpc(disc, w0, dt, q, kmax, nsteps):
    """w after nsteps HBPC(q, kmax) steps, exact per Fourier mode (advection)."""
    L = fourier_symbols(disc)
    P = L.shape[-1]
    stepper = dense_stepper(L, dt, q, kmax)
    eye = np.broadcast_to(np.eye(P, dtype=np.complex128), L.shape).copy()
    Phi = stepper(eye)                       # one-step amplification per mode
    Phin = np.linalg.matrix_power(Phi, nsteps)
    wh = _to_modes(disc, w0)
    return _from_modes(disc, np.einsum("...ij,...j->...i", Phin, wh))


def fourier_semidiscrete(disc, w0, t):
    """exp(t L) w0, the time-exact solution of the semi-discrete system."""
    L = fourier_symbols(disc)
    wh = _to_modes(disc, w0)
    out = np.empty_like(wh)
    for idx in np.ndindex(*L.shape[:-2]):
        out[idx] = scipy.linalg.expm(t * L[idx]) @ wh[idx]
    return _from_modes(disc, out)
