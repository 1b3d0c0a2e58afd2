"""Pins of the numerical flux's dissipation coefficient (Eq. 13) in the oracle.

Eq. 13 is f* = 1/2 (F(wL) + F(wR)) . n + kappa (wL - wR).  Two choices of kappa
are used:
  * global Lax-Friedrichs: the constant of the paper, lambda = |a . n| for
    advection (Sec. 4.1.1) and diag(1/eps, 1, 1, 1/eps) for Euler (Sec. 4.1.2,
    stored in tests/golden/euler_lf_lambda.txt);
  * Rusanov (local Lax-Friedrichs, the Euler workload's flux): half the largest
    wave speed of the two traces.

Each pin measures kappa from outside the flux code: from the energy balance of
the discrete advection operator, from the face terms of R1 on a piecewise
constant state, and from the eigenvalues of the flux Jacobian (numpy.linalg)."""
import os

import numpy as np
import pytest

from oracle import dgsem, laws
from oracle.basis import GAUSS, LOBATTO

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "euler_lf_lambda.txt")


def _energy_rate_and_jumps(disc, w):
    """w^T M R1(w) and, per direction, the face integral of the squared jump."""
    r = dgsem.R1(disc, w)
    rate = dgsem.cell_integral(disc, w * r)[0]
    b, mesh = disc.basis, disc.mesh
    W = disc.to_grid(w)
    jumps = []
    for m in range(disc.d):
        na, ea = disc.node_axis(m), disc.elem_axis(m)
        wp = np.tensordot(W, b.l_p, axes=([na], [0]))
        wm = np.tensordot(W, b.l_m, axes=([na], [0]))
        tot = (wp - np.roll(wm, -1, axis=ea)) ** 2
        for k in reversed([k for k in range(disc.d) if k != m]):
            tot = np.tensordot(tot, b.weights, axes=([tot.ndim - 1], [0])) * mesh.h[k] / 2
        jumps.append(tot.sum())
    return rate, jumps


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("fam", [LOBATTO, GAUSS])
def test_rusanov_advection_is_upwind(dim, fam):
    """For linear advection the Rusanov flux is the upwind (exact Riemann)
    flux, kappa = |a . n| / 2: the energy of the semi-discrete operator then
    decays at exactly 1/2 |a . n| times the squared face jumps (the collocated
    quadrature is exact for a linear flux).  A kappa twice or half as large
    changes the rate by the whole dissipation term."""
    a = (0.8, -0.45)
    ph = laws.Physics(laws.ADVECTION, dim, a=a, flux="rusanov")
    disc = dgsem.Disc(dgsem.Mesh(dim, (4, 3), (0, 0), (1.0, 0.6)), 3, ph, fam)
    w = np.random.default_rng(5).standard_normal(disc.shape)
    rate, jumps = _energy_rate_and_jumps(disc, w)
    diss = sum(0.5 * abs(a[m]) * jumps[m] for m in range(dim))
    assert diss > 0
    assert abs(rate + diss) < 1e-12 * diss
    # the same operator as global LF at half the paper's lambda
    ph_lf = laws.Physics(laws.ADVECTION, dim, a=a, flux="lf", lf_scale=0.5)
    disc_lf = dgsem.Disc(disc.mesh, 3, ph_lf, fam)
    assert np.array_equal(dgsem.R1(disc, w), dgsem.R1(disc_lf, w))


def _flux_jacobian(w, m, ph):
    """dF^m/dw at one state by complex step (independent of laws.flux_jvp)."""
    nv = w.shape[0]
    J = np.empty((nv, nv))
    h = 1e-30
    for c in range(nv):
        z = w.astype(complex)
        z[c] += 1j * h
        J[:, c] = np.imag(laws.flux(z, m, ph)) / h
    return J


def _random_euler(rng, dim, eps, gamma=1.4):
    rho = 0.5 + rng.uniform()
    v = rng.uniform(-1.0, 1.0, dim)
    p = 0.3 + rng.uniform()
    return np.concatenate([[rho], rho * v, [p / (gamma - 1) + 0.5 * eps ** 2 * rho * v @ v]])


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("eps", [1.0, 0.3])
def test_max_speed_is_spectral_radius(dim, eps):
    """The wave speed the Rusanov coefficient uses equals the spectral radius of
    the flux Jacobian (eigenvalues by LAPACK), with the eps-scaled sound speed."""
    rng = np.random.default_rng(11 + dim)
    ph = laws.Physics(laws.EULER, dim, eps=eps)
    for _ in range(5):
        w = _random_euler(rng, dim, eps)
        for m in range(dim):
            rad = np.max(np.abs(np.linalg.eigvals(_flux_jacobian(w, m, ph))))
            s = laws.max_speed(w[:, None], m, ph)[0]
            assert abs(s - rad) < 1e-12 * rad
    phb = laws.Physics(laws.BURGERS, dim)
    for u in (-1.7, 0.4):
        w = np.array([u])
        rad = abs(_flux_jacobian(w, 0, phb)[0, 0])
        assert abs(laws.max_speed(w[:, None], 0, phb)[0] - rad) < 1e-14


def _face_kappa(disc_diss, disc_central, wA, wB):
    """kappa per variable as the operator applies it: on two periodic 1-D
    elements holding the constant states wA, wB both faces of element 0 see
    (wL, wR) = (wA, wB) and the volume terms of the two fluxes agree, so with
    Lobatto nodes R1_diss - R1_central at element 0's last node equals
    -(2/h) kappa (wA - wB) / omega_N."""
    w = np.zeros(disc_diss.shape)
    w[0] = wA[:, None]
    w[1] = wB[:, None]
    d = dgsem.R1(disc_diss, w) - dgsem.R1(disc_central, w)
    h = disc_diss.mesh.h[0]
    om = disc_diss.basis.weights[-1]
    return -d[0, :, -1] * h * om / (2.0 * (wA - wB))


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            f = line.split()
            rows.append((int(f[0]), float(f[1]), np.array([float(x) for x in f[2:]])))
    return rows


def test_golden_rows_match_the_printed_rule():
    """The fixture has 1/eps on density and energy, 1 on momentum."""
    for dim, eps, lam in _golden():
        assert lam.size == dim + 2
        assert abs(lam[0] - 1 / eps) < 1e-15 * lam[0] and abs(lam[-1] - 1 / eps) < 1e-15 * lam[-1]
        assert np.all(lam[1:-1] == 1.0)


@pytest.mark.parametrize("row", range(6))
def test_euler_global_lf_lambda_in_the_operator(row):
    """The global-LF coefficient the Euler operator applies at a face equals the
    paper's lambda = diag(1/eps, 1, .., 1, 1/eps) (Sec. 4.1.2)."""
    dim, eps, lam = _golden()[row]
    # measured along x on a mesh with one element in the other directions: the
    # transverse faces see the same state on both sides and add nothing
    rng = np.random.default_rng(40 + row)
    wA, wB = _random_euler(rng, dim, eps), _random_euler(rng, dim, eps)
    n = (2, 1, 1)
    mesh = dgsem.Mesh(dim, n, (0, 0, 0), (1.0, 1.0, 1.0))
    disc = dgsem.Disc(mesh, 3, laws.Physics(laws.EULER, dim, eps=eps, flux="lf"))
    disc_c = dgsem.Disc(mesh, 3, laws.Physics(laws.EULER, dim, eps=eps, flux="lf", lf_scale=0.0))
    w = np.zeros(disc.shape)
    w[0] = wA.reshape((-1,) + (1,) * dim)
    w[1] = wB.reshape((-1,) + (1,) * dim)
    d = dgsem.R1(disc, w) - dgsem.R1(disc_c, w)
    # element 0, the x-last node (the other node indices arbitrary: take 0)
    idx = (0, slice(None)) + (0,) * (dim - 1) + (-1,)
    kappa = -d[idx] * mesh.h[0] * disc.basis.weights[-1] / (2.0 * (wA - wB))
    assert np.allclose(kappa, lam, rtol=1e-10, atol=0)


@pytest.mark.parametrize("eps", [1.0, 0.4])
def test_euler_rusanov_coefficient_in_the_operator(eps):
    """The Rusanov coefficient the Euler operator applies at a face is half the
    larger spectral radius of the two traces' flux Jacobians, the same for
    every variable."""
    rng = np.random.default_rng(7)
    ph = laws.Physics(laws.EULER, 1, eps=eps, flux="rusanov")
    mesh = dgsem.Mesh(1, (2,), (0,), (1.0,))
    disc = dgsem.Disc(mesh, 4, ph)
    disc_c = dgsem.Disc(mesh, 4, laws.Physics(laws.EULER, 1, eps=eps, flux="lf", lf_scale=0.0))
    for _ in range(4):
        wA, wB = _random_euler(rng, 1, eps), _random_euler(rng, 1, eps)
        rad = max(np.max(np.abs(np.linalg.eigvals(_flux_jacobian(x, 0, ph)))) for x in (wA, wB))
        kappa = _face_kappa(disc, disc_c, wA, wB)
        assert np.allclose(kappa, 0.5 * rad, rtol=1e-10, atol=0)
