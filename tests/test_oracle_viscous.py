"""Pins of the oracle's BR2 viscous operator (Sec. 5.1, Eqs. 26-30 in their
scalar form F^v = nu grad u) against what mathematics fixes: the Laplacian it
approximates, the exact derivative of a continuous function, conservation,
symmetry and definiteness of the BR2 bilinear form, the element-diagonal block,
and the heat equation's exact decay through a whole HBPC step."""
import numpy as np
import pytest

from oracle import dgsem, exact, laws
from oracle.basis import GAUSS, LOBATTO


def make(dim, n, N, family=LOBATTO, law=laws.BURGERS, nu=0.05, eta=None, a=(1.0, 1.0, 1.0),
         hi=1.0):
    ph = laws.Physics(law, dim, a=a, nu=nu, eta_br2=eta)
    mesh = dgsem.Mesh(dim, n, (0.0,) * dim, (hi,) * dim)
    return dgsem.Disc(mesh, N, ph, family)


def dense_viscous(disc):
    nd = disc.ndof
    A = np.zeros((nd, nd))
    for j in range(nd):
        e = np.zeros(nd)
        e[j] = 1.0
        A[:, j] = dgsem.viscous(disc, e.reshape(disc.shape)).ravel()
    return A


def mass_diag(disc):
    wq = disc.basis.weights
    M = wq
    for _ in range(disc.d - 1):
        M = np.multiply.outer(wq, M)
    return np.tile(M.ravel(), disc.mesh.nE) * np.prod(disc.mesh.h / 2.0)


@pytest.mark.parametrize("family", [LOBATTO, GAUSS])
@pytest.mark.parametrize("dim", [1, 2, 3])
def test_constant_in_kernel_and_conservation(family, dim):
    n = {1: (5,), 2: (3, 4), 3: (2, 3, 2)}[dim]
    disc = make(dim, n, 3, family)
    c = np.full(disc.shape, 1.7)
    assert np.abs(dgsem.viscous(disc, c)).max() < 1e-12
    u = np.random.default_rng(1).standard_normal(disc.shape)
    V = dgsem.viscous(disc, u)
    # central viscous flux: what leaves one element enters its neighbour
    assert abs(dgsem.cell_integral(disc, V)[0]) < 1e-12 * np.abs(V).max()


@pytest.mark.parametrize("family", [LOBATTO, GAUSS])
@pytest.mark.parametrize("dim,n", [(1, (6,)), (2, (3, 4))])
def test_symmetric_negative_semidefinite(family, dim, n):
    """M L_h is symmetric (BR2 with central fluxes is a symmetric interior
    penalty form) and, with eta = 2 dim, negative semi-definite; its kernel is
    the constants only."""
    disc = make(dim, n, 3, family)
    A = dense_viscous(disc)
    MA = mass_diag(disc)[:, None] * A
    assert np.abs(MA - MA.T).max() < 1e-12 * np.abs(MA).max()
    ev = np.linalg.eigvalsh(0.5 * (MA + MA.T))
    assert ev.max() < 1e-12 * np.abs(ev).max()
    assert np.sum(np.abs(ev) < 1e-10 * np.abs(ev).max()) == 1


@pytest.mark.parametrize("family,tol", [(LOBATTO, 2e-6), (GAUSS, 8e-6)])
def test_spectral_convergence_to_laplacian(family, tol):
    errs = []
    for N in (3, 5, 7):
        disc = make(2, (6, 6), N, family, nu=0.01)
        x, y = disc.node_coords()
        u = (np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y))[:, None]
        ex = -8.0 * np.pi ** 2 * 0.01 * u
        V = dgsem.viscous(disc, u)
        errs.append(np.linalg.norm(V - ex) / np.linalg.norm(ex))
    assert errs[0] > 30 * errs[1] > 900 * errs[2]
    assert errs[2] < tol


def test_gradient_of_continuous_function_is_its_derivative():
    """For nodal values of a continuous function on Lobatto nodes the traces
    agree (u* = u), so the lifted gradient is the derivative of the element
    interpolant: (2/h) D u along each line."""
    disc = make(2, (4, 3), 4, LOBATTO)
    x, y = disc.node_coords()
    u = (np.sin(2 * np.pi * x) + np.cos(4 * np.pi * y) * np.sin(2 * np.pi * x))[:, None]
    b = disc.basis
    for m in range(2):
        d = dgsem.br2_gradient(disc, u, m)
        U = u.reshape((disc.mesh.nE, 1) + (disc.p,) * 2)
        ax = 3 if m == 0 else 2            # node axes (k, j, i) -> i is last
        Du = np.moveaxis(np.tensordot(b.D, U, axes=([1], [ax])), 0, ax) * (2.0 / disc.mesh.h[m])
        assert np.abs(d.reshape(U.shape) - Du).max() < 1e-12 * np.abs(Du).max()


@pytest.mark.parametrize("family", [LOBATTO, GAUSS])
def test_gradient_single_element_polynomial(family):
    """One periodic element on [0, 1], u = 1 - xi^2 (xi = 2x - 1) takes the same
    value 0 at both ends, so the lifting adds nothing and d = du/dx = -4 xi."""
    disc = make(1, (1,), 4, family)
    xi = 2.0 * disc.node_coords()[0] - 1.0
    u = (1.0 - xi * xi)[:, None]
    d = dgsem.br2_gradient(disc, u, 0)
    assert np.abs(d[:, 0] - (-4.0 * xi)).max() < 1e-12


@pytest.mark.parametrize("family", [LOBATTO, GAUSS])
def test_frozen_neighbour_block(family):
    """frozen_neighbor gives the element-diagonal block: the output on element e
    of L_h applied to the input restricted to e."""
    disc = make(2, (3, 3), 3, family)
    u = np.random.default_rng(4).standard_normal(disc.shape)
    F = dgsem.viscous(disc, u, frozen_neighbor=True)
    for e in range(disc.mesh.nE):
        ue = np.zeros_like(u)
        ue[e] = u[e]
        assert np.abs(dgsem.viscous(disc, ue)[e] - F[e]).max() < 1e-13 * np.abs(F).max()


def test_R2_is_directional_derivative_with_viscosity():
    """R2(w, s) = d/de R1(w + e s) (complex step) for viscous Burgers."""
    disc = make(2, (3, 4), 3, LOBATTO, nu=0.03)
    rng = np.random.default_rng(7)
    w = 1.0 + 0.3 * rng.standard_normal(disc.shape)
    s = rng.standard_normal(disc.shape)
    h = 1e-30
    cs = np.imag(dgsem.R1(disc, w + 1j * h * s)) / h
    assert np.abs(dgsem.R2(disc, w, s) - cs).max() < 1e-12 * np.abs(cs).max()


def test_heat_equation_decay_through_hbpc():
    """u_t = nu u_xx (advection speed 0) from sin(2 pi x): one HBPC(6, 2) step
    with dense stage solves damps the mode by exp(-4 pi^2 nu dt) up to the
    spatial and temporal error."""
    nu, dt = 0.05, 0.05
    disc = make(1, (8,), 7, LOBATTO, law=laws.ADVECTION, nu=nu, a=(0.0,))
    L = exact.linear_matrix(disc)
    x = disc.node_coords()[0]
    u0 = np.sin(2 * np.pi * x)[:, None]
    step = exact.dense_stepper(L, dt, 6, 2)
    u1 = step(u0.ravel()).reshape(u0.shape)
    ex = np.exp(-4 * np.pi ** 2 * nu * dt) * u0
    assert np.linalg.norm(u1 - ex) / np.linalg.norm(ex) < 1e-9


def test_fourier_symbol_matches_dense_with_viscosity():
    """The Kronecker-sum Fourier symbol (1-D blocks) reproduces the dense 2-D
    advection-diffusion operator: one HBPC step agrees both ways."""
    disc = make(2, (4, 5), 3, LOBATTO, law=laws.ADVECTION, nu=0.02, a=(1.0, 0.5))
    u0 = np.random.default_rng(2).standard_normal(disc.shape)
    L = exact.linear_matrix(disc)
    dense = exact.dense_stepper(L, 0.05, 4, 1)(u0.ravel()).reshape(u0.shape)
    four = exact.fourier_hbpc(disc, u0, 0.05, 4, 1, 1)
    assert np.abs(dense - four).max() < 1e-12 * np.abs(dense).max()
