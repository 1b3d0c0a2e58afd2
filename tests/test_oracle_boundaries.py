"""Pins of the oracle's non-periodic boundaries (constant Dirichlet exterior
states and the Euler slip wall, imposed weakly through the numerical flux of
Eq. 13 with an exterior state).

* Linear advection: the discrete energy rate w^T M R1(w) equals, face by face,
  -kappa [[w]]^2 at interior faces and the closed forms of a boundary face with
  exterior value g (own trace u):  upper end  -a g u / 2 - kappa (u - g) u,
  lower end  a g u / 2 + kappa (g - u) u  (quadrature exact for a linear flux).
* Euler in a box of slip walls: mass, energy and tangential momentum are
  conserved exactly, the normal momentum changes by the wall forces
  rho v_n^2 + p / eps^2 +- 2 kappa m_n integrated over the walls, and a gas at
  rest stays at rest.  A Dirichlet exterior equal to a uniform state keeps it.
* R2 at the boundaries is the derivative of R1 (complex step; global LF), which
  fixes the exterior sigma: zero for constant data, mirrored at a wall.
* The element blocks J_i, H_i at boundary elements are the diagonal blocks of
  the full complex-step dR1/dW, dR2/dW."""
import numpy as np
import pytest

from oracle import dgsem, laws, newton
from oracle.basis import GAUSS, LOBATTO
from tests.test_oracle_bjext_h import dense_derivative, diag_blocks


def face_integral(disc, vals, m):
    """Integrate a face array (grid layout, node axis m removed) over the face
    points with the quadrature of the other directions."""
    b, tot = disc.basis, vals
    for k in reversed([k for k in range(disc.d) if k != m]):
        tot = np.tensordot(tot, b.weights, axes=([tot.ndim - 1], [0])) * disc.mesh.h[k] / 2
    return tot


@pytest.mark.parametrize("fam", [LOBATTO, GAUSS])
@pytest.mark.parametrize("flux", ["lf", "rusanov"])
@pytest.mark.parametrize("g", [0.0, 0.7])
def test_advection_energy_rate_with_dirichlet_boundaries(fam, flux, g):
    dim = 2
    ph = laws.Physics(laws.ADVECTION, dim, a=(0.8, -0.45), flux=flux)
    spec = ("dirichlet", [g])
    mesh = dgsem.Mesh(dim, (4, 3), (0, 0), (1.0, 0.6), bc=[(spec, spec), None])
    disc = dgsem.Disc(mesh, 3, ph, fam)
    w = np.random.default_rng(61).standard_normal(disc.shape)
    rate = dgsem.cell_integral(disc, w * dgsem.R1(disc, w))[0]
    b, W = disc.basis, disc.to_grid(w)
    expect = 0.0
    for m in range(dim):
        na, ea = disc.node_axis(m), disc.elem_axis(m)
        a = ph.a[m]
        kappa = abs(a) * (0.5 if flux == "rusanov" else 1.0)
        wp = np.tensordot(W, b.l_p, axes=([na], [0]))[0]
        wm = np.tensordot(W, b.l_m, axes=([na], [0]))[0]
        jump = wp - np.roll(wm, -1, axis=ea - 1)
        inner = -kappa * jump ** 2
        if mesh.bc[m] is not None:
            last = [slice(None)] * inner.ndim
            last[ea - 1] = -1
            last = tuple(last)
            first = [slice(None)] * inner.ndim
            first[ea - 1] = 0
            first = tuple(first)
            inner[last] = 0.0
            expect += face_integral(disc, -0.5 * a * g * wp[last] - kappa * (wp[last] - g) * wp[last], m).sum()
            expect += face_integral(disc, 0.5 * a * g * wm[first] + kappa * (g - wm[first]) * wm[first], m).sum()
        expect += face_integral(disc, inner, m).sum()
    assert abs(rate - expect) <= 1e-12 * abs(expect)


def euler_box(N, n, fam, flux, eps=1.0, walls=True):
    ph = laws.Physics(laws.EULER, 2, flux=flux, eps=eps)
    wall = ("wall",)
    bc = [(wall, wall), (wall, wall)] if walls else None
    return dgsem.Disc(dgsem.Mesh(2, n, (-1, -1), (1, 0.5), bc=bc), N, ph, fam)


def random_gas(disc, seed):
    from paper_2109_04804_gb300 import inputs
    rng = np.random.default_rng(seed)
    X = disc.node_coords()
    rho = 1.0 + 0.2 * np.sin(2.1 * X[0] + 0.3) * np.cos(1.3 * X[1]) + 0.02 * rng.standard_normal(X[0].shape)
    v = [0.3 * np.cos(1.7 * X[1] + 0.2) + 0.05 * rng.standard_normal(X[0].shape),
         -0.2 * np.sin(1.1 * X[0]) + 0.05 * rng.standard_normal(X[0].shape)]
    p = 1.0 + 0.1 * np.cos(X[0] + X[1])
    return inputs.euler_from_primitive(rho, v, p, disc.ph.gamma, disc.ph.eps)


@pytest.mark.parametrize("fam", [LOBATTO, GAUSS])
@pytest.mark.parametrize("flux,eps", [("lf", 1.0), ("rusanov", 1.0), ("lf", 0.3)])
def test_euler_slip_walls_conservation_and_wall_force(fam, flux, eps):
    disc = euler_box(3, (4, 3), fam, flux, eps)
    ph, b = disc.ph, disc.basis
    w = random_gas(disc, 62)
    rate = dgsem.cell_integral(disc, dgsem.R1(disc, w))
    scale = np.abs(rate).max()
    assert abs(rate[0]) <= 1e-12 * scale and abs(rate[3]) <= 1e-12 * scale
    W = disc.to_grid(w)
    for M in range(2):
        na, ea = disc.node_axis(M), disc.elem_axis(M)
        force = 0.0
        for side, lvec in ((1, b.l_p), (0, b.l_m)):
            t = np.tensordot(W, lvec, axes=([na], [0]))
            end = [slice(None)] * t.ndim
            end[ea] = -1 if side else 0
            t = t[tuple(end)]
            rho, v, E, p = laws.euler_primitives(t, ph)
            kap = np.broadcast_to(laws.dissipation(t, laws.exterior_state(t, ("wall",), M, ph), M, ph),
                                  t.shape)[1 + M]
            fstar = rho * v[M] ** 2 + p / ph.eps ** 2 + (2 * kap * t[1 + M] if side else -2 * kap * t[1 + M])
            # the element's outward flux at an upper wall leaves, at a lower wall enters
            force += (-1.0 if side else 1.0) * face_integral(disc, fstar, M).sum()
        assert abs(rate[1 + M] - force) <= 1e-12 * scale, (M, rate[1 + M], force)


@pytest.mark.parametrize("fam", [LOBATTO, GAUSS])
def test_gas_at_rest_in_a_box_and_dirichlet_free_stream(fam):
    from paper_2109_04804_gb300 import inputs
    disc = euler_box(4, (3, 3), fam, "rusanov")
    X = disc.node_coords()
    w = inputs.euler_from_primitive(np.full_like(X[0], 1.3), [0 * X[0], 0 * X[0]], np.full_like(X[0], 0.8))
    assert np.abs(dgsem.R1(disc, w)).max() <= 1e-13
    state = inputs.euler_from_primitive(np.array([1.1]), [np.array([0.4]), np.array([-0.3])], np.array([0.9]))[0]
    spec = ("dirichlet", state)
    ph = laws.Physics(laws.EULER, 2, flux="rusanov")
    d2 = dgsem.Disc(dgsem.Mesh(2, (3, 4), (0, 0), (1, 1), bc=[(spec, spec), (spec, spec)]), 3, ph, fam)
    w2 = np.broadcast_to(state.reshape(1, 4, 1, 1), d2.shape).copy()
    assert np.abs(dgsem.R1(d2, w2)).max() <= 1e-12


def mixed_bc_euler(fam, flux):
    """Walls along y, an inflow/outflow Dirichlet pair along x."""
    from paper_2109_04804_gb300 import inputs
    st = inputs.euler_from_primitive(np.array([1.0]), [np.array([0.3]), np.array([0.0])], np.array([1.0]))[0]
    bc = [(("dirichlet", st), ("dirichlet", 1.05 * st)), (("wall",), ("wall",))]
    ph = laws.Physics(laws.EULER, 2, flux=flux)
    return dgsem.Disc(dgsem.Mesh(2, (3, 2), (0, 0), (1, 1), bc=bc), 2, ph, fam)


@pytest.mark.parametrize("fam", [LOBATTO, GAUSS])
def test_r2_is_the_derivative_of_r1_at_boundaries(fam):
    disc = mixed_bc_euler(fam, "lf")
    w = random_gas(disc, 63)
    s = np.random.default_rng(64).standard_normal(disc.shape)
    h = 1e-30
    ref = np.imag(dgsem.R1(disc, w + 1j * h * s)) / h
    r2 = dgsem.R2(disc, w, s)
    assert np.abs(r2 - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("fam", [LOBATTO, GAUSS])
def test_element_blocks_at_boundaries(fam):
    """J_i and H_i (LF flux) equal the diagonal blocks of the full complex-step
    dR1/dW and dR2/dW, boundary elements included."""
    disc = mixed_bc_euler(fam, "lf")
    w = random_gas(disc, 65)
    S = np.random.default_rng(66).standard_normal(disc.shape)
    nE = disc.mesh.nE
    J = newton.element_jacobians(disc, w)
    Jd = diag_blocks(dense_derivative(disc, lambda x: dgsem.operator(disc, x, mode="R1"), w), nE)
    assert np.abs(J - Jd).max() <= 1e-11 * np.abs(Jd).max()
    H = newton.element_hessian_blocks(disc, w, S)
    Hd = diag_blocks(dense_derivative(disc, lambda x: dgsem.operator(disc, x, S, mode="R2"), w), nE)
    assert np.abs(H - Hd).max() <= 1e-11 * np.abs(Hd).max()


def test_periodic_connection_unchanged():
    """A mesh whose bc list is all None is the periodic mesh (same values)."""
    ph = laws.Physics(laws.EULER, 2, flux="rusanov")
    d0 = dgsem.Disc(dgsem.Mesh(2, (3, 2), (0, 0), (1, 1)), 3, ph)
    d1 = dgsem.Disc(dgsem.Mesh(2, (3, 2), (0, 0), (1, 1), bc=[None, None]), 3, ph)
    w = random_gas(d0, 67)
    assert np.array_equal(dgsem.R1(d0, w), dgsem.R1(d1, w))


def test_linear_jv_is_the_derivative_of_G_with_dirichlet_data():
    """With nonzero Dirichlet data R1 of a linear flux is affine: the linear
    Jacobian-vector product (Eq. 24) must be the derivative of G, which the
    complex step of the residual gives exactly."""
    ph = laws.Physics(laws.ADVECTION, 2, a=(0.8, -0.45))
    bc = [(("dirichlet", [0.7]), ("dirichlet", [-0.3])), (("dirichlet", [0.2]), ("dirichlet", [0.1]))]
    disc = dgsem.Disc(dgsem.Mesh(2, (3, 4), (0, 0), (1, 1), bc=bc), 3, ph, GAUSS)
    rng = np.random.default_rng(68)
    sysm = newton.StageSystem(disc, rng.standard_normal(disc.shape), 0.5, 1.0 / 6.0, 0.1)
    X = rng.standard_normal(2 * disc.ndof)
    dX = rng.standard_normal(2 * disc.ndof)
    G, r1, r2 = sysm.residual(X)
    h = 1e-30
    ref = np.imag(sysm.residual(X + 1j * h * dX)[0]) / h
    out = sysm.jv(X, r1, r2, dX, "linear")
    assert np.linalg.norm(out - ref) <= 1e-13 * np.linalg.norm(ref)


# ---- Navier-Stokes: adiabatic no-slip walls and Dirichlet states ---------------

def ns_disc(bc, fam=LOBATTO, flux="lf", n=(3, 3), N=2):
    ph = laws.Physics(laws.NAVIER_STOKES, 2, flux=flux, mu=0.05, eps=1.0)
    return dgsem.Disc(dgsem.Mesh(2, n, (0, 0), (1, 1), bc=bc), N, ph, fam)


NOSLIP = ("noslip",)


def lid_state():
    from paper_2109_04804_gb300 import inputs
    return inputs.euler_from_primitive(np.array([1.0]), [np.array([0.4]), np.array([0.0])], np.array([1.0]))[0]


@pytest.mark.parametrize("fam", [LOBATTO, GAUSS])
def test_ns_r2_is_the_derivative_of_r1_at_walls(fam):
    """Global LF: R2 (with the linearised ghost channels) equals the complex-step
    derivative of R1 with walls and a lid."""
    disc = ns_disc([(NOSLIP, NOSLIP), (NOSLIP, ("dirichlet", lid_state()))], fam)
    w = random_gas(disc, 91)
    s = np.random.default_rng(92).standard_normal(disc.shape)
    h = 1e-30
    ref = np.imag(dgsem.R1(disc, w + 1j * h * s)) / h
    r2 = dgsem.R2(disc, w, s)
    assert np.abs(r2 - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("fam", [LOBATTO, GAUSS])
@pytest.mark.parametrize("flux", ["lf", "rusanov"])
def test_ns_noslip_box_conserves_mass_and_energy(fam, flux):
    """Walls pass no mass (reversed momentum, equal density) and no energy (no
    work at zero wall velocity, no heat through an adiabatic wall): the
    totals of R1's density and energy rows vanish."""
    disc = ns_disc([(NOSLIP, NOSLIP), (NOSLIP, NOSLIP)], fam, flux, n=(4, 3), N=3)
    w = random_gas(disc, 93)
    rate = dgsem.cell_integral(disc, dgsem.R1(disc, w))
    scale = np.abs(dgsem.R1(disc, w)).max()
    assert abs(rate[0]) <= 1e-13 * scale and abs(rate[3]) <= 1e-13 * scale
    assert abs(rate[1]) > 1e-8 * scale          # the walls do push on the gas


@pytest.mark.parametrize("fam", [LOBATTO, GAUSS])
def test_ns_gas_at_rest_and_dirichlet_free_stream(fam):
    from paper_2109_04804_gb300 import inputs
    disc = ns_disc([(NOSLIP, NOSLIP), (NOSLIP, NOSLIP)], fam, "rusanov", N=3)
    X = disc.node_coords()
    w = inputs.euler_from_primitive(np.full_like(X[0], 1.2), [0 * X[0], 0 * X[0]], np.full_like(X[0], 0.9))
    assert np.abs(dgsem.R1(disc, w)).max() <= 1e-12
    st = lid_state()
    d2 = ns_disc([(("dirichlet", st), ("dirichlet", st)), (("dirichlet", st), ("dirichlet", st))], fam, "rusanov")
    w2 = np.broadcast_to(st.reshape(1, 4, 1, 1), d2.shape).copy()
    assert np.abs(dgsem.R1(d2, w2)).max() <= 1e-12


def test_ns_element_blocks_at_walls():
    """The frozen-neighbour element blocks J_i (global LF) are the diagonal
    blocks of the full complex-step dR1/dW, wall and lid elements included."""
    disc = ns_disc([(NOSLIP, NOSLIP), (NOSLIP, ("dirichlet", lid_state()))], LOBATTO, "lf", n=(3, 2))
    w = random_gas(disc, 94)
    J = newton.element_jacobians(disc, w)
    Jd = diag_blocks(dense_derivative(disc, lambda x: dgsem.operator(disc, x, mode="R1"), w), disc.mesh.nE)
    assert np.abs(J - Jd).max() <= 1e-11 * np.abs(Jd).max()
