"""Pins of the oracle's Navier-Stokes viscous operator (Sec. 5, Eq. 25-33)
against what the mathematics fixes, independently of its own formulas:

* a manufactured smooth state: the discrete viscous term converges spectrally
  to div F^v computed symbolically (sympy differentiates the closed form of
  Eq. 25 -- stress tensor, heat flux, T from the ideal-gas law);
* special states where the system reduces exactly to the pinned scalar BR2
  operator: v = 0 leaves lambda L_h(T) in the energy row; a shear v = (0, f(x))
  leaves mu L_h(f) in the y-momentum row;
* R^(2) equals the complex-step derivative of R^(1) (Eq. 32-33 are the exact
  linearisation with the central viscous and lifting fluxes);
* the frozen-neighbour R^(2) (element-diagonal block) equals R^(2) with the
  direction restricted to one element, read on that element;
* discrete conservation of every variable (central viscous fluxes);
* mu = 0 gives the Euler operator."""
import numpy as np
import pytest

from oracle import dgsem, laws, newton
from oracle.basis import GAUSS, LOBATTO


def ns_disc(dim, n, N, mu=0.01, family=LOBATTO, flux="lf", eps=1.0, lo=None, hi=None, eta=None):
    ph = laws.Physics(laws.NAVIER_STOKES, dim, mu=mu, flux=flux, eps=eps, eta_br2=eta)
    lo = lo if lo is not None else (0.0,) * dim
    hi = hi if hi is not None else (1.0,) * dim
    return dgsem.Disc(dgsem.Mesh(dim, n, lo, hi), N, ph, family)


def random_state(disc, seed):
    """A positive-density, positive-pressure state with random perturbations."""
    rng = np.random.default_rng(seed)
    d = disc.d
    w = np.zeros(disc.shape)
    w[:, 0] = 1.0 + 0.2 * rng.random(w[:, 0].shape)
    for k in range(d):
        w[:, 1 + k] = 0.3 * rng.standard_normal(w[:, 0].shape)
    w[:, d + 1] = 2.5 + 0.3 * rng.random(w[:, 0].shape)
    return w


def state_from_primitives(disc, rho, vel, p):
    ph = disc.ph
    d = disc.d
    w = np.zeros(disc.shape)
    w[:, 0] = rho
    v2 = sum(v * v for v in vel)
    for k in range(d):
        w[:, 1 + k] = rho * vel[k]
    w[:, d + 1] = p / (ph.gamma - 1.0) + 0.5 * ph.eps ** 2 * rho * v2
    return w


# -- manufactured solution ---------------------------------------------------

def exact_viscous_divergence(dim, mu, gamma=1.4, eps=1.0, prandtl=0.72):
    """Closed-form div F^v of Eq. 25 for a smooth periodic state, by sympy."""
    sp = pytest.importorskip("sympy")
    X = sp.symbols("x0:%d" % dim, real=True)
    tp = 2 * sp.pi
    if dim == 1:
        rho = 1 + sp.Rational(1, 5) * sp.sin(tp * X[0])
        vel = [sp.Rational(3, 10) * sp.cos(tp * X[0])]
        p = 1 + sp.Rational(1, 10) * sp.sin(2 * tp * X[0])
    elif dim == 2:
        rho = 1 + sp.Rational(1, 5) * sp.sin(tp * X[0]) * sp.cos(tp * X[1])
        vel = [sp.Rational(3, 10) * sp.sin(tp * X[1]) + sp.Rational(1, 10) * sp.cos(tp * X[0]),
               sp.Rational(1, 5) * sp.cos(tp * X[0]) * sp.sin(tp * X[1])]
        p = 1 + sp.Rational(1, 10) * sp.sin(tp * (X[0] + X[1]))
    else:
        rho = 1 + sp.Rational(1, 5) * sp.sin(tp * X[0]) * sp.cos(tp * X[2])
        vel = [sp.Rational(3, 10) * sp.sin(tp * X[1]),
               sp.Rational(1, 5) * sp.cos(tp * X[2]) * sp.sin(tp * X[0]),
               sp.Rational(1, 10) * sp.sin(tp * (X[0] + X[1]))]
        p = 1 + sp.Rational(1, 10) * sp.cos(tp * (X[1] - X[2]))
    R = 1 / (sp.Float(gamma) * eps ** 2)
    cp = R * gamma / (gamma - 1)
    lam = cp * mu / prandtl
    T = p / (rho * R)
    div_v = sum(sp.diff(vel[k], X[k]) for k in range(dim))
    tau = [[mu * (sp.diff(vel[j], X[i]) + sp.diff(vel[i], X[j]) - (sp.Rational(2, 3) * div_v if i == j else 0))
            for j in range(dim)] for i in range(dim)]
    rows = [sp.Integer(0)]
    for k in range(dim):
        rows.append(sum(sp.diff(tau[k][m], X[m]) for m in range(dim)))
    rows.append(sum(sp.diff(sum(tau[m][k] * vel[k] for k in range(dim)) + lam * sp.diff(T, X[m]), X[m])
                    for m in range(dim)))
    f_state = sp.lambdify(X, [rho] + vel + [p], "numpy")
    f_rows = sp.lambdify(X, rows, "numpy")
    return f_state, f_rows


def manufactured_error(dim, n, N, family=LOBATTO, mu=0.05):
    disc = ns_disc(dim, (n,) * dim, N, mu=mu, family=family)
    f_state, f_rows = exact_viscous_divergence(dim, mu)
    xs = disc.node_coords()
    st = [np.broadcast_to(np.asarray(a, dtype=float), xs[0].shape) for a in f_state(*xs)]
    w = state_from_primitives(disc, st[0], st[1:1 + dim], st[1 + dim])
    got = dgsem.viscous_ns(disc, w)
    ref = np.stack([np.broadcast_to(np.asarray(a, dtype=float), xs[0].shape) for a in f_rows(*xs)], axis=1)
    return np.abs(got - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("family", [LOBATTO, GAUSS])
def test_manufactured_2d_converges_spectrally(family):
    e_lo = manufactured_error(2, 4, 4, family)
    e_hi = manufactured_error(2, 4, 11, family)
    assert e_hi < 2e-5, e_hi
    assert e_hi < 1e-3 * e_lo, (e_lo, e_hi)


def test_manufactured_1d_and_3d():
    e1_lo, e1_hi = manufactured_error(1, 6, 6), manufactured_error(1, 6, 14)
    assert e1_hi < 1e-8 and e1_hi < 1e-5 * e1_lo, (e1_lo, e1_hi)
    e3_lo = manufactured_error(3, 3, 3)
    e3_hi = manufactured_error(3, 3, 7)
    assert e3_hi < 1e-2, e3_hi
    assert e3_hi < 0.03 * e3_lo, (e3_lo, e3_hi)


# -- reductions to the scalar BR2 operator ------------------------------------

@pytest.mark.parametrize("family", [LOBATTO, GAUSS])
def test_no_velocity_leaves_the_heat_flux(family):
    """v = 0: tau = 0 and F^v = (0, 0, lambda grad T): the energy row is lambda
    times the scalar BR2 operator applied to the nodal T."""
    disc = ns_disc(2, (3, 4), 3, family=family, eta=3.0)
    rng = np.random.default_rng(3)
    shp = disc.shape[:1] + disc.shape[2:]
    rho = 1.0 + 0.3 * rng.random(shp)
    p = 1.0 + 0.2 * rng.random(shp)
    w = state_from_primitives(disc, rho, [0 * rho, 0 * rho], p)
    got = dgsem.viscous_ns(disc, w)
    ph = disc.ph
    T = p / (rho * ph.R_gas)
    sc = dgsem.Disc(disc.mesh, 3, laws.Physics(laws.BURGERS, 2, nu=1.0, eta_br2=3.0), family)
    ref = ph.kappa_heat * dgsem.viscous(sc, T[:, None])[:, 0]
    assert np.abs(got[:, :3]).max() == 0.0
    np.testing.assert_allclose(got[:, 3], ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_shear_leaves_the_scalar_operator_in_the_momentum_row():
    """v = (0, f(x)): tau_yy = 0 (d_y f = 0, div v = 0) and tau_yx = mu d_x f, so
    the y-momentum row is mu L_h(f) even for f discontinuous across x faces.
    For a continuous f (a smooth function on the shared Lobatto face nodes) the
    lifted and broken x-derivatives agree and the x-momentum row (the
    y-divergence of tau_xy = mu d_x f) vanishes too."""
    disc = ns_disc(2, (4, 3), 4, mu=0.02)
    x, _ = disc.node_coords()
    rng = np.random.default_rng(5)
    ex = np.arange(disc.mesh.nE) % disc.mesh.n[0]
    vals = rng.standard_normal((disc.mesh.n[0], disc.p))
    f_jump = vals[ex][:, None, :] * np.ones((1, disc.p, 1))     # the same 1-D values on every y line
    f_cont = np.sin(2 * np.pi * x) + 0.3 * np.cos(4 * np.pi * x)
    sc = dgsem.Disc(disc.mesh, 4, laws.Physics(laws.BURGERS, 2, nu=0.02), LOBATTO)
    for f in (f_jump, f_cont):
        w = state_from_primitives(disc, 1.0 + 0.0 * x, [0 * x, f], 1.0 + 0 * x)
        got = dgsem.viscous_ns(disc, w)
        ref = dgsem.viscous(sc, f[:, None])[:, 0]
        np.testing.assert_allclose(got[:, 2], ref, rtol=0, atol=1e-12 * np.abs(ref).max())
        assert np.abs(got[:, 0]).max() == 0.0
    assert np.abs(got[:, 1]).max() <= 1e-12 * np.abs(ref).max()


# -- linearisation, frozen neighbours, conservation ---------------------------

@pytest.mark.parametrize("dim,n,N,family", [(2, (3, 4), 3, LOBATTO), (2, (2, 3), 2, GAUSS), (3, (2, 2, 3), 2, LOBATTO),
                                            (1, (5,), 4, LOBATTO)])
def test_r2_is_the_complex_step_derivative(dim, n, N, family):
    disc = ns_disc(dim, n, N, family=family)
    w = random_state(disc, 11)
    s = np.random.default_rng(12).standard_normal(disc.shape)
    h = 1e-30
    cs = np.imag(dgsem.R1(disc, w + 1j * h * s)) / h
    r2 = dgsem.R2(disc, w, s)
    assert np.abs(r2 - cs).max() <= 1e-13 * np.abs(cs).max()
    csv = np.imag(dgsem.viscous_ns(disc, w + 1j * h * s)) / h
    assert np.abs(dgsem.viscous_ns(disc, w, s) - csv).max() <= 1e-13 * np.abs(csv).max()


@pytest.mark.parametrize("family", [LOBATTO, GAUSS])
def test_frozen_neighbour_is_the_element_block(family):
    disc = ns_disc(2, (3, 2), 2, family=family, flux="rusanov")
    w = random_state(disc, 21)
    s = np.random.default_rng(22).standard_normal(disc.shape)
    frozen = dgsem.operator(disc, w, s, mode="R2", frozen_neighbor=True)
    for e in range(disc.mesh.nE):
        se = np.zeros_like(s)
        se[e] = s[e]
        ref = dgsem.R2(disc, w, se)[e]
        assert np.abs(frozen[e] - ref).max() <= 1e-13 * np.abs(ref).max(), e


def test_bjext_block_of_the_viscous_law_is_its_element_jacobian():
    """The BJ_ext J_i of the oracle (frozen-neighbour R2 on unit vectors) is the
    complex-step Jacobian of R1 with the other elements held fixed (LF flux)."""
    disc = ns_disc(2, (2, 3), 2, mu=0.03)
    w = random_state(disc, 31)
    st = newton.StageSystem(disc, np.zeros(disc.ndof), 0.5, 0.1, 0.01)
    pc = newton.BJExt(st, w)
    nb = disc.ndof // disc.mesh.nE
    e = 4
    Jref = np.zeros((nb, nb))
    for c in range(nb):
        x = w.astype(complex).reshape(disc.mesh.nE, nb)
        x[e, c] += 1e-30j
        Jref[:, c] = np.imag(dgsem.R1(disc, x.reshape(disc.shape)).reshape(disc.mesh.nE, nb)[e]) / 1e-30
    assert np.abs(pc.J[e] - Jref).max() <= 1e-12 * np.abs(Jref).max()


@pytest.mark.parametrize("dim,n", [(2, (3, 4)), (3, (2, 3, 2))])
def test_viscous_term_conserves_every_variable(dim, n):
    disc = ns_disc(dim, n, 3, mu=0.05, lo=(-1.0,) * dim, hi=(1.0, 2.0, 0.5)[:dim])
    w = random_state(disc, 41)
    s = np.random.default_rng(42).standard_normal(disc.shape)
    for r in (dgsem.viscous_ns(disc, w), dgsem.viscous_ns(disc, w, s)):
        tot = dgsem.cell_integral(disc, r)
        scale = dgsem.cell_integral(disc, np.abs(r)).max()
        assert np.abs(tot).max() <= 1e-13 * scale, tot


def test_zero_viscosity_is_euler():
    disc = ns_disc(2, (3, 3), 3, mu=0.0, flux="rusanov")
    eu = dgsem.Disc(disc.mesh, 3, laws.Physics(laws.EULER, 2, flux="rusanov"), LOBATTO)
    w = random_state(disc, 51)
    s = np.random.default_rng(52).standard_normal(disc.shape)
    np.testing.assert_array_equal(dgsem.R1(disc, w), dgsem.R1(eu, w))
    np.testing.assert_array_equal(dgsem.R2(disc, w, s), dgsem.R2(eu, w, s))


def test_invalid_viscosity_arguments():
    with pytest.raises(ValueError):
        laws.Physics(laws.EULER, 2, mu=0.1)
    with pytest.raises(ValueError):
        laws.Physics(laws.NAVIER_STOKES, 2, nu=0.1)
    ph = laws.Physics(laws.NAVIER_STOKES, 3, mu=2e-3, eps=0.5)
    assert ph.R_gas == pytest.approx(1.0 / (1.4 * 0.25))
    assert ph.cp == pytest.approx(ph.R_gas * 1.4 / 0.4)
    assert ph.kappa_heat == pytest.approx(ph.cp * 2e-3 / 0.72)


@pytest.mark.parametrize("dim,flux", [(2, "lf"), (2, "rusanov"), (3, "lf")])
def test_navier_stokes_jfnk_matches_dense_newton(dim, flux):
    """The matrix-free Newton-GMRES stage solve of the viscous law (Eq. 17 with
    the Eq. 23 quotients) reaches the root of a dense Newton whose Jacobian is
    built column by column by complex step and solved by LU."""
    from oracle import exact
    n = (2, 2) if dim == 2 else (2, 1, 2)   # 3-D: one element in y, its own periodic neighbour
    disc = ns_disc(dim, n, 2 if dim == 2 else 1, mu=0.05, flux=flux)
    W0 = random_state(disc, 61)
    b = W0 + 0.01 * np.random.default_rng(62).standard_normal(disc.shape)
    dt, a1, a2 = 0.05, 0.5, 1.0 / 6.0
    Wd, Sd = exact.dense_newton(lambda w: dgsem.R1(disc, w), lambda w, s: dgsem.R2(disc, w, s), b, a1, a2, dt, W0)
    for jv in ("fd", "analytic"):
        opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-14, gmres_tol=1e-8, restart=400, jv=jv)
        W, S, st = newton.newton_solve(disc, b, a1, a2, dt, W0, opts)
        assert st.converged
        assert np.linalg.norm(W - Wd) / np.linalg.norm(Wd) < 1e-12, jv
