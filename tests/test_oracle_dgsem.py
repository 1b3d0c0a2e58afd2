"""Pins of the oracle's R^(1) (Eq. 12) and R^(2) (Eq. 16) against properties the
mathematics fixes: free stream, discrete conservation, polynomial exactness,
the derivative identity dR1/dw v = R2(w, v) (Sec. 3.2.1) by complex step, and
R2(w, s) = R1(s) for a linear flux."""
import numpy as np
import pytest

from oracle import dgsem, laws
from oracle.basis import GAUSS, LOBATTO


def make(law, dim, N, n=(3, 2, 2), family=LOBATTO, flux="lf", eps=1.0):
    ph = laws.Physics(law, dim, a=(1.0, -0.6, 0.35), eps=eps, flux=flux)
    mesh = dgsem.Mesh(dim, n, (0.0, -1.0, 0.5), (1.0, 1.0, 2.0))
    return dgsem.Disc(mesh, N, ph, family)


def euler_state(disc, rng, amp=0.1):
    d = disc.d
    w = np.zeros(disc.shape)
    rho = 1.0 + amp * rng.standard_normal(disc.shape[:1] + disc.shape[2:])
    v = [0.3 + amp * rng.standard_normal(rho.shape) for _ in range(d)]
    p = 1.0 + amp * rng.standard_normal(rho.shape)
    w[:, 0] = rho
    for k in range(d):
        w[:, 1 + k] = rho * v[k]
    eps2 = disc.ph.eps ** 2
    w[:, d + 1] = p / (disc.ph.gamma - 1) + 0.5 * eps2 * rho * sum(x * x for x in v)
    return w


def state(disc, rng):
    if disc.ph.law == laws.EULER:
        return euler_state(disc, rng)
    return rng.standard_normal(disc.shape)


CASES = [(law, dim, fam, flux) for law in (laws.ADVECTION, laws.BURGERS, laws.EULER)
         for dim in (1, 2, 3) for fam in (LOBATTO, GAUSS) for flux in ("lf", "rusanov")]


@pytest.mark.parametrize("law,dim,fam,flux", CASES)
def test_free_stream(law, dim, fam, flux):
    disc = make(law, dim, 3, family=fam, flux=flux)
    w = np.ones(disc.shape)
    if law == laws.EULER:
        w = euler_state(disc, np.random.default_rng(0), amp=0.0)
    r = dgsem.R1(disc, w)
    assert np.abs(r).max() < 1e-12 * max(1.0, np.abs(w).max())


@pytest.mark.parametrize("law,dim,fam,flux", CASES)
def test_discrete_conservation(law, dim, fam, flux):
    disc = make(law, dim, 3, family=fam, flux=flux)
    rng = np.random.default_rng(1)
    w = state(disc, rng)
    s = rng.standard_normal(disc.shape)
    for r in (dgsem.R1(disc, w), dgsem.R2(disc, w, s)):
        tot = dgsem.cell_integral(disc, r)
        scale = dgsem.cell_integral(disc, np.abs(r))
        assert np.all(np.abs(tot) <= 1e-13 * scale)


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("fam", [LOBATTO, GAUSS])
def test_polynomial_exactness_advection(dim, fam):
    """w = prod_m x_m(1-x_m) on [0,1]^d is continuous and periodic; with N >= 2 the
    flux is represented exactly and R1 = -a . grad w at every node."""
    ph = laws.Physics(laws.ADVECTION, dim, a=(1.0, -0.6, 0.35))
    disc = dgsem.Disc(dgsem.Mesh(dim, (3, 4, 2), (0, 0, 0), (1, 1, 1)), 3, ph, fam)
    X = disc.node_coords()
    f = [x * (1 - x) for x in X]
    df = [1 - 2 * x for x in X]
    w = np.prod(f, axis=0)[:, None]
    grad = 0.0
    for m in range(dim):
        term = df[m]
        for k in range(dim):
            if k != m:
                term = term * f[k]
        grad = grad + ph.a[m] * term
    np.testing.assert_allclose(dgsem.R1(disc, w), -grad[:, None], atol=1e-12)


@pytest.mark.parametrize("fam", [LOBATTO, GAUSS])
def test_polynomial_exactness_burgers(fam):
    ph = laws.Physics(laws.BURGERS, 1)
    disc = dgsem.Disc(dgsem.Mesh(1, (5,), (0,), (1,)), 4, ph, fam)
    x = disc.node_coords()[0]
    w = (x * (1 - x))[:, None]
    expect = -(x * (1 - x)) * (1 - 2 * x)
    np.testing.assert_allclose(dgsem.R1(disc, w)[:, 0], expect, atol=1e-12)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_euler_flux_jvp_complex_step(dim):
    ph = laws.Physics(laws.EULER, dim, eps=0.3)
    rng = np.random.default_rng(2)
    disc = make(laws.EULER, dim, 2, eps=0.3)
    w = euler_state(disc, rng)
    s = rng.standard_normal(w.shape)
    wg, sg = disc.to_grid(w), disc.to_grid(s)
    h = 1e-30
    for m in range(dim):
        cs = np.imag(laws.flux(wg + 1j * h * sg, m, ph)) / h
        np.testing.assert_allclose(laws.flux_jvp(wg, sg, m, ph), cs, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("law,dim,fam", [(l, d, f) for l in (laws.ADVECTION, laws.BURGERS, laws.EULER)
                                         for d in (1, 2, 3) for f in (LOBATTO, GAUSS)])
def test_r2_is_derivative_of_r1_lf(law, dim, fam):
    """Global Lax-Friedrichs: dR1/dw v = R2(w, v) exactly (Sec. 3.2.1)."""
    disc = make(law, dim, 3, family=fam)
    rng = np.random.default_rng(4)
    w = state(disc, rng)
    v = rng.standard_normal(disc.shape)
    h = 1e-30
    cs = np.imag(dgsem.R1(disc, w + 1j * h * v)) / h
    r2 = dgsem.R2(disc, w, v)
    np.testing.assert_allclose(r2, cs, rtol=1e-12, atol=1e-11 * np.abs(cs).max())


@pytest.mark.parametrize("law,dim", [(laws.ADVECTION, 2), (laws.BURGERS, 2), (laws.EULER, 2),
                                     (laws.EULER, 3)])
def test_r2_rusanov_at_uniform_state(law, dim):
    """Rusanov: R2 freezes the dissipation coefficient; at a uniform state the
    jump w^L - w^R vanishes, so R2 equals the full derivative of R1."""
    disc = make(law, dim, 3, flux="rusanov")
    rng = np.random.default_rng(5)
    if law == laws.EULER:
        w = euler_state(disc, rng, amp=0.0)
    else:
        w = np.full(disc.shape, 0.7)
    v = rng.standard_normal(disc.shape)
    h = 1e-30
    cs = np.imag(dgsem.R1(disc, w + 1j * h * v)) / h
    np.testing.assert_allclose(dgsem.R2(disc, w, v), cs, rtol=1e-12, atol=1e-11 * np.abs(cs).max())


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_linear_flux_r2_equals_r1_of_sigma(dim):
    disc = make(laws.ADVECTION, dim, 4)
    rng = np.random.default_rng(6)
    w, s = rng.standard_normal(disc.shape), rng.standard_normal(disc.shape)
    np.testing.assert_allclose(dgsem.R2(disc, w, s), dgsem.R1(disc, s), atol=1e-12)


def test_r2_finite_difference_first_order():
    disc = make(laws.EULER, 2, 3)
    rng = np.random.default_rng(7)
    w = euler_state(disc, rng)
    v = rng.standard_normal(disc.shape)
    r2 = dgsem.R2(disc, w, v)
    errs = []
    for e in (1e-3, 5e-4):
        fd = (dgsem.R1(disc, w + e * v) - dgsem.R1(disc, w)) / e
        errs.append(np.abs(fd - r2).max())
    assert 1.7 < errs[0] / errs[1] < 2.3   # O(eps)


def test_spatial_convergence_rate():
    """R1 of sin(2 pi x) converges like h^N in the max norm (Lobatto N=3)."""
    errs = []
    for n in (8, 16, 32):
        ph = laws.Physics(laws.ADVECTION, 1)
        disc = dgsem.Disc(dgsem.Mesh(1, (n,), (0,), (1,)), 3, ph)
        x = disc.node_coords()[0]
        r = dgsem.R1(disc, np.sin(2 * np.pi * x)[:, None])[:, 0]
        errs.append(np.abs(r + 2 * np.pi * np.cos(2 * np.pi * x)).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 2.7)


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("fam", [LOBATTO, GAUSS])
@pytest.mark.parametrize("lf_scale", [1.0, 0.5])
def test_advection_energy_identity(dim, fam, lf_scale):
    """For a linear flux the collocated quadrature is exact, so the discrete
    energy rate is  w^T M R1(w) = - sum_faces int kappa [[w]]^2  with
    kappa = lf_scale |a.n| the dissipation coefficient of Eq. 13."""
    ph = laws.Physics(laws.ADVECTION, dim, a=(0.8, -0.45), lf_scale=lf_scale)
    mesh = dgsem.Mesh(dim, (4, 3), (0, 0), (1.0, 0.6))
    disc = dgsem.Disc(mesh, 3, ph, fam)
    rng = np.random.default_rng(21)
    w = rng.standard_normal(disc.shape)
    r = dgsem.R1(disc, w)
    rate = dgsem.cell_integral(disc, w * r)[0]
    b = disc.basis
    W = disc.to_grid(w)
    diss = 0.0
    for m in range(dim):
        na, ea = disc.node_axis(m), disc.elem_axis(m)
        wp = np.tensordot(W, b.l_p, axes=([na], [0]))
        wm = np.tensordot(W, b.l_m, axes=([na], [0]))
        jump = wp - np.roll(wm, -1, axis=ea)
        kappa = lf_scale * abs(ph.a[m])
        tot = kappa * jump ** 2
        # remaining node axes are the last (dim-1) axes; integrate each
        for k in reversed([k for k in range(dim) if k != m]):
            tot = np.tensordot(tot, b.weights, axes=([tot.ndim - 1], [0])) * mesh.h[k] / 2
        diss += tot.sum()
    assert abs(rate + diss) < 1e-12 * abs(diss)


def test_euler_isentropic_vortex_time_derivative():
    """The isentropic vortex translates with the stream: w_t = -u_inf dw/dx.
    R1 of the vortex converges spectrally to it (pins every term of Eq. 21 at
    eps = 1)."""
    from paper_2109_04804_gb300 import inputs
    errs = []
    for n in (16, 32):
        ph = laws.Physics(laws.EULER, 2, flux="rusanov")
        disc = dgsem.Disc(dgsem.Mesh(2, (n, n), (-10, -10), (10, 10)), 6, ph)
        X = disc.node_coords()
        w = inputs.isentropic_vortex(X)
        dt = 1e-5
        wt = (inputs.isentropic_vortex(X, t=dt) - inputs.isentropic_vortex(X, t=-dt)) / (2 * dt)
        errs.append(np.abs(dgsem.R1(disc, w) - wt).max())
    assert errs[1] < 1e-3 and errs[1] < errs[0] / 16


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_euler_eps_scaling(dim):
    """Eq. 21 with reference Mach eps equals the eps = 1 flux of the state with
    E / eps^2, the energy row scaled by eps^2 (p = eps^2 p_1)."""
    rng = np.random.default_rng(22)
    eps = 0.2
    ph, ph1 = laws.Physics(laws.EULER, dim, eps=eps), laws.Physics(laws.EULER, dim, eps=1.0)
    disc = make(laws.EULER, dim, 2, eps=eps)
    w = disc.to_grid(euler_state(disc, rng))
    w1 = w.copy()
    w1[-1] = w1[-1] / eps ** 2
    for m in range(dim):
        F, F1 = laws.flux(w, m, ph), laws.flux(w1, m, ph1)
        F1[-1] = F1[-1] * eps ** 2
        np.testing.assert_allclose(F, F1, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(laws.max_speed(w, m, ph), laws.max_speed(w1, m, ph1), rtol=1e-13)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_euler_max_speed_is_spectral_radius(dim):
    rng = np.random.default_rng(23)
    ph = laws.Physics(laws.EULER, dim, eps=0.5)
    nv = dim + 2
    for _ in range(5):
        rho = 1 + 0.2 * rng.random()
        v = 0.5 * rng.standard_normal(dim)
        p = 1 + 0.2 * rng.random()
        w = np.array([rho, *(rho * v), p / 0.4 + 0.5 * 0.25 * rho * v @ v])
        for m in range(dim):
            A = np.zeros((nv, nv))
            for k in range(nv):
                e = np.zeros(nv)
                e[k] = 1.0
                A[:, k] = laws.flux_jvp(w, e, m, ph)
            lam = np.abs(np.linalg.eigvals(A)).max()
            assert abs(laws.max_speed(w, m, ph) - lam) < 1e-12 * lam
