"""Pins of the oracle's stage solver (Sec. 3.2, 4.2) and full HBPC-DGSEM steps:
matrix-free Newton-GMRES against a dense complex-step Newton with LU, the
BJ_ext inverse against the explicit block matrix, and linear advection
against the exact per-Fourier-mode HBPC and semi-discrete solutions."""
import numpy as np
import pytest

from oracle import dgsem, exact, hbpc, laws, newton
from tests.test_oracle_dgsem import euler_state


def tiny(law, dim, N=2, n=(2, 2, 2), flux="lf"):
    ph = laws.Physics(law, dim, a=(1.0, 0.5, 0.25), flux=flux)
    return dgsem.Disc(dgsem.Mesh(dim, n, (0, 0, 0), (1, 1, 1)), N, ph)


def stage_inputs(disc, rng):
    if disc.ph.law == laws.EULER:
        w = euler_state(disc, rng)
    else:
        w = 0.5 + 0.3 * rng.standard_normal(disc.shape)
    b = w + 0.01 * rng.standard_normal(disc.shape)
    return w, b


CASES = [(laws.ADVECTION, 1, "lf"), (laws.ADVECTION, 2, "lf"), (laws.BURGERS, 1, "rusanov"),
         (laws.BURGERS, 2, "lf"), (laws.EULER, 2, "lf"), (laws.EULER, 2, "rusanov"),
         (laws.EULER, 1, "rusanov")]


@pytest.mark.parametrize("law,dim,flux", CASES)
@pytest.mark.parametrize("alphas", [(0.5, 1.0 / 6.0), (1.0, 1.0)])
def test_jfnk_matches_dense_newton(law, dim, flux, alphas):
    disc = tiny(law, dim, flux=flux)
    rng = np.random.default_rng(11)
    W0, b = stage_inputs(disc, rng)
    dt = 0.05
    a1, a2 = alphas
    R1 = lambda w: dgsem.R1(disc, w)
    R2 = lambda w, s: dgsem.R2(disc, w, s)
    Wd, Sd = exact.dense_newton(R1, R2, b, a1, a2, dt, W0)
    for jv in ("fd", "analytic") if not disc.ph.linear else ("linear", "fd"):
        opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-14, gmres_tol=1e-8,
                                    restart=400, jv=jv)
        W, S, st = newton.newton_solve(disc, b, a1, a2, dt, W0, opts)
        assert st.converged
        err = np.linalg.norm(W - Wd) / np.linalg.norm(Wd)
        assert err < 1e-12, (jv, err)


@pytest.mark.parametrize("law,dim,flux", [(laws.EULER, 2, "lf"), (laws.ADVECTION, 2, "lf"),
                                          (laws.BURGERS, 1, "rusanov")])
def test_bjext_blocks(law, dim, flux):
    """J_i equals the diagonal block of dR1/dw (complex step, LF flux) and the
    four blocks D,E,F,G invert the element block matrix [[A, B], [C, I]]."""
    disc = tiny(law, dim, flux=flux)
    rng = np.random.default_rng(12)
    W, b = stage_inputs(disc, rng)
    sysm = newton.StageSystem(disc, b, 0.5, 1.0 / 6.0, 0.07)
    pc = newton.BJExt(sysm, W)
    nE, nb = pc.nE, pc.nb
    if flux == "lf":
        h = 1e-30
        for k in range(nb):
            v = np.zeros((nE, nb))
            v[:, k] = 1.0
            # perturb only element 0, read element 0's rows
            v[1:] = 0.0
            col = np.imag(dgsem.R1(disc, W + 1j * h * v.reshape(disc.shape))) / h
            np.testing.assert_allclose(pc.J[0, :, k], col.reshape(nE, nb)[0], atol=1e-10)
    I = np.eye(nb)
    for e in range(nE):
        J = pc.J[e]
        P = np.block([[I - sysm.c1 * J, sysm.c2 * J], [-J, I]])
        D, E, F, G = (x[e] for x in pc.blocks())
        Pinv = np.block([[D, E], [F, G]])
        np.testing.assert_allclose(Pinv @ P, np.eye(2 * nb), atol=1e-11)


def test_bjext_preconditioned_newton_same_root_fewer_iterations():
    """Smooth Euler stage (density wave of Eq. 22) at a large time step."""
    from paper_2109_04804_gb300 import inputs
    ph = laws.Physics(laws.EULER, 2, flux="lf")
    disc = dgsem.Disc(dgsem.Mesh(2, (3, 3), (-1, -1), (1, 1)), 3, ph)
    W0 = inputs.density_wave(disc.node_coords())
    b = W0.copy()
    res = {}
    for pc in ("none", "bjext"):
        opts = newton.NewtonOptions(tol_rel=1e-12, tol_abs=1e-14, gmres_tol=1e-6, restart=300,
                                    gmres_maxiter=600, newton_max=8, jv="fd", pc=pc)
        W, S, st = newton.newton_solve(disc, b, 0.5, 1 / 6, 0.2, W0, opts)
        assert st.converged
        res[pc] = (W, st.gmres_its)
    assert np.linalg.norm(res["none"][0] - res["bjext"][0]) < 1e-11 * np.linalg.norm(W)
    assert res["bjext"][1] < res["none"][1]


def test_c1_advection_hbpc4_matches_fourier_exact():
    """1-D advection, 16 elements N=3, HBPC(4,0), CFL 1 (dt = 1/64), 16 steps:
    the matrix-free path equals the exact per-mode HBPC to Newton tolerance."""
    ph = laws.Physics(laws.ADVECTION, 1)
    disc = dgsem.Disc(dgsem.Mesh(1, (16,), (0,), (1,)), 3, ph)
    x = disc.node_coords()[0]
    w0 = np.sin(2 * np.pi * x)[:, None]
    dt = 1.0 / 64
    opts = newton.NewtonOptions(tol_rel=1e-12, tol_abs=1e-14, gmres_tol=1e-8, restart=100,
                                jv="linear")
    adv = hbpc.dg_stepper(disc, dt, 4, 0, opts)
    w = w0
    for _ in range(16):
        w = adv(w)
    wf = exact.fourier_hbpc(disc, w0, dt, 4, 0, 16)
    assert np.abs(w - wf).max() < 1e-12
    # and the dense-matrix route gives the same fully discrete answer
    L = exact.linear_matrix(disc)
    st = exact.dense_stepper(L, dt, 4, 0)
    wd = w0.ravel()
    for _ in range(16):
        wd = st(wd)
    assert np.abs(wd - wf.ravel()).max() < 1e-12


@pytest.mark.parametrize("q,kmax", [(6, 1), (8, 2)])
def test_2d_advection_matches_fourier_exact(q, kmax):
    ph = laws.Physics(laws.ADVECTION, 2, a=(1.0, 1.0))
    disc = dgsem.Disc(dgsem.Mesh(2, (4, 4), (0, 0), (1, 1)), 3, ph)
    X = disc.node_coords()
    w0 = (np.sin(2 * np.pi * X[0]) * np.sin(2 * np.pi * X[1]))[:, None]
    dt = 0.02
    opts = newton.NewtonOptions(tol_rel=1e-12, tol_abs=1e-14, gmres_tol=1e-8, restart=200,
                                jv="linear")
    adv = hbpc.dg_stepper(disc, dt, q, kmax, opts)
    w = w0
    for _ in range(3):
        w = adv(w)
    wf = exact.fourier_hbpc(disc, w0, dt, q, kmax, 3)
    assert np.abs(w - wf).max() < 1e-12


def test_temporal_order_pde_fourier():
    """Order min(4+k, q) of the fully discrete scheme against exp(T L) for 1-D
    advection (exact per-mode evaluation; Sec. 4.3.1)."""
    ph = laws.Physics(laws.ADVECTION, 1)
    disc = dgsem.Disc(dgsem.Mesh(1, (4,), (0,), (1,)), 2, ph)
    x = disc.node_coords()[0]
    w0 = np.sin(2 * np.pi * x)[:, None]
    T = 1.0
    ref = exact.fourier_semidiscrete(disc, w0, T)
    for q, kmax in [(4, 0), (6, 0), (6, 1), (6, 2), (8, 1), (8, 2), (8, 4)]:
        errs = []
        for n in (16, 32):
            errs.append(np.abs(exact.fourier_hbpc(disc, w0, T / n, q, kmax, n) - ref).max())
        order = np.log2(errs[0] / errs[1])
        expect = min(4 + kmax, q)
        assert expect - 0.5 < order < expect + 1.5, (q, kmax, order, errs)


def test_hbpc4_independent_of_k_pde():
    """HBPC(4, k) gives the same answer for every k (Sec. 4.3.1)."""
    disc = tiny(laws.BURGERS, 1, N=3, n=(6,), flux="rusanov")
    x = disc.node_coords()[0]
    w0 = (0.5 + 0.3 * np.sin(2 * np.pi * x))[:, None]
    opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-15, gmres_tol=1e-10, restart=200)
    out = []
    for k in (0, 1, 2):
        adv = hbpc.dg_stepper(disc, 0.05, 4, k, opts)
        out.append(adv(w0))
    assert np.abs(out[1] - out[0]).max() < 1e-12
    assert np.abs(out[2] - out[0]).max() < 1e-12


def test_conservation_over_steps():
    disc = tiny(laws.EULER, 2, N=2, n=(3, 3), flux="rusanov")
    rng = np.random.default_rng(14)
    w0 = euler_state(disc, rng)
    opts = newton.NewtonOptions(tol_rel=1e-12, tol_abs=1e-14, gmres_tol=1e-6, restart=200)
    adv = hbpc.dg_stepper(disc, 0.05, 6, 1, opts)
    w = adv(w0)
    c0, c1 = dgsem.cell_integral(disc, w0), dgsem.cell_integral(disc, w)
    assert np.all(np.abs(c1 - c0) < 1e-11 * np.abs(c0).max())
