"""Pins of the oracle's Schur-complement Newton (Sec. 3.2.4, Eq. 19): its root
is the root of G(X) = 0 that the dense complex-step Newton with LU finds, its
system matrix is I - c1 L + c2 L^2 for a linear flux (L the dense matrix of
R1), and the element blocks of its preconditioner invert the element-local
Schur matrix."""
import numpy as np
import pytest

from oracle import dgsem, exact, laws, newton
from tests.test_oracle_newton import CASES, stage_inputs, tiny


@pytest.mark.parametrize("law,dim,flux", CASES)
@pytest.mark.parametrize("pc", ["none", "bjext"])
def test_schur_newton_matches_dense_newton(law, dim, flux, pc):
    disc = tiny(law, dim, flux=flux)
    rng = np.random.default_rng(31)
    W0, b = stage_inputs(disc, rng)
    dt, a1, a2 = 0.05, 0.5, 1.0 / 6.0
    R1 = lambda w: dgsem.R1(disc, w)
    R2 = lambda w, s: dgsem.R2(disc, w, s)
    Wd, Sd = exact.dense_newton(R1, R2, b, a1, a2, dt, W0)
    jv = "linear" if disc.ph.linear else "fd"
    opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-14, gmres_tol=1e-9, restart=400, jv=jv, pc=pc)
    W, S, st = newton.schur_newton_solve(disc, b, a1, a2, dt, W0, opts)
    assert st.converged
    assert np.linalg.norm(W - Wd) <= 1e-12 * np.linalg.norm(Wd)
    assert np.linalg.norm(S - Sd) <= 1e-10 * max(np.linalg.norm(Sd), 1.0)


def test_schur_matrix_of_linear_advection():
    """For a linear flux J_Schur = I - c1 L + c2 L^2 (Eq. 19 with dR2/dw = 0):
    the oracle's Schur products, column by column, equal that dense matrix."""
    disc = tiny(laws.ADVECTION, 2, N=2, n=(3, 2))
    L = exact.linear_matrix(disc)
    n = disc.ndof
    dt, a1, a2 = 0.07, 1.0, 1.0
    c1, c2 = a1 * dt, a2 * dt * dt / 2
    sysm = newton.StageSystem(disc, np.zeros(disc.shape), a1, a2, dt)
    X = np.concatenate([np.zeros(n), np.zeros(n)])
    _, r1, r2 = sysm.residual(X)
    ref = np.eye(n) - c1 * L + c2 * L @ L
    zero = np.zeros(n)
    cols = []
    for k in range(n):
        v = np.zeros(n)
        v[k] = 1.0
        t = -sysm.jv(X, r1, r2, np.concatenate([v, zero]), "linear")[n:]
        cols.append(sysm.jv(X, r1, r2, np.concatenate([v, t]), "linear")[:n])
    assert np.abs(np.array(cols).T - ref).max() <= 1e-12 * np.abs(ref).max()


def test_schur_and_extended_newton_agree_on_euler():
    """A nonlinear stage (Euler, Rusanov) solved both ways: the same root."""
    disc = tiny(laws.EULER, 2, N=3, n=(3, 2), flux="rusanov")
    rng = np.random.default_rng(32)
    W0, b = stage_inputs(disc, rng)
    opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-14, gmres_tol=1e-9, restart=400, jv="fd", pc="bjext")
    We, Se, _ = newton.newton_solve(disc, b, 1.0, 1.0, 0.04, W0, opts)
    Ws, Ss, st = newton.schur_newton_solve(disc, b, 1.0, 1.0, 0.04, W0, opts)
    assert st.converged
    assert np.linalg.norm(Ws - We) <= 1e-11 * np.linalg.norm(We)


@pytest.mark.parametrize("law,dim,flux", [(laws.ADVECTION, 2, "lf"), (laws.EULER, 2, "lf"), (laws.BURGERS, 1, "rusanov")])
def test_schur_step_is_the_extended_step(law, dim, flux):
    """The Schur form is an exact block elimination of the extended Newton
    system (Sec. 3.2.4): at a point X with G2 != 0 (sigma not R1(W)) and with
    the linear systems solved tightly, the Schur increment equals the extended
    one, -J^-1 G, in both halves."""
    disc = tiny(law, dim, flux=flux)
    rng = np.random.default_rng(33)
    W, b = stage_inputs(disc, rng)
    sysm = newton.StageSystem(disc, b, 0.5, 1.0 / 6.0, 0.05)
    S = dgsem.R1(disc, W) + 0.05 * rng.standard_normal(disc.shape)
    X = np.concatenate([W.ravel(), S.ravel()])
    G, r1, r2 = sysm.residual(X)
    assert np.linalg.norm(G[sysm.n:]) > 1e-3 * np.linalg.norm(G)
    # dR1/dW exactly (R2 of Sec. 3.2.1) in both forms; the Hessian block is an
    # Eq. 23 quotient in both, along different directions (1e-9 apart)
    jv = "linear" if disc.ph.linear else "analytic"
    opts = newton.NewtonOptions(gmres_tol=1e-13, restart=400, jv=jv)
    de, _, _ = newton.gmres(lambda v: sysm.jv(X, r1, r2, v, jv), -G, 1e-13, 400, 7000)
    ds, _ = newton.schur_step(sysm, X, r1, r2, G, opts)
    n = sysm.n
    tol = 1e-10 if disc.ph.linear else 1e-7
    assert np.linalg.norm(ds[:n] - de[:n]) <= tol * np.linalg.norm(de[:n])
    assert np.linalg.norm(ds[n:] - de[n:]) <= tol * np.linalg.norm(de[n:])
