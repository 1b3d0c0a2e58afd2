"""Pins of the oracle's BJ^H_ext preconditioner (Sec. 3.2.3).

The element blocks H_i = dR2/dW|_i (the Hessian contribution, Sec. 3.2.2) are
compared with the diagonal blocks of the full dR2/dW built one global unknown
at a time by complex step of the plain operator (no neighbour freezing); J_i
likewise with the full dR1/dW.  The closed-form inverse blocks D, E, F, G are
compared with a dense solve of the assembled block-diagonal P.  A linear flux
has H = 0 (Sec. 3.2.1), where BJ^H_ext and BJ_ext coincide.  A stage solved
with BJ^H_ext reaches the root of the dense complex-step Newton."""
import numpy as np
import pytest

from oracle import dgsem, exact, laws, newton
from oracle.basis import GAUSS, LOBATTO
from tests.test_oracle_newton import euler_state


def disc_of(law, dim, N, n, flux, family=LOBATTO, nu=0.0):
    ph = laws.Physics(law, dim, a=(1.0, 0.5, 0.25), flux=flux, nu=nu)
    return dgsem.Disc(dgsem.Mesh(dim, n, (0, 0, 0), (1, 1, 1)), N, ph, family=family)


def state(disc, rng):
    if disc.ph.law == laws.EULER:
        return euler_state(disc, rng)
    return 0.6 + 0.3 * rng.standard_normal(disc.shape)


def smooth_sigma(disc):
    """A sigma continuous across element faces at Lobatto nodes (the nodal
    values of smooth periodic functions), so that its face jumps vanish."""
    x = disc.node_coords()
    f = [np.sin(2 * np.pi * x[0]) + 0.3, np.cos(2 * np.pi * x[-1]) - 0.2,
         np.sin(2 * np.pi * (x[0] + x[-1])), 0.5 * np.cos(2 * np.pi * x[0]) + 0.1]
    return np.stack([f[v % 4] for v in range(disc.ph.nv)], axis=1)   # (n_E, n_var, nodes)


def dense_derivative(disc, fun, W, h=1e-30):
    """d fun / dW by complex step, one global unknown at a time (n x n)."""
    n = disc.ndof
    W0 = np.asarray(W, dtype=np.complex128).ravel()
    D = np.zeros((n, n))
    for g in range(n):
        Wc = W0.copy()
        Wc[g] += 1j * h
        D[:, g] = np.imag(fun(Wc.reshape(disc.shape))).ravel() / h
    return D


def diag_blocks(D, nE):
    nb = D.shape[0] // nE
    return np.stack([D[e * nb:(e + 1) * nb, e * nb:(e + 1) * nb] for e in range(nE)])


HCASES = [
    # law, dim, N, n, flux, family, smooth sigma (needed when kappa depends on W)
    (laws.EULER, 2, 2, (3, 3), "lf", LOBATTO, False),
    (laws.EULER, 2, 2, (3, 2), "lf", GAUSS, False),
    (laws.EULER, 1, 3, (4,), "rusanov", LOBATTO, True),
    (laws.EULER, 2, 2, (3, 3), "rusanov", LOBATTO, True),
    (laws.BURGERS, 2, 3, (3, 2), "lf", GAUSS, False),
    (laws.BURGERS, 1, 4, (5,), "rusanov", LOBATTO, True),
]


@pytest.mark.parametrize("law,dim,N,n,flux,family,smooth", HCASES)
def test_hessian_blocks_are_the_diagonal_blocks_of_dR2_dW(law, dim, N, n, flux, family, smooth):
    """H_i equals the element-diagonal block of the full dR2/dW at fixed sigma.
    With the Rusanov flux kappa depends on W; its derivative multiplies the
    sigma jump, which a face-continuous sigma makes zero, so the comparison is
    exact there too (the oracle's blocks do not differentiate kappa)."""
    disc = disc_of(law, dim, N, n, flux, family)
    rng = np.random.default_rng(41)
    W = state(disc, rng)
    S = smooth_sigma(disc) if smooth else rng.standard_normal(disc.shape)
    H = newton.element_hessian_blocks(disc, W, S)
    Hd = diag_blocks(dense_derivative(disc, lambda w: dgsem.operator(disc, w, S, mode="R2"), W), disc.mesh.nE)
    scale = np.abs(Hd).max()
    assert scale > 1e-3              # the Hessian contribution is not zero here
    assert np.abs(H - Hd).max() <= 1e-11 * scale


@pytest.mark.parametrize("law,dim,N,n,flux,family,smooth", HCASES[:2] + HCASES[4:5])
def test_element_jacobians_are_the_diagonal_blocks_of_dR1_dW(law, dim, N, n, flux, family, smooth):
    """J_i (R2 with a unit sigma and the neighbours' sigma zero) equals the
    element-diagonal block of the full dR1/dW (constant kappa: global LF)."""
    disc = disc_of(law, dim, N, n, flux, family)
    W = state(disc, np.random.default_rng(42))
    J = newton.element_jacobians(disc, W)
    Jd = diag_blocks(dense_derivative(disc, lambda w: dgsem.operator(disc, w, mode="R1"), W), disc.mesh.nE)
    assert np.abs(J - Jd).max() <= 1e-11 * np.abs(Jd).max()


@pytest.mark.parametrize("law,dim,N,n,flux,family", [
    (laws.EULER, 2, 2, (3, 2), "lf", LOBATTO), (laws.EULER, 2, 2, (2, 3), "lf", GAUSS),
    (laws.BURGERS, 1, 3, (4,), "lf", LOBATTO)])
def test_apply_is_the_inverse_of_the_assembled_P(law, dim, N, n, flux, family):
    """P^-1 of BJ^H_ext against a dense solve with P assembled from the
    definitions of Sec. 3.2.3, A_i = I - a1 dt dR1/dW|_i + (a2 dt^2/2) dR2/dW|_i,
    B_i = (a2 dt^2/2) dR1/dW|_i, C_i = -dR1/dW|_i, with the element blocks taken
    from the full complex-step matrices."""
    disc = disc_of(law, dim, N, n, flux, family)
    rng = np.random.default_rng(43)
    W = state(disc, rng)
    S = rng.standard_normal(disc.shape)
    dt, a1, a2 = 0.3, 0.5, 1.0 / 6.0
    sysm = newton.StageSystem(disc, W, a1, a2, dt)
    X = np.concatenate([W.ravel(), S.ravel()])
    pc = newton.make_preconditioner(sysm, X, "bjext_h")
    nE, n_ = disc.mesh.nE, disc.ndof
    nb = n_ // nE
    Jd = diag_blocks(dense_derivative(disc, lambda w: dgsem.operator(disc, w, mode="R1"), W), nE)
    Hd = diag_blocks(dense_derivative(disc, lambda w: dgsem.operator(disc, w, S, mode="R2"), W), nE)
    c1, c2 = a1 * dt, a2 * dt * dt / 2
    P = np.zeros((2 * n_, 2 * n_))
    for e in range(nE):
        iw = slice(e * nb, (e + 1) * nb)
        isg = slice(n_ + e * nb, n_ + (e + 1) * nb)
        P[iw, iw] = np.eye(nb) - c1 * Jd[e] + c2 * Hd[e]
        P[iw, isg] = c2 * Jd[e]
        P[isg, iw] = -Jd[e]
        P[isg, isg] = np.eye(nb)
    assert np.abs(c2 * Hd).max() > 1e-4 * np.abs(c1 * Jd).max()
    for trial in range(3):
        x = rng.standard_normal(2 * n_)
        ref = np.linalg.solve(P, x)
        assert np.linalg.norm(pc(x) - ref) <= 1e-11 * np.linalg.norm(ref)


def test_linear_flux_has_no_hessian_and_matches_bjext():
    disc = disc_of(laws.ADVECTION, 2, 3, (3, 2), "lf")
    rng = np.random.default_rng(44)
    W = rng.standard_normal(disc.shape)
    S = rng.standard_normal(disc.shape)
    sysm = newton.StageSystem(disc, W, 1.0, 1.0, 0.2)
    X = np.concatenate([W.ravel(), S.ravel()])
    ph = newton.make_preconditioner(sysm, X, "bjext_h")
    p = newton.make_preconditioner(sysm, X, "bjext")
    assert np.abs(ph.H).max() == 0.0
    for _ in range(2):
        x = rng.standard_normal(2 * disc.ndof)
        assert np.linalg.norm(ph(x) - p(x)) <= 1e-13 * np.linalg.norm(p(x))


@pytest.mark.parametrize("law,dim,flux", [(laws.EULER, 2, "rusanov"), (laws.BURGERS, 1, "rusanov"),
                                          (laws.EULER, 2, "lf")])
def test_newton_with_bjext_h_reaches_the_dense_root(law, dim, flux):
    """A stage at a large time step: the JFNK Newton right preconditioned by
    BJ^H_ext reaches the dense Newton's root, and the preconditioner cuts the
    GMRES iterations against no preconditioner."""
    disc = disc_of(law, dim, 2, (3, 3)[:dim] if dim == 2 else (4,), flux)
    rng = np.random.default_rng(45)
    W0 = state(disc, rng)
    b = W0 + 0.01 * rng.standard_normal(disc.shape)
    dt, a1, a2 = 0.3, 0.5, 1.0 / 6.0
    Wd, Sd = exact.dense_newton(lambda w: dgsem.R1(disc, w), lambda w, s: dgsem.R2(disc, w, s), b, a1, a2, dt, W0)
    its = {}
    for pc in ("none", "bjext_h"):
        opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-14, gmres_tol=1e-10, restart=600, jv="fd", pc=pc)
        W, S, st = newton.newton_solve(disc, b, a1, a2, dt, W0, opts)
        assert st.converged
        assert np.linalg.norm(W - Wd) <= 1e-10 * np.linalg.norm(Wd)
        its[pc] = st.gmres_its
    assert its["bjext_h"] < its["none"]
