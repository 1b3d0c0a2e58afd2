"""Implicit stage solve of the HBPC scheme: extended residual, matrix-free
Jacobian-vector product, GMRES, Newton and the BJ_ext and BJ^H_ext preconditioners.
Test infrastructure only (see ``oracle/__init__``).

Extended unknown X = (W, sigma) (Sec. 3.2.1).  Residual (reading: the printed
G_1 = W - b - g(W) subtracts W twice; the Jacobian of Eq. 18 fixes it as)
    G_1 = W - b - alpha1 dt R1(W) + (alpha2 dt^2 / 2) R2(W, sigma)
    G_2 = sigma - R1(W)
Newton (Eq. 17): J dX = -G, X <- X + dX, stopped when ||G(X^r)|| <= tol_rel
||G(X^0)|| or when ||dW|| <= tol_abs (Sec. 5.2 adds the absolute test).

Jv (Sec. 4.2):
  "fd"     Eq. 23 with eps_FD = sqrt(eps_machine) / (eps ||d.||_2) per block,
           eps_machine = 2^-52 (the Fortran epsilon of a double);
  "linear" the right-hand form of Eq. 24 (exact for a linear flux), R1 of a
           direction taken as its linear part R2(W, .) (boundary data dropped);
  "analytic" Eq. 18 with dR1/dW v = R2(W, v) (identity of Sec. 3.2.1) and the
           Hessian block by the FD quotient of Eq. 23.

Schur form (Sec. 3.2.4, Eq. 19): Newton with the linear system reduced to the
W unknowns, J_Schur dW = -G1 + (a2 dt^2/2) dR2/dsigma . G2,
dsigma = -G2 + dR1/dW dW, J_Schur = I - a1 dt dR1/dW + (a2 dt^2/2) dR2/dW
+ (a2 dt^2/2) (dR1/dW)^2; its products reuse the extended product above on
(v, dR1/dW v), whose first half is J_Schur v.

GMRES: restarted, right preconditioned, modified Gram-Schmidt Arnoldi with
Givens rotations and zero initial guess (textbook form, Saad 2003, Alg. 6.9 /
9.5), relative tolerance against the norm of the right-hand side.
"""
import numpy as np

from . import dgsem

EPS_MACHINE = 2.0 ** -52


class Stats:
    def __init__(self):
        self.newton_its = 0
        self.gmres_its = 0
        self.r1_evals = 0
        self.r2_evals = 0
        self.converged = True


class StageSystem:
    """G(X) = 0 of one predictor or corrector stage (Eq. 7 with Eq. 8/9)."""

    def __init__(self, disc, b, alpha1, alpha2, dt, stats=None):
        self.disc, self.b = disc, b
        self.c1 = alpha1 * dt
        self.c2 = alpha2 * dt * dt / 2.0
        self.n = disc.ndof
        self.stats = stats if stats is not None else Stats()

    def split(self, X):
        return X[:self.n].reshape(self.disc.shape), X[self.n:].reshape(self.disc.shape)

    def R1(self, w):
        self.stats.r1_evals += 1
        return dgsem.R1(self.disc, w)

    def R2(self, w, s):
        self.stats.r2_evals += 1
        return dgsem.R2(self.disc, w, s)

    def residual(self, X):
        W, S = self.split(X)
        r1 = self.R1(W)
        r2 = self.R2(W, S)
        G1 = W - self.b - self.c1 * r1 + self.c2 * r2
        G2 = S - r1
        return np.concatenate([G1.ravel(), G2.ravel()]), r1, r2

    def jv(self, X, r1, r2, dX, mode):
        W, S = self.split(X)
        dW, dS = self.split(dX)
        eps_ref = self.disc.ph.eps
        if mode == "linear":
            # Eq. 24 for a linear flux: R1 of the direction, taken as its
            # linear part dR1/dW v = R2(W, v) (Sec. 3.2.1), which equals R1(v)
            # on a periodic mesh and drops the data of a Dirichlet boundary,
            # where R1 is affine
            q1 = self.R2(W, dW)
            top = dW - self.c1 * q1 + self.c2 * self.R2(W, dS)
            bot = -q1 + dS
            return np.concatenate([top.ravel(), bot.ravel()])
        nw, ns = np.linalg.norm(dW), np.linalg.norm(dS)
        if nw > 0:
            ew = np.sqrt(EPS_MACHINE) / (eps_ref * nw)
            Wp = W + ew * dW
            if mode == "fd":
                dr1 = (self.R1(Wp) - r1) / ew
            else:
                dr1 = self.R2(W, dW)
            dr2w = (self.R2(Wp, S) - r2) / ew
        else:
            dr1 = np.zeros_like(W)
            dr2w = np.zeros_like(W)
        if ns > 0:
            if mode == "fd":
                es = np.sqrt(EPS_MACHINE) / (eps_ref * ns)
                dr2s = (self.R2(W, S + es * dS) - r2) / es
            else:
                dr2s = self.R2(W, dS)
        else:
            dr2s = np.zeros_like(W)
        top = dW - self.c1 * dr1 + self.c2 * dr2w + self.c2 * dr2s
        bot = -dr1 + dS
        return np.concatenate([top.ravel(), bot.ravel()])


def gmres(matvec, rhs, tol, restart, maxiter, precond=None):
    """Solve A x = rhs from x0 = 0 with restarted right-preconditioned GMRES.
    Returns (x, iterations, converged)."""
    n = rhs.size
    x = np.zeros(n, dtype=rhs.dtype)
    bnorm = np.linalg.norm(rhs)
    if bnorm == 0.0:
        return x, 0, True
    target = tol * bnorm
    its = 0
    r = rhs.copy()
    while True:
        beta = np.linalg.norm(r)
        if beta <= target:
            return x, its, True
        m = restart
        V = np.zeros((m + 1, n), dtype=rhs.dtype)
        Z = np.zeros((m, n), dtype=rhs.dtype)
        H = np.zeros((m + 1, m), dtype=rhs.dtype)
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_end = 0
        done = False
        for j in range(m):
            Z[j] = precond(V[j]) if precond is not None else V[j]
            wv = matvec(Z[j])
            for i in range(j + 1):              # modified Gram-Schmidt
                H[i, j] = np.dot(wv, V[i])
                wv = wv - H[i, j] * V[i]
            hnext = np.linalg.norm(wv)
            H[j + 1, j] = hnext
            if hnext > 0:
                V[j + 1] = wv / hnext
            for i in range(j):                   # apply previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_end = j + 1
            if abs(g[j + 1]) <= target or its >= maxiter or hnext == 0.0:
                done = abs(g[j + 1]) <= target or hnext == 0.0
                break
        y = np.zeros(j_end)
        for i in range(j_end - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:j_end], y[i + 1:j_end])) / H[i, i]
        x = x + y @ Z[:j_end]
        if done:
            return x, its, True
        if its >= maxiter:
            return x, its, False
        r = rhs - matvec(x)


def element_jacobians(disc, W):
    """J_i = dR1/dW restricted to element i (neighbours frozen), column k of
    every element at once as R2(W, e_k) with the neighbours' sigma traces zero
    (dR2/dsigma = dR1/dW, Sec. 3.2.1).  Returns (n_E, n_b, n_b)."""
    nE = disc.mesh.nE
    nb = disc.ndof // nE
    J = np.zeros((nE, nb, nb))
    for k in range(nb):
        v = np.zeros((nE, nb))
        v[:, k] = 1.0
        col = dgsem.operator(disc, W, v.reshape(disc.shape), mode="R2", frozen_neighbor=True)
        J[:, :, k] = col.reshape(nE, nb)
    return J


def element_hessian_blocks(disc, W, S, h=1e-30):
    """H_i = dR2/dW restricted to element i at fixed sigma = S (neighbour
    states and sigma fixed), the Hessian contribution of Sec. 3.2.2, column k
    of every element at once by complex step in the elements' own node k:
        H_i[:, k] = Im R2(W + i h e_k, S) / h
    with the neighbours' traces real (operator's frozen_neighbor_state).
    Exact to rounding for h = 1e-30 (no subtraction).  Returns (n_E, n_b, n_b)."""
    nE = disc.mesh.nE
    nb = disc.ndof // nE
    H = np.zeros((nE, nb, nb))
    W0 = np.asarray(W, dtype=np.complex128).reshape(nE, nb)
    for k in range(nb):
        Wc = W0.copy()
        Wc[:, k] += 1j * h
        col = dgsem.operator(disc, Wc.reshape(disc.shape), S, mode="R2", frozen_neighbor_state=True)
        H[:, :, k] = np.imag(col).reshape(nE, nb) / h
    return H


class BJExt:
    """BJ_ext preconditioner (Sec. 3.2.3): per element J_i = dR1/dW restricted
    to the element (neighbour dependencies neglected), M_i = (A_i - B_i C_i)^-1
    = (I - a1 dt J_i + (a2 dt^2/2) J_i^2)^-1 by LU, and
        P^-1 (w, s) = (D w + E s, F w + G s),  D = M, E = -B M, F = -C M, G = A M
    with A = I - a1 dt J, B = (a2 dt^2/2) J, C = -J."""

    def __init__(self, system, W):
        disc = system.disc
        nE = disc.mesh.nE
        nb = disc.ndof // nE
        J = element_jacobians(disc, W)
        I = np.eye(nb)[None]
        S = I - system.c1 * J + system.c2 * (J @ J)
        self.J = J
        self.M = np.linalg.inv(S)
        self.c1, self.c2 = system.c1, system.c2
        self.nE, self.nb, self.n = nE, nb, disc.ndof
        self._blocks = self.blocks()

    def blocks(self):
        I = np.eye(self.nb)[None]
        A = I - self.c1 * self.J
        B = self.c2 * self.J
        C = -self.J
        return self.M, -B @ self.M, -C @ self.M, A @ self.M

    def __call__(self, X):
        D, E, F, G = self._blocks
        w = X[:self.n].reshape(self.nE, self.nb, 1)
        s = X[self.n:].reshape(self.nE, self.nb, 1)
        top = D @ w + E @ s
        bot = F @ w + G @ s
        return np.concatenate([top.ravel(), bot.ravel()])


class BJExtH:
    """BJ^H_ext preconditioner (Sec. 3.2.3): the blocks of P keep the Hessian
    contribution in A,
        A_i = I - a1 dt J_i + (a2 dt^2/2) H_i,  B_i = (a2 dt^2/2) J_i,  C_i = -J_i,
    with J_i of BJ_ext and H_i = element_hessian_blocks at the current (W,
    sigma).  A_i no longer commutes with B_i, so the inverse blocks are
        D = M, E = -M B, F = -C M, G = I + C M B,  M = (A - B C)^-1
    with A - B C = I - a1 dt J + (a2 dt^2/2) H + (a2 dt^2/2) J^2 (one LU per
    element), and P^-1 (w, s) = (D w + E s, F w + G s)."""

    def __init__(self, system, W, S):
        disc = system.disc
        nE = disc.mesh.nE
        nb = disc.ndof // nE
        self.J = element_jacobians(disc, W)
        self.H = element_hessian_blocks(disc, W, S)
        I = np.eye(nb)[None]
        self.c1, self.c2 = system.c1, system.c2
        A = I - self.c1 * self.J + self.c2 * self.H
        B = self.c2 * self.J
        C = -self.J
        self.M = np.linalg.inv(A - B @ C)
        self.nE, self.nb, self.n = nE, nb, disc.ndof
        self._blocks = (self.M, -self.M @ B, -C @ self.M, I + C @ self.M @ B)

    def __call__(self, X):
        D, E, F, G = self._blocks
        w = X[:self.n].reshape(self.nE, self.nb, 1)
        s = X[self.n:].reshape(self.nE, self.nb, 1)
        top = D @ w + E @ s
        bot = F @ w + G @ s
        return np.concatenate([top.ravel(), bot.ravel()])


def make_preconditioner(sysm, X, kind):
    """None, BJ_ext ("bjext") or BJ^H_ext ("bjext_h") at X = (W, sigma)."""
    W, S = sysm.split(X)
    if kind == "bjext":
        return BJExt(sysm, W)
    if kind == "bjext_h":
        return BJExtH(sysm, W, S)
    if kind == "none":
        return None
    raise ValueError(kind)


class NewtonOptions:
    def __init__(self, tol_rel=1e-12, tol_abs=0.0, gmres_tol=1e-5, restart=100,
                 gmres_maxiter=7000, newton_max=50, jv="fd", pc="none"):
        self.tol_rel, self.tol_abs = tol_rel, tol_abs
        self.gmres_tol, self.restart = gmres_tol, restart
        self.gmres_maxiter, self.newton_max = gmres_maxiter, newton_max
        self.jv, self.pc = jv, pc


def newton_solve(disc, b, alpha1, alpha2, dt, W0, opts, stats=None):
    """Solve G(X) = 0 from X^0 = (W0, R1(W0)).  Returns (W, sigma, stats)."""
    sysm = StageSystem(disc, b, alpha1, alpha2, dt, stats)
    st = sysm.stats
    X = np.concatenate([W0.ravel(), sysm.R1(W0).ravel()])
    G, r1, r2 = sysm.residual(X)
    g0 = np.linalg.norm(G)
    converged = g0 == 0.0
    r = 0
    while not converged and r < opts.newton_max:
        pc = make_preconditioner(sysm, X, opts.pc)
        dX, its, _ = gmres(lambda v: sysm.jv(X, r1, r2, v, opts.jv), -G,
                           opts.gmres_tol, opts.restart, opts.gmres_maxiter, pc)
        st.gmres_its += its
        X = X + dX
        r += 1
        st.newton_its += 1
        G, r1, r2 = sysm.residual(X)
        converged = (np.linalg.norm(G) <= opts.tol_rel * g0
                     or np.linalg.norm(dX[:sysm.n]) <= opts.tol_abs)
    st.converged = st.converged and converged
    W, S = sysm.split(X)
    return W.copy(), S.copy(), st


def schur_step(sysm, X, r1, r2, G, opts):
    """One Newton increment dX = (dW, dsigma) of Sec. 3.2.4 at X (residual G,
    r1 = R1(W), r2 = R2(W, sigma)):
        J_Schur dW = -G1 + (a2 dt^2/2) (dR2/dsigma) G2,
        dsigma     = -G2 + (dR1/dW) dW,
    J_Schur of Eq. 19.  R2 is linear in sigma, so (dR2/dsigma) G2 = R2(W, G2).
    dR1/dW v is the second half of the extended product on (v, 0) with the sign
    turned, and J_Schur v the first half of the extended product on
    (v, dR1/dW v), in the same form (opts.jv) as newton_solve.  With
    opts.pc == "bjext" GMRES is right preconditioned by the element blocks
    (I - a1 dt J_i + (a2 dt^2/2) J_i^2)^-1 (the D block of BJ_ext, the
    element-local J_Schur without the Hessian); with "bjext_h" by the D block
    of BJ^H_ext, (I - a1 dt J_i + (a2 dt^2/2) (H_i + J_i^2))^-1.  Returns (dX, GMRES iterations)."""
    disc, n = sysm.disc, sysm.n
    zero = np.zeros(n)
    W, _ = sysm.split(X)
    G1, G2 = G[:n], G[n:]

    def dr1(v):
        return -sysm.jv(X, r1, r2, np.concatenate([v, zero]), opts.jv)[n:]

    def jschur(v):
        return sysm.jv(X, r1, r2, np.concatenate([v, dr1(v)]), opts.jv)[:n]

    rhs = -G1 + sysm.c2 * sysm.R2(W, G2.reshape(disc.shape)).ravel()
    pc = None
    if opts.pc in ("bjext", "bjext_h"):
        blocks = make_preconditioner(sysm, X, opts.pc)

        def pc(v, M=blocks.M):
            return (M @ v.reshape(blocks.nE, blocks.nb, 1)).ravel()

    dW, its, _ = gmres(jschur, rhs, opts.gmres_tol, opts.restart, opts.gmres_maxiter, pc)
    dS = -G2 + dr1(dW)
    return np.concatenate([dW, dS]), its


def schur_newton_solve(disc, b, alpha1, alpha2, dt, W0, opts, stats=None):
    """Solve G(X) = 0 from X^0 = (W0, R1(W0)) with the Schur-complement linear
    system of Sec. 3.2.4 in every Newton step (schur_step); the same stopping
    tests as newton_solve.  Returns (W, sigma, stats)."""
    sysm = StageSystem(disc, b, alpha1, alpha2, dt, stats)
    st = sysm.stats
    n = sysm.n
    X = np.concatenate([W0.ravel(), sysm.R1(W0).ravel()])
    G, r1, r2 = sysm.residual(X)
    g0 = np.linalg.norm(G)
    converged = g0 == 0.0
    r = 0
    while not converged and r < opts.newton_max:
        dX, its = schur_step(sysm, X, r1, r2, G, opts)
        st.gmres_its += its
        X = X + dX
        r += 1
        st.newton_its += 1
        G, r1, r2 = sysm.residual(X)
        converged = (np.linalg.norm(G) <= opts.tol_rel * g0
                     or np.linalg.norm(dX[:n]) <= opts.tol_abs)
    st.converged = st.converged and converged
    W, S = sysm.split(X)
    return W.copy(), S.copy(), st
