"""HBPC(q, k_max) time stepping, Algorithm 1 (Sec. 2.1), with the two-derivative
Butcher tableaux of Appendix A (Eq. A.1-A.3).  Test infrastructure only (see
``oracle/__init__``).

One step from w^{n-1} (stage 1 of every level is w^{n-1}):
  predictor, l = 2..s:   solve  W - a1 dt R1(W) + (a2 dt^2/2) R2(W)
                              = w_{l-1} + a1 dt R1(w_{l-1}) + (a2 dt^2/2) R2(w_{l-1})
                         with a1 = dc_l / 2, a2 = dc_l^2 / 6, dc_l = c_l - c_{l-1}
                         (Eq. 5 written as Eq. 7/8)
  corrector, k = 0..k_max-1, l = 2..s:
                         solve  W - dt R1(W) + (dt^2/2) R2(W)
                              = w^{n-1} - dt R1(w_l^k) + (dt^2/2) R2(w_l^k) + I_l^k
                         I_l^k = dt sum_j B1_lj R1(w_j^k) + dt^2 sum_j B2_lj R2(w_j^k)
                         (Eq. 6; reading: Eq. 9 omits I_l, Eq. 6 keeps it)
  update                 w^n = w_s^{k_max}
Here R2(w) means R2(w, R1(w)) (remark in Sec. 2.1).  The stage solver is a
callback solve(b, a1, a2, guess); its initial guess is w_{l-1} in the predictor
and w_l^k in the corrector (the paper does not state one).
"""
from fractions import Fraction as Fr

import numpy as np


def tableau_exact(q):
    """(c, B1, B2) as Fractions, Eq. A.1 (q=4), A.2 (q=6), A.3 (q=8)."""
    if q == 4:
        c = [Fr(0), Fr(1)]
        B1 = [[Fr(0), Fr(0)], [Fr(1, 2), Fr(1, 2)]]
        B2 = [[Fr(0), Fr(0)], [Fr(1, 12), Fr(-1, 12)]]
    elif q == 6:
        c = [Fr(0), Fr(1, 2), Fr(1)]
        B1 = [[Fr(0)] * 3,
              [Fr(101, 480), Fr(8, 30), Fr(55, 2400)],
              [Fr(7, 30), Fr(16, 30), Fr(7, 30)]]
        B2 = [[Fr(0)] * 3,
              [Fr(65, 4800), Fr(-25, 600), Fr(-25, 8000)],
              [Fr(5, 300), Fr(0), Fr(-5, 300)]]
    elif q == 8:
        c = [Fr(0), Fr(1, 3), Fr(2, 3), Fr(1)]
        B1 = [[Fr(0)] * 4,
              [Fr(6893, 54432), Fr(313, 2016), Fr(89, 2016), Fr(397, 54432)],
              [Fr(223, 1701), Fr(20, 63), Fr(13, 63), Fr(20, 1701)],
              [Fr(31, 224), Fr(81, 224), Fr(81, 224), Fr(31, 224)]]
        B2 = [[Fr(0)] * 4,
              [Fr(1283, 272160), Fr(-851, 30240), Fr(-269, 30240), Fr(-163, 272160)],
              [Fr(43, 8505), Fr(-16, 945), Fr(-19, 945), Fr(-8, 8505)],
              [Fr(19, 3360), Fr(-9, 1120), Fr(9, 1120), Fr(-19, 3360)]]
    else:
        raise ValueError("q must be 4, 6 or 8")
    return c, B1, B2


def tableau(q):
    c, B1, B2 = tableau_exact(q)
    return (np.array([float(x) for x in c]),
            np.array([[float(x) for x in r] for r in B1]),
            np.array([[float(x) for x in r] for r in B2]))


def step(w_prev, dt, q, kmax, R1, R2, solve):
    """One HBPC(q, kmax) step of Algorithm 1.  R1(w), R2(w, sigma) and
    solve(b, a1, a2, guess) -> W are callbacks."""
    c, B1, B2 = tableau(q)
    s = len(c)
    w = [None] * s
    r1 = [None] * s
    r2 = [None] * s
    w[0] = w_prev
    r1[0] = R1(w_prev)
    r2[0] = R2(w_prev, r1[0])
    # predictor
    for l in range(1, s):
        dc = c[l] - c[l - 1]
        a1, a2 = dc / 2.0, dc * dc / 6.0
        b = w[l - 1] + a1 * dt * r1[l - 1] + (a2 * dt * dt / 2.0) * r2[l - 1]
        w[l] = solve(b, a1, a2, w[l - 1])
        r1[l] = R1(w[l])
        r2[l] = R2(w[l], r1[l])
    # corrector sweeps
    for k in range(kmax):
        wn, r1n, r2n = list(w), list(r1), list(r2)
        for l in range(1, s):
            I = dt * sum(B1[l, j] * r1[j] for j in range(s)) \
                + dt * dt * sum(B2[l, j] * r2[j] for j in range(s))
            b = w[0] - dt * r1[l] + (dt * dt / 2.0) * r2[l] + I
            wn[l] = solve(b, 1.0, 1.0, w[l])
            r1n[l] = R1(wn[l])
            r2n[l] = R2(wn[l], r1n[l])
        w, r1, r2 = wn, r1n, r2n
    return w[s - 1]


def dg_stepper(disc, dt, q, kmax, opts, stats=None):
    """Return a function w -> w^{n+1} for the DGSEM discretisation `disc`, with
    every stage solved by Newton-GMRES (oracle.newton)."""
    from . import dgsem, newton
    st = stats if stats is not None else newton.Stats()

    def R1(w):
        st.r1_evals += 1
        return dgsem.R1(disc, w)

    def R2(w, s):
        st.r2_evals += 1
        return dgsem.R2(disc, w, s)

    def solve(b, a1, a2, guess):
        W, _, _ = newton.newton_solve(disc, b, a1, a2, dt, guess, opts, st)
        return W

    def advance(w):
        return step(w, dt, q, kmax, R1, R2, solve)

    advance.stats = st
    return advance
