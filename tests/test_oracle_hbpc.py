"""Pins of the oracle's HBPC driver (Algorithm 1) and tableaux (Appendix A)."""
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import exact, hbpc


@pytest.mark.parametrize("q", [4, 6, 8])
def test_tableau_order_conditions(q):
    """Row l integrates exactly to order q: for r = 0..q-1
       sum_j B1_lj c_j^r + r sum_j B2_lj c_j^(r-1) = c_l^(r+1) / (r+1),
    i.e. the quadrature of int_0^{c_l} t^r using y' and y'' data (Sec. 2.1)."""
    c, B1, B2 = hbpc.tableau_exact(q)
    s = len(c)
    for l in range(1, s):
        for r in range(q):
            lhs = sum(B1[l][j] * c[j] ** r for j in range(s))
            if r > 0:
                lhs += r * sum(B2[l][j] * c[j] ** (r - 1) for j in range(s))
            assert lhs == c[l] ** (r + 1) / (r + 1), (q, l, r)
    assert all(x == 0 for x in B1[0] + B2[0])


def scalar(lam):
    R1 = lambda w: lam * w
    R2 = lambda w, s: lam * s
    return R1, R2


def scalar_stepper(dt, q, kmax, R1, R2):
    def solve(b, a1, a2, guess):
        W, _ = exact.dense_newton(R1, R2, b, a1, a2, dt, np.atleast_1d(guess))
        return W
    return lambda w: hbpc.step(np.atleast_1d(w), dt, q, kmax, R1, R2, solve)


@pytest.mark.parametrize("kmax", [0, 1, 2])
@pytest.mark.parametrize("z", [-0.3, -2.0, -10.0, 0.5 + 1.2j, -1.0 + 4.0j])
def test_hbpc4_is_pade22(z, kmax):
    """HBPC(4, k) on y' = lam y has the (2,2) Pade amplification
    (1 + z/2 + z^2/12) / (1 - z/2 + z^2/12), independent of k."""
    R1, R2 = scalar(z)
    I = np.eye(1)
    solve = lambda b, a1, a2, g: b / (1 - a1 * z + a2 / 2 * z * z)
    y = hbpc.step(np.array([1.0 + 0j]), 1.0, 4, kmax, R1, R2, solve)
    pade = (1 + z / 2 + z * z / 12) / (1 - z / 2 + z * z / 12)
    assert abs(y[0] - pade) < 1e-14 * max(1, abs(pade))


@pytest.mark.parametrize("q,kmax", [(4, 0), (6, 0), (6, 1), (6, 2), (8, 1), (8, 2), (8, 3), (8, 4)])
def test_order_nonlinear_scalar(q, kmax):
    """y' = -y^2 + cos(y) ... use y' = -y^2, y(0)=1: y = 1/(1+t).  Observed order
    equals min(4 + k_max, q) (remark after Algorithm 1)."""
    R1 = lambda w: -w * w
    R2 = lambda w, s: -2.0 * w * s
    T = 1.0
    errs = []
    ns = (4, 8) if q == 8 and kmax >= 3 else (8, 16)
    for n in ns:
        dt = T / n
        step = scalar_stepper(dt, q, kmax, R1, R2)
        y = np.array([1.0])
        for _ in range(n):
            y = step(y)
        errs.append(abs(y[0] - 1.0 / (1.0 + T)))
    order = np.log2(errs[0] / errs[1])
    expect = min(4 + kmax, q)
    assert expect - 0.6 < order < expect + 1.3, (order, errs)


@pytest.mark.parametrize("q", [6, 8])
def test_corrector_fixed_point_is_collocation(q):
    """With many corrections the stages converge to the limiting Hermite-Birkhoff
    RK solution: w_l = w_1 + I_l for every stage (Sec. 2.1)."""
    z = -1.5
    R1, R2 = scalar(z)
    dt = 1.0
    c, B1, B2 = hbpc.tableau(q)
    s = len(c)
    # limiting method: solve the linear collocation system for the stage values
    A = np.eye(s) - dt * z * B1 - dt * dt * z * z * B2
    A[0] = 0.0
    A[0, 0] = 1.0
    rhs = np.zeros(s)
    rhs[0] = 1.0
    rhs[1:] = 1.0
    ws = np.linalg.solve(A, rhs)
    solve = lambda b, a1, a2, g: b / (1 - a1 * z + a2 / 2 * z * z)
    y = hbpc.step(np.array([1.0]), dt, q, 60, R1, R2, solve)
    assert abs(y[0] - ws[-1]) < 1e-12
