"""Pins of the oracle's 1-D basis (Sec. 3.1.1) against textbook facts."""
import numpy as np
import pytest

from oracle.basis import Basis, GAUSS, LOBATTO, gauss_legendre, gauss_lobatto


def test_lobatto_n2_closed_form():
    x, w = gauss_lobatto(2)
    np.testing.assert_allclose(x, [-1.0, 0.0, 1.0], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 3, 4 / 3, 1 / 3], rtol=1e-15)


def test_gauss_n1_closed_form():
    x, w = gauss_legendre(1)
    np.testing.assert_allclose(x, [-1 / np.sqrt(3), 1 / np.sqrt(3)], rtol=1e-15)
    np.testing.assert_allclose(w, [1.0, 1.0], rtol=1e-15)


def test_lobatto_n4_closed_form():
    x, w = gauss_lobatto(4)
    r = np.sqrt(3.0 / 7.0)
    np.testing.assert_allclose(x, [-1, -r, 0, r, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], rtol=1e-14)


@pytest.mark.parametrize("family,extra", [(LOBATTO, -1), (GAUSS, 1)])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_quadrature_exactness(N, family, extra):
    b = Basis(N, family)
    deg = 2 * N + extra
    for k in range(deg + 1):
        exact = (1 - (-1) ** (k + 1)) / (k + 1)
        assert abs(np.dot(b.weights, b.nodes ** k) - exact) < 1e-13
    # one degree higher is not exact (the rule is sharp)
    k = deg + 1
    if k % 2 == 0:
        exact = 2.0 / (k + 1)
        assert abs(np.dot(b.weights, b.nodes ** k) - exact) > 1e-10


@pytest.mark.parametrize("family", [LOBATTO, GAUSS])
@pytest.mark.parametrize("N", [1, 3, 5, 7])
def test_derivative_matrix_exact_on_polynomials(N, family):
    b = Basis(N, family)
    for k in range(N + 1):
        f = b.nodes ** k
        df = k * b.nodes ** (k - 1) if k > 0 else np.zeros_like(b.nodes)
        np.testing.assert_allclose(b.D @ f, df, atol=1e-12)
    np.testing.assert_allclose(b.D.sum(axis=1), 0.0, atol=1e-13)


@pytest.mark.parametrize("family", [LOBATTO, GAUSS])
@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_dhat_weak_form_identity(N, family):
    """Dhat from the weak form: omega_i Dhat_ij = -omega_j l_i'(xi_j).  Check it
    by integrating the test function derivative against a polynomial: for f of
    degree <= N, sum_j Dhat_ij f_j = -(1/omega_i) int l_i' f  (exact quadrature
    for degree 2N-1)."""
    b = Basis(N, family)
    xq, wq = gauss_legendre(N + 2)
    from oracle.basis import lagrange_eval, derivative_matrix
    Lq = lagrange_eval(b.nodes, xq)            # l_i at quadrature points
    Dq = Lq @ b.D                              # l_j'(xq) ... for interpolant derivative
    rng = np.random.default_rng(3)
    f = rng.standard_normal(N + 1)             # nodal values of a degree-N poly
    fq = Lq @ f
    for i in range(N + 1):
        e = np.zeros(N + 1)
        e[i] = 1.0
        dli = Lq @ (b.D @ e)                   # l_i'(xq)
        integral = np.dot(wq, dli * fq)
        assert abs((b.Dhat @ f)[i] + integral / b.weights[i]) < 1e-12


@pytest.mark.parametrize("family", [LOBATTO, GAUSS])
@pytest.mark.parametrize("N", [2, 3, 4, 5, 6])
def test_dhat_centro_symmetry(N, family):
    b = Basis(N, family)
    np.testing.assert_allclose(b.Dhat[::-1, ::-1], -b.Dhat, atol=1e-12)


@pytest.mark.parametrize("N", [2, 3, 5])
def test_lobatto_sbp(N):
    """Summation by parts for Lobatto: M D + (M D)^T = diag(-1, 0, .., 0, 1)."""
    b = Basis(N, LOBATTO)
    Q = np.diag(b.weights) @ b.D
    B = np.zeros((N + 1, N + 1))
    B[0, 0], B[-1, -1] = -1.0, 1.0
    np.testing.assert_allclose(Q + Q.T, B, atol=1e-13)
    np.testing.assert_allclose(b.lhat_p, np.eye(N + 1)[-1] / b.weights[-1], atol=1e-15)
