"""1-D nodal basis of the DGSEM (Sec. 3.1.1, Eq. 11 and the abbreviations after
Eq. 12).  Test infrastructure only (see ``oracle/__init__``).

The solution in one direction is the Lagrange interpolant through N+1 nodes
xi_0..xi_N on [-1, 1]; quadrature collocates on the same nodes with weights
omega_i.  The paper names Gauss-Legendre nodes; Gauss-Lobatto nodes are the other
supported family (both are textbook quadratures, Kopriva 2009, ch. 1).

Quantities (all FP64):
  nodes, weights           xi_i, omega_i
  D[i, j]   = l_j'(xi_i)   polynomial derivative matrix
  Dhat[i, j] = -(omega_j / omega_i) l_i'(xi_j)      (= -M^-1 D^T M)
  lhat_m[i] = l_i(-1) / omega_i,  lhat_p[i] = l_i(+1) / omega_i
  l_m[i] = l_i(-1), l_p[i] = l_i(+1)   (evaluation of the polynomial at the edges)

Reading of the paper: the printed Dhat has the weight ratio omega_i/omega_j; the
weak form (Eq. 10) with collocation gives omega_j/omega_i.  The tests pin the
latter by the free-stream property, discrete conservation and polynomial
exactness of the full operator.
"""
import numpy as np

LOBATTO = "lobatto"
GAUSS = "gauss"


def legendre(n, x):
    """P_n(x) and P_n'(x) by the three-term recurrence (Bonnet)."""
    x = np.asarray(x, dtype=np.float64)
    p0, p1 = np.ones_like(x), x.copy()
    if n == 0:
        return p0, np.zeros_like(x)
    d0, d1 = np.zeros_like(x), np.ones_like(x)
    for k in range(2, n + 1):
        p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
        d2 = d0 + (2 * k - 1) * p1
        p0, p1, d0, d1 = p1, p2, d1, d2
    return p1, d1


def gauss_legendre(N):
    """N+1 Gauss-Legendre nodes (roots of P_{N+1}) and weights."""
    n = N + 1
    x = -np.cos(np.pi * (np.arange(n) + 0.75) / (n + 0.5))
    for _ in range(100):
        p, dp = legendre(n, x)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    p, dp = legendre(n, x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    return x, w


def gauss_lobatto(N):
    """N+1 Gauss-Lobatto nodes (+-1 and the roots of P_N') and weights."""
    if N == 1:
        return np.array([-1.0, 1.0]), np.array([1.0, 1.0])
    x = -np.cos(np.pi * np.arange(N + 1) / N)  # Chebyshev-Lobatto start
    for _ in range(100):
        # roots of q(x) = P_{N+1} - P_{N-1} = (2N+1)/(N(N+1)) (x^2-1) P_N'
        pN1, dN1 = legendre(N + 1, x[1:-1])
        pNm1, dNm1 = legendre(N - 1, x[1:-1])
        q = pN1 - pNm1
        dq = dN1 - dNm1
        dx = q / dq
        x[1:-1] = x[1:-1] - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    x[0], x[-1] = -1.0, 1.0
    pN, _ = legendre(N, x)
    w = 2.0 / (N * (N + 1) * pN * pN)
    return x, w


def nodes_weights(N, family):
    if family == LOBATTO:
        return gauss_lobatto(N)
    if family == GAUSS:
        return gauss_legendre(N)
    raise ValueError(family)


def lagrange_eval(nodes, x):
    """Matrix L[k, i] = l_i(x_k) of the Lagrange basis through `nodes`, by the
    product definition l_i(x) = prod_{m != i} (x - xi_m)/(xi_i - xi_m)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    L = np.ones((len(x), n))
    for i in range(n):
        for m in range(n):
            if m != i:
                L[:, i] *= (x - nodes[m]) / (nodes[i] - nodes[m])
    return L


def derivative_matrix(nodes):
    """D[i, j] = l_j'(xi_i).  Off-diagonal from the barycentric formula
    l_j'(xi_i) = (b_j / b_i) / (xi_i - xi_j); the diagonal is the negative row
    sum, since the derivative of the constant 1 = sum_j l_j is zero."""
    n = len(nodes)
    b = np.ones(n)
    for j in range(n):
        for m in range(n):
            if m != j:
                b[j] /= (nodes[j] - nodes[m])
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (b[j] / b[i]) / (nodes[i] - nodes[j])
        D[i, i] = -np.sum(D[i, :])
    return D


class Basis:
    """All 1-D operators of the DGSEM for degree N on the given node family."""

    def __init__(self, N, family=LOBATTO):
        self.N = N
        self.p = N + 1
        self.family = family
        self.nodes, self.weights = nodes_weights(N, family)
        self.D = derivative_matrix(self.nodes)
        w = self.weights
        # Dhat[i, j] = -(w_j / w_i) * l_i'(xi_j) = -(w_j / w_i) * D[j, i]
        self.Dhat = -(w[None, :] / w[:, None]) * self.D.T
        self.l_m = lagrange_eval(self.nodes, -1.0)[0]
        self.l_p = lagrange_eval(self.nodes, 1.0)[0]
        self.lhat_m = self.l_m / w
        self.lhat_p = self.l_p / w
