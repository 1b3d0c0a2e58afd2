// Host computation of the 1-D DGSEM basis (Sec. 3.1.1): Gauss-Legendre or
// Gauss-Lobatto nodes and weights, the Lagrange derivative matrix, the weak-form
// matrix Dhat = -M^-1 D^T M and the edge evaluations l_i(+-1).
#include "hbpc_internal.h"

#include <cmath>
#include <vector>

namespace hbpc {

// Legendre polynomial P_n and its derivative at x (three-term recurrence).
static void legendre(int n, double x, double& p, double& dp) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) { p = 1.0; dp = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    const double d2 = d0 + (2.0 * k - 1.0) * p1;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  p = p1; dp = d1;
}

static const double kPi = 3.14159265358979323846;

bool basis_1d(int N, int family, Basis1D& b) {
  if (N < 1 || N + 1 > kMaxNodes) return false;
  const int p = N + 1;
  b.N = N;
  b.xi.assign(p, 0.0);
  b.w.assign(p, 0.0);
  if (family == 1) {  // Gauss-Legendre: roots of P_{N+1}
    for (int k = 0; k < p; ++k) {
      double x = -std::cos(kPi * (k + 0.75) / (p + 0.5));
      for (int it = 0; it < 100; ++it) {
        double P, dP;
        legendre(p, x, P, dP);
        const double dx = P / dP;
        x -= dx;
        if (std::fabs(dx) < 1e-16) break;
      }
      double P, dP;
      legendre(p, x, P, dP);
      b.xi[k] = x;
      b.w[k] = 2.0 / ((1.0 - x * x) * dP * dP);
    }
  } else {            // Gauss-Lobatto: +-1 and roots of P_N'
    b.xi[0] = -1.0;
    b.xi[N] = 1.0;
    for (int k = 1; k < N; ++k) {
      double x = -std::cos(kPi * k / N);
      for (int it = 0; it < 100; ++it) {
        // f = (1 - x^2) P_N'(x); f' = -N(N+1) P_N(x)
        double P, dP;
        legendre(N, x, P, dP);
        const double f = (1.0 - x * x) * dP;
        const double df = -N * (N + 1.0) * P;
        const double dx = f / df;
        x -= dx;
        if (std::fabs(dx) < 1e-16) break;
      }
      b.xi[k] = x;
    }
    for (int k = 0; k < p; ++k) {
      double P, dP;
      legendre(N, b.xi[k], P, dP);
      b.w[k] = 2.0 / (N * (N + 1.0) * P * P);
    }
  }
  // barycentric weights and derivative matrix D[i][j] = l_j'(xi_i)
  std::vector<double> bw(p, 1.0);
  for (int j = 0; j < p; ++j)
    for (int m = 0; m < p; ++m)
      if (m != j) bw[j] /= (b.xi[j] - b.xi[m]);
  std::vector<double> D(p * p, 0.0);
  for (int i = 0; i < p; ++i) {
    double diag = 0.0;
    for (int j = 0; j < p; ++j) {
      if (i == j) continue;
      D[i * p + j] = (bw[j] / bw[i]) / (b.xi[i] - b.xi[j]);
      diag -= D[i * p + j];
    }
    D[i * p + i] = diag;
  }
  b.D = D;
  // Dhat[i][j] = -(w_j / w_i) l_i'(xi_j) = -(w_j / w_i) D[j][i]
  b.Dhat.assign(p * p, 0.0);
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j) b.Dhat[i * p + j] = -(b.w[j] / b.w[i]) * D[j * p + i];
  // l_i(+-1) by the barycentric interpolation formula
  b.lm.assign(p, 0.0);
  b.lp.assign(p, 0.0);
  for (int side = 0; side < 2; ++side) {
    const double x = side ? 1.0 : -1.0;
    std::vector<double>& out = side ? b.lp : b.lm;
    int hit = -1;
    for (int j = 0; j < p; ++j)
      if (x == b.xi[j]) hit = j;
    if (hit >= 0) { out[hit] = 1.0; continue; }
    double den = 0.0;
    for (int j = 0; j < p; ++j) den += bw[j] / (x - b.xi[j]);
    for (int j = 0; j < p; ++j) out[j] = (bw[j] / (x - b.xi[j])) / den;
  }
  // derivative of the interpolant at the edges: l_j'(+-1) = sum_i l_i(+-1) D[i][j]
  // (l_j' has degree N - 1, so its interpolant through the nodes is exact)
  b.dm.assign(p, 0.0);
  b.dp.assign(p, 0.0);
  for (int j = 0; j < p; ++j)
    for (int i = 0; i < p; ++i) {
      b.dm[j] += b.lm[i] * D[i * p + j];
      b.dp[j] += b.lp[i] * D[i * p + j];
    }
  return true;
}

void br2_tables(const Basis1D& b, double h, double eta, double* Dg, double* gp, double* gm,
                double* bp, double* bm, double* Vloc) {
  const int p = b.N + 1;
  const double H = 2.0 / h;
  double cp = 0.0, cm = 0.0;
  for (int i = 0; i < p; ++i) {
    cp += b.lp[i] * b.lp[i] / b.w[i];
    cm += b.lm[i] * b.lm[i] / b.w[i];
  }
  for (int i = 0; i < p; ++i) {
    for (int j = 0; j < p; ++j) Dg[i * p + j] = H * b.D[i * p + j];
    gp[i] = H * b.dp[i];
    gm[i] = H * b.dm[i];
  }
  *bp = H * eta * cp;
  *bm = H * eta * cm;
  // element-diagonal block of the viscous operator along one line (neighbours'
  // values zero), per unit viscosity: column j is the response to u = e_j.
  //   u*_+ = u(+1)/2, u*_- = u(-1)/2
  //   face gradients (averages of the two face-local liftings):
  //     + face: 1/2 [u'(+1) + eta c_p (u*_+ - u(+1)) + eta c_m (0 - u*_+)]
  //     - face: 1/2 [eta c_p (u*_- - 0) + u'(-1) + eta c_m (u(-1) - u*_-)]   (times H)
  //   lifted gradient d_l = H [ (D u)_l + lhat_l(+1)(u*_+ - u(+1)) - lhat_l(-1)(u*_- - u(-1)) ]
  //   V_ij = H [ sum_l Dhat_il d_l + lhat_i(+1) fgrad_+ - lhat_i(-1) fgrad_- ]
  std::vector<double> d(p);
  for (int j = 0; j < p; ++j) {
    const double up = b.lp[j], um = b.lm[j];
    const double usp = 0.5 * up, usm = 0.5 * um;
    const double fgp = 0.5 * (H * b.dp[j] + H * eta * cp * (usp - up) + H * eta * cm * (0.0 - usp));
    const double fgm = 0.5 * (H * eta * cp * (usm - 0.0) + H * b.dm[j] + H * eta * cm * (um - usm));
    for (int l = 0; l < p; ++l)
      d[l] = H * (b.D[l * p + j] + (b.lp[l] / b.w[l]) * (usp - up) - (b.lm[l] / b.w[l]) * (usm - um));
    for (int i = 0; i < p; ++i) {
      double acc = 0.0;
      for (int l = 0; l < p; ++l) acc += b.Dhat[i * p + l] * d[l];
      Vloc[i * p + j] = H * (acc + (b.lp[i] / b.w[i]) * fgp - (b.lm[i] / b.w[i]) * fgm);
    }
  }
}

}  // namespace hbpc
