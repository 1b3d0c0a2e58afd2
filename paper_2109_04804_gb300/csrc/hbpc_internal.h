// Internal interfaces of libhbpc shared by its translation units.
#pragma once
#include <cuda_runtime.h>
#include <vector>

#include "dg_common.cuh"

namespace hbpc {

constexpr int kMaxNodes = kMaxP;

struct Basis1D {
  int N = 0;
  std::vector<double> xi, w, D, Dhat, lm, lp;
  std::vector<double> dm, dp;   // l_j'(-1), l_j'(+1)
};
bool basis_1d(int N, int family, Basis1D& b);

// Tables of the BR2 viscous term (Sec. 5.1.1) for one direction with element
// size h: Dg = (2/h) D (p x p, row-major), gp/gm = (2/h) l_j'(+-1),
// bp/bm = (2/h) eta c_pm with c_pm = sum_i l_i(+-1)^2 / omega_i, and Vloc, the
// element-diagonal block of the viscous operator along one line per unit
// viscosity (p x p, row-major; neighbours' values zero).
void br2_tables(const Basis1D& b, double h, double eta, double* Dg, double* gp, double* gm,
                double* bp, double* bm, double* Vloc);

template <typename S> struct JvInputT;
using JvInput = JvInputT<double>;
struct JvCoef;

// Launchers of the element operator for one (law, dim, P, node family).
struct OpsTable {
  int nv = 0;
  void (*r1)(const DGParams<double>&, const double* w, double* out, cudaStream_t) = nullptr;
  void (*r2)(const DGParams<double>&, const double* w, const double* s, double* out,
             cudaStream_t) = nullptr;
  void (*residual)(const DGParams<double>&, const double* W, const double* S, const double* b,
                   double c1, double c2, double* G1, double* G2, double* r1, double* r2,
                   cudaStream_t) = nullptr;
  // Jv per Eq. 23 (two launches) or Eq. 24 (one launch, linear flux)
  void (*jv_fd)(const DGParams<double>&, const double* W, const double* S, const double* r1,
                const double* r2, const JvInput&, const JvCoef&, cudaStream_t) = nullptr;
  void (*jv_linear)(const DGParams<double>&, const JvInput&, const JvCoef&, cudaStream_t) = nullptr;
  // mixed precision: FP32 Jacobian-vector product at the FP32 copy (Wf, Sf)
  void (*jv_f)(const DGParams<float>&, const JvInputT<float>&, const JvCoef&, const float* Wf,
               const float* Sf, cudaStream_t) = nullptr;
  // BJ_ext element Jacobians J_i (Sec. 3.2.3), column-major n_b x n_b per element
  void (*pc_assemble)(const DGParams<double>&, const double* W, double* J, cudaStream_t) = nullptr;
  void (*pc_assemble_f)(const DGParams<float>&, const double* W, float* J, cudaStream_t) = nullptr;
  // BJ^H_ext Hessian blocks H_i = dR2/dW|_i at (W, sigma = S), same layout;
  // null for a linear flux (H = 0) and for Navier-Stokes
  void (*pc_hessian)(const DGParams<double>&, const double* W, const double* S, double* H,
                     cudaStream_t) = nullptr;
  void (*pc_hessian_f)(const DGParams<float>&, const double* W, const double* S, float* H,
                       cudaStream_t) = nullptr;
};

// Returns false if the combination was not compiled.
bool get_ops(int law, int dim, int P, bool lobatto, OpsTable& out);

}  // namespace hbpc
