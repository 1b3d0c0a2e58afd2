// Internal interfaces of libhbpc shared by its translation units.
#pragma once
#include <cuda_runtime.h>
#include <vector>

#include "dg_common.cuh"

namespace hbpc {

constexpr int kMaxNodes = kMaxP;

struct Basis1D {
  int N = 0;
  std::vector<double> xi, w, Dhat, lm, lp;
};
bool basis_1d(int N, int family, Basis1D& b);

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
};

// Returns false if the combination was not compiled.
bool get_ops(int law, int dim, int P, bool lobatto, OpsTable& out);

}  // namespace hbpc
