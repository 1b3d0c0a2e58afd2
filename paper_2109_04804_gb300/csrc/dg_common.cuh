// Shared definitions of the DGSEM kernels: operator parameters and the
// physical fluxes of the supported conservation laws.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace hbpc {

constexpr int kMaxP = 8;     // nodes per direction (N + 1 <= 8)

constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

enum Law { LAW_ADV = 0, LAW_BURGERS = 1, LAW_EULER = 2 };

// Operator parameters, passed by value (kernel parameter space).  All matrices
// already carry the Cartesian metric -(2/h_m) of the reference-element
// transformation (Sec. 3.1.1), so the element operator of Eq. 12 is
//   R1_i = sum_m [ sum_l Dvol[m][i][l] G^m_l + sp[m][i] f*_{+m} + sm[m][i] f*_{-m} ]
// with G^m the nodal flux (for advection the state itself, a_m folded in Dvol).
template <typename T>
struct DGParams {
  int n[3];                 // elements per direction (1 for unused directions)
  int nE;
  T Dvol[3][kMaxP][kMaxP];  // -(2/h_m) Dhat (times a_m for advection)
  T sp[3][kMaxP];           // -(2/h_m) lhat_i(+1)
  T sm[3][kMaxP];           // -(2/h_m) lhat_i(-1)
  T lp[kMaxP], lm[kMaxP];   // l_i(+1), l_i(-1): traces
  T a[3];
  T gm1;                    // gamma - 1
  T gamma;
  T eps2, inv_eps2, inv_eps;
  T lam[3][5];              // global-LF kappa per direction and variable
  int rusanov;
};

// ---------------------------------------------------------------------------
// Physical fluxes.  flux_all: F^m(w) for every direction m; jvp_all: the
// directional derivative (dF^m/dw) s; speed: max |eigenvalue| of dF^m/dw.
// ---------------------------------------------------------------------------
template <int DIM, typename T>
struct Advection {
  static constexpr int NV = 1;
  static constexpr bool LINEAR = true;
  __device__ __forceinline__ static void flux_all(const T* w, T (*F)[NV], const DGParams<T>& p) {
#pragma unroll
    for (int m = 0; m < DIM; ++m) F[m][0] = p.a[m] * w[0];
  }
  __device__ __forceinline__ static void flux(const T* w, int m, T* F, const DGParams<T>& p) {
    F[0] = p.a[m] * w[0];
  }
  __device__ __forceinline__ static void jvp(const T* w, const T* s, int m, T* J, const DGParams<T>& p) {
    J[0] = p.a[m] * s[0];
  }
  __device__ __forceinline__ static T speed(const T* w, int m, const DGParams<T>& p) {
    return fabs(p.a[m]);
  }
};

template <int DIM, typename T>
struct Burgers {
  static constexpr int NV = 1;
  static constexpr bool LINEAR = false;
  __device__ __forceinline__ static void flux_all(const T* w, T (*F)[NV], const DGParams<T>& p) {
    const T f = T(0.5) * w[0] * w[0];
#pragma unroll
    for (int m = 0; m < DIM; ++m) F[m][0] = f;
  }
  __device__ __forceinline__ static void jvp_all(const T* w, const T* s, T (*J)[NV], const DGParams<T>& p) {
    const T f = w[0] * s[0];
#pragma unroll
    for (int m = 0; m < DIM; ++m) J[m][0] = f;
  }
  __device__ __forceinline__ static void flux(const T* w, int m, T* F, const DGParams<T>& p) {
    F[0] = T(0.5) * w[0] * w[0];
  }
  __device__ __forceinline__ static void jvp(const T* w, const T* s, int m, T* J, const DGParams<T>& p) {
    J[0] = w[0] * s[0];
  }
  __device__ __forceinline__ static T speed(const T* w, int m, const DGParams<T>& p) {
    return fabs(w[0]);
  }
};

// Euler with reference Mach number eps (Eq. 21):
//   F^m = (rho v_m, rho v_m v + p/eps^2 e_m, v_m (E + p)),
//   p = (gamma - 1)(E - eps^2/2 rho |v|^2),  c = sqrt(gamma p / rho) / eps.
template <int DIM, typename T>
struct Euler {
  static constexpr int NV = DIM + 2;
  static constexpr bool LINEAR = false;
  __device__ __forceinline__ static void flux_all(const T* w, T (*F)[NV], const DGParams<T>& p) {
    const T ir = T(1) / w[0];
    T v[DIM], v2 = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) { v[k] = w[1 + k] * ir; v2 += v[k] * v[k]; }
    const T E = w[DIM + 1];
    const T pr = p.gm1 * (E - T(0.5) * p.eps2 * w[0] * v2);
    const T pe = pr * p.inv_eps2;
#pragma unroll
    for (int m = 0; m < DIM; ++m) {
      F[m][0] = w[1 + m];
#pragma unroll
      for (int k = 0; k < DIM; ++k) F[m][1 + k] = w[1 + m] * v[k] + (k == m ? pe : T(0));
      F[m][DIM + 1] = v[m] * (E + pr);
    }
  }
  __device__ __forceinline__ static void flux(const T* w, int m, T* F, const DGParams<T>& p) {
    const T ir = T(1) / w[0];
    T v[DIM], v2 = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) { v[k] = w[1 + k] * ir; v2 += v[k] * v[k]; }
    const T E = w[DIM + 1];
    const T pr = p.gm1 * (E - T(0.5) * p.eps2 * w[0] * v2);
    F[0] = w[1 + m];
#pragma unroll
    for (int k = 0; k < DIM; ++k) F[1 + k] = w[1 + m] * v[k] + (k == m ? pr * p.inv_eps2 : T(0));
    F[DIM + 1] = v[m] * (E + pr);
  }
  // (dF^m/dw) s with dp = (gamma-1)(s_E - eps^2 v.s_mom + eps^2/2 |v|^2 s_rho)
  __device__ __forceinline__ static void jvp_all(const T* w, const T* s, T (*J)[NV], const DGParams<T>& p) {
    const T ir = T(1) / w[0];
    T v[DIM], v2 = 0, vs = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) { v[k] = w[1 + k] * ir; v2 += v[k] * v[k]; vs += v[k] * s[1 + k]; }
    const T E = w[DIM + 1];
    const T pr = p.gm1 * (E - T(0.5) * p.eps2 * w[0] * v2);
    const T dp = p.gm1 * (s[DIM + 1] - p.eps2 * vs + T(0.5) * p.eps2 * v2 * s[0]);
    const T dpe = dp * p.inv_eps2;
#pragma unroll
    for (int m = 0; m < DIM; ++m) {
      J[m][0] = s[1 + m];
#pragma unroll
      for (int k = 0; k < DIM; ++k)
        J[m][1 + k] = v[m] * s[1 + k] + v[k] * s[1 + m] - v[m] * v[k] * s[0] + (k == m ? dpe : T(0));
      const T dvm = (s[1 + m] - v[m] * s[0]) * ir;
      J[m][DIM + 1] = dvm * (E + pr) + v[m] * (s[DIM + 1] + dp);
    }
  }
  __device__ __forceinline__ static void jvp(const T* w, const T* s, int m, T* J, const DGParams<T>& p) {
    const T ir = T(1) / w[0];
    T v[DIM], v2 = 0, vs = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) { v[k] = w[1 + k] * ir; v2 += v[k] * v[k]; vs += v[k] * s[1 + k]; }
    const T E = w[DIM + 1];
    const T pr = p.gm1 * (E - T(0.5) * p.eps2 * w[0] * v2);
    const T dp = p.gm1 * (s[DIM + 1] - p.eps2 * vs + T(0.5) * p.eps2 * v2 * s[0]);
    J[0] = s[1 + m];
#pragma unroll
    for (int k = 0; k < DIM; ++k)
      J[1 + k] = v[m] * s[1 + k] + v[k] * s[1 + m] - v[m] * v[k] * s[0] + (k == m ? dp * p.inv_eps2 : T(0));
    const T dvm = (s[1 + m] - v[m] * s[0]) * ir;
    J[DIM + 1] = dvm * (E + pr) + v[m] * (s[DIM + 1] + dp);
  }
  __device__ __forceinline__ static T speed(const T* w, int m, const DGParams<T>& p) {
    const T ir = T(1) / w[0];
    T v2 = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) { const T vk = w[1 + k] * ir; v2 += vk * vk; }
    const T pr = p.gm1 * (w[DIM + 1] - T(0.5) * p.eps2 * w[0] * v2);
    return fabs(w[1 + m] * ir) + sqrt(p.gamma * pr * ir) * p.inv_eps;
  }
};

template <int LAW, int DIM, typename T> struct LawOf;
template <int DIM, typename T> struct LawOf<LAW_ADV, DIM, T> { using type = Advection<DIM, T>; };
template <int DIM, typename T> struct LawOf<LAW_BURGERS, DIM, T> { using type = Burgers<DIM, T>; };
template <int DIM, typename T> struct LawOf<LAW_EULER, DIM, T> { using type = Euler<DIM, T>; };

}  // namespace hbpc
