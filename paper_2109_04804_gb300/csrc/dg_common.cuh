// Shared definitions of the DGSEM kernels: operator parameters and the
// physical fluxes of the supported conservation laws.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace hbpc {

constexpr int kMaxP = 8;     // nodes per direction (N + 1 <= 8)

constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }


// Forward-mode dual number x + eps dx (eps^2 = 0).  Evaluating the flux
// Jacobian-vector product at the dual state (w + eps t, s + eps u) gives, in the
// eps part, d/deps [A(w + eps t)(s + eps u)] = A(w) u + H(w)[s, t]: the
// directional derivative of R2 used by the analytic (mixed-precision) Jacobian-
// vector product.  Only + - * / are needed by the fluxes' derivatives.
template <typename T>
struct Dual {
  T v, d;
  __host__ __device__ Dual() : v(0), d(0) {}
  __host__ __device__ Dual(T a) : v(a), d(0) {}
  __host__ __device__ Dual(T a, T b) : v(a), d(b) {}
};
template <typename T> __device__ __forceinline__ Dual<T> operator+(Dual<T> a, Dual<T> b) { return {a.v + b.v, a.d + b.d}; }
template <typename T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a, Dual<T> b) { return {a.v - b.v, a.d - b.d}; }
template <typename T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a) { return {-a.v, -a.d}; }
template <typename T> __device__ __forceinline__ Dual<T> operator*(Dual<T> a, Dual<T> b) { return {a.v * b.v, a.v * b.d + a.d * b.v}; }
template <typename T> __device__ __forceinline__ Dual<T> operator*(T a, Dual<T> b) { return {a * b.v, a * b.d}; }
template <typename T> __device__ __forceinline__ Dual<T> operator*(Dual<T> a, T b) { return {a.v * b, a.d * b}; }
template <typename T> __device__ __forceinline__ Dual<T> operator/(Dual<T> a, Dual<T> b) {
  const T iv = T(1) / b.v;
  const T q = a.v * iv;
  return {q, (a.d - q * b.d) * iv};
}
template <typename T> __device__ __forceinline__ Dual<T>& operator+=(Dual<T>& a, Dual<T> b) { a.v += b.v; a.d += b.d; return a; }
template <typename T> __device__ __forceinline__ Dual<T>& operator-=(Dual<T>& a, Dual<T> b) { a.v -= b.v; a.d -= b.d; return a; }

// base (real) type of a value type and its real part
template <class V> struct BaseOf { using type = V; };
template <class T> struct BaseOf<Dual<T>> { using type = T; };
template <class V> __device__ __forceinline__ typename BaseOf<V>::type real_part(const V& x) { return x; }
template <class T> __device__ __forceinline__ T real_part(const Dual<T>& x) { return x.v; }

enum Law { LAW_ADV = 0, LAW_BURGERS = 1, LAW_EULER = 2, LAW_NS = 3,
           LAW_ADV2 = 4 };   // internal: two advected components (both halves of a Krylov vector)

// Operator parameters, passed by value (kernel parameter space).  All matrices
// already carry the Cartesian metric -(2/h_m) of the reference-element
// transformation (Sec. 3.1.1), so the element operator of Eq. 12 is
//   R1_i = sum_m [ sum_l Dvol[m][i][l] G^m_l + sp[m][i] f*_{+m} + sm[m][i] f*_{-m} ]
// with G^m the nodal flux (for advection the state itself, a_m folded in Dvol).
// Launch shape of the element operator kernel: one thread per node, EPB
// elements per block.
template <int DIM, int P>
struct Geo {
  static constexpr int NN = ipow(P, DIM);        // nodes per element
  static constexpr int NF = ipow(P, DIM - 1);    // nodes per face
  static constexpr int EPB = NN >= 256 ? 1 : 256 / NN;
  static constexpr int THREADS = EPB * NN;
};

// Geometry of one instance of a batch of independent problems that share the
// law, the node family and N: one element numbering in which every instance's
// elements are contiguous and start at a multiple of the operator kernel's
// elements per block, so that a block never spans two instances.
template <typename T>
struct InstGeo {
  int n[3];   // elements per direction
  int e0;     // first element of the instance
  int nE;     // elements of the instance
  T hs[3];    // 2 / h_m; the matrices of DGParams are then those of h_m = 2
  T nu;       // viscosity of the instance
};

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
  // BR2 viscous term nu Laplace(w) of a scalar law (Sec. 5.1.1); visc = 0: none.
  // With visc != 0 Dvol does not carry a_m (the advective flux goes through
  // the nodal-flux path like a nonlinear flux).
  int visc;
  T nu;
  T bp[3], bm[3];           // (2/h_m) eta c_+, (2/h_m) eta c_-
  const T* vtab;            // device: Dg[DIM][P][P] = (2/h) D, gp[DIM][P], gm[DIM][P] = (2/h) l_j'(+-1)
  const double* vloc;       // device: element-diagonal viscous block per direction [DIM][P][P], unit nu
  // Navier-Stokes viscous flux (Sec. 5, Eq. 25): dynamic viscosity, heat
  // conductivity lambda = c_p mu / Pr and 1/R = gamma eps^2 (T = p / (rho R))
  T mu, kheat, invR;
  // batch of instances (null for a single problem): per-instance geometry and,
  // per block of the operator kernel, the instance it belongs to
  const InstGeo<T>* inst;
  const int* blk_inst;
  // boundaries of a non-periodic direction m (single problems): bck[m][side]
  // (side 0 = lower, 1 = upper end) is BC_PERIODIC, BC_DIRICHLET (exterior
  // state bcw[m][side], constant in time), BC_WALL (Euler slip wall: the own
  // trace with its momentum along m reversed) or BC_NOSLIP (Navier-Stokes
  // adiabatic no-slip wall: the own trace with its whole momentum reversed)
  int bck[3][2];
  T bcw[3][2][5];
};

enum BoundaryKind { BC_PERIODIC = 0, BC_DIRICHLET = 1, BC_WALL = 2, BC_NOSLIP = 3 };

// The state and the direction the numerical flux sees outside a boundary face
// of direction m (Sec. 3.1.1 with an exterior trace): Dirichlet data are
// constant, so their direction is zero; the wall state is linear in the own
// trace, so its direction is the mirrored own direction.
// p.bck[m][side] and p.bcw[m][side][v] read with constant indices (selects),
// so that a runtime face keeps the parameters out of local memory
template <typename T>
__device__ __forceinline__ int bc_kind(const DGParams<T>& p, int m, int side) {
  int k = side ? p.bck[0][1] : p.bck[0][0];
  if (m == 1) k = side ? p.bck[1][1] : p.bck[1][0];
  if (m == 2) k = side ? p.bck[2][1] : p.bck[2][0];
  return k;
}
template <typename T>
__device__ __forceinline__ T bc_value(const DGParams<T>& p, int m, int side, int v) {
  T x = side ? p.bcw[0][1][v] : p.bcw[0][0][v];
  if (m == 1) x = side ? p.bcw[1][1][v] : p.bcw[1][0][v];
  if (m == 2) x = side ? p.bcw[2][1][v] : p.bcw[2][0][v];
  return x;
}

template <int NV, typename V, typename T>
__device__ __forceinline__ void exterior_state(const DGParams<T>& p, int m, int side, const V* own, V* ext) {
  const int kind = bc_kind(p, m, side);
  if (kind == BC_WALL) {
#pragma unroll
    for (int v = 0; v < NV; ++v) ext[v] = (v == 1 + m) ? -own[v] : own[v];
  } else if (kind == BC_NOSLIP) {
#pragma unroll
    for (int v = 0; v < NV; ++v) ext[v] = (v >= 1 && v < NV - 1) ? -own[v] : own[v];
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) ext[v] = V(bc_value(p, m, side, v));
  }
}
template <int NV, typename V, typename T>
__device__ __forceinline__ void exterior_dir(const DGParams<T>& p, int m, int side, const V* own, V* ext) {
  const int kind = bc_kind(p, m, side);
  if (kind == BC_WALL) {
#pragma unroll
    for (int v = 0; v < NV; ++v) ext[v] = (v == 1 + m) ? -own[v] : own[v];
  } else if (kind == BC_NOSLIP) {
#pragma unroll
    for (int v = 0; v < NV; ++v) ext[v] = (v >= 1 && v < NV - 1) ? -own[v] : own[v];
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) ext[v] = V(T(0));
  }
}

// Geometry of the instance that operator block `blk` works on.
template <typename T>
__device__ __forceinline__ InstGeo<T> inst_geo(const DGParams<T>& p, int blk) {
  if (p.inst) return p.inst[p.blk_inst[blk]];
  InstGeo<T> g;
  g.n[0] = p.n[0]; g.n[1] = p.n[1]; g.n[2] = p.n[2];
  g.e0 = 0; g.nE = p.nE;
  g.hs[0] = T(1); g.hs[1] = T(1); g.hs[2] = T(1);
  g.nu = p.nu;
  return g;
}

// ---------------------------------------------------------------------------
// Physical fluxes, templated on the value type V (double, float or a Dual of
// either; T is the real type of the parameters).  flux_all: F^m(w) for every
// direction m; jvp_all: the directional derivative (dF^m/dw) s; speed: the
// largest |eigenvalue| of dF^m/dw (real values only).
// ---------------------------------------------------------------------------
template <int DIM, typename T>
struct Advection {
  static constexpr int NV = 1;
  static constexpr bool LINEAR = true;
  template <class V>
  __device__ __forceinline__ static void flux_all(const V* w, V (*F)[NV], const DGParams<T>& p) {
#pragma unroll
    for (int m = 0; m < DIM; ++m) F[m][0] = p.a[m] * w[0];
  }
  template <class V>
  __device__ __forceinline__ static void jvp_all(const V* w, const V* s, V (*J)[NV], const DGParams<T>& p) {
#pragma unroll
    for (int m = 0; m < DIM; ++m) J[m][0] = p.a[m] * s[0];
  }
  template <class V>
  __device__ __forceinline__ static void flux(const V* w, int m, V* F, const DGParams<T>& p) {
    F[0] = p.a[m] * w[0];
  }
  template <class V>
  __device__ __forceinline__ static void jvp(const V* w, const V* s, int m, V* J, const DGParams<T>& p) {
    J[0] = p.a[m] * s[0];
  }
  __device__ __forceinline__ static T speed(const T* w, int m, const DGParams<T>& p) {
    return fabs(p.a[m]);
  }
};

// Two independent components advected with the same velocity: the linear
// operator of Eq. 24 applied to both halves (dW, dsigma) of a Krylov vector in
// one element pass instead of two.
template <int DIM, typename T>
struct AdvectionPair {
  static constexpr int NV = 2;
  static constexpr bool LINEAR = true;
  template <class V>
  __device__ __forceinline__ static void flux_all(const V* w, V (*F)[NV], const DGParams<T>& p) {
#pragma unroll
    for (int m = 0; m < DIM; ++m) { F[m][0] = p.a[m] * w[0]; F[m][1] = p.a[m] * w[1]; }
  }
  template <class V>
  __device__ __forceinline__ static void jvp_all(const V* w, const V* s, V (*J)[NV], const DGParams<T>& p) {
#pragma unroll
    for (int m = 0; m < DIM; ++m) { J[m][0] = p.a[m] * s[0]; J[m][1] = p.a[m] * s[1]; }
  }
  template <class V>
  __device__ __forceinline__ static void flux(const V* w, int m, V* F, const DGParams<T>& p) {
    F[0] = p.a[m] * w[0];
    F[1] = p.a[m] * w[1];
  }
  template <class V>
  __device__ __forceinline__ static void jvp(const V* w, const V* s, int m, V* J, const DGParams<T>& p) {
    J[0] = p.a[m] * s[0];
    J[1] = p.a[m] * s[1];
  }
  __device__ __forceinline__ static T speed(const T* w, int m, const DGParams<T>& p) {
    return fabs(p.a[m]);
  }
};

template <int DIM, typename T>
struct Burgers {
  static constexpr int NV = 1;
  static constexpr bool LINEAR = false;
  template <class V>
  __device__ __forceinline__ static void flux_all(const V* w, V (*F)[NV], const DGParams<T>& p) {
    const V f = T(0.5) * (w[0] * w[0]);
#pragma unroll
    for (int m = 0; m < DIM; ++m) F[m][0] = f;
  }
  template <class V>
  __device__ __forceinline__ static void jvp_all(const V* w, const V* s, V (*J)[NV], const DGParams<T>& p) {
    const V f = w[0] * s[0];
#pragma unroll
    for (int m = 0; m < DIM; ++m) J[m][0] = f;
  }
  template <class V>
  __device__ __forceinline__ static void flux(const V* w, int m, V* F, const DGParams<T>& p) {
    F[0] = T(0.5) * (w[0] * w[0]);
  }
  template <class V>
  __device__ __forceinline__ static void jvp(const V* w, const V* s, int m, V* J, const DGParams<T>& p) {
    J[0] = w[0] * s[0];
  }
  __device__ __forceinline__ static T speed(const T* w, int m, const DGParams<T>& p) {
    return fabs(w[0]);
  }
};

// a[m] of a short register array for a runtime m (selects over unrolled
// indices, so the array stays in registers; a constant m folds)
template <int K, class V>
__device__ __forceinline__ V pick(const V* a, int m) {
  V r = a[0];
#pragma unroll
  for (int k = 1; k < K; ++k)
    if (k == m) r = a[k];
  return r;
}

// Euler with reference Mach number eps (Eq. 21):
//   F^m = (rho v_m, rho v_m v + p/eps^2 e_m, v_m (E + p)),
//   p = (gamma - 1)(E - eps^2/2 rho |v|^2),  c = sqrt(gamma p / rho) / eps.
template <int DIM, typename T>
struct Euler {
  static constexpr int NV = DIM + 2;
  static constexpr bool LINEAR = false;
  template <class V>
  __device__ __forceinline__ static void flux_all(const V* w, V (*F)[NV], const DGParams<T>& p) {
    const V ir = V(T(1)) / w[0];
    V v[DIM], v2 = V(T(0));
#pragma unroll
    for (int k = 0; k < DIM; ++k) { v[k] = w[1 + k] * ir; v2 += v[k] * v[k]; }
    const V E = w[DIM + 1];
    const V pr = p.gm1 * (E - (T(0.5) * p.eps2) * (w[0] * v2));
    const V pe = pr * p.inv_eps2;
#pragma unroll
    for (int m = 0; m < DIM; ++m) {
      F[m][0] = w[1 + m];
#pragma unroll
      for (int k = 0; k < DIM; ++k) F[m][1 + k] = (k == m) ? w[1 + m] * v[k] + pe : w[1 + m] * v[k];
      F[m][DIM + 1] = v[m] * (E + pr);
    }
  }
  template <class V>
  __device__ __forceinline__ static void flux(const V* w, int m, V* F, const DGParams<T>& p) {
    const V ir = V(T(1)) / w[0];
    V v[DIM], v2 = V(T(0));
#pragma unroll
    for (int k = 0; k < DIM; ++k) { v[k] = w[1 + k] * ir; v2 += v[k] * v[k]; }
    const V E = w[DIM + 1];
    const V pr = p.gm1 * (E - (T(0.5) * p.eps2) * (w[0] * v2));
    const V wm = pick<DIM>(w + 1, m), vm = pick<DIM>(v, m);
    F[0] = wm;
#pragma unroll
    for (int k = 0; k < DIM; ++k) F[1 + k] = (k == m) ? wm * v[k] + pr * p.inv_eps2 : wm * v[k];
    F[DIM + 1] = vm * (E + pr);
  }
  // (dF^m/dw) s with dp = (gamma-1)(s_E - eps^2 v.s_mom + eps^2/2 |v|^2 s_rho)
  template <class V>
  __device__ __forceinline__ static void jvp_all(const V* w, const V* s, V (*J)[NV], const DGParams<T>& p) {
    const V ir = V(T(1)) / w[0];
    V v[DIM], v2 = V(T(0)), vs = V(T(0));
#pragma unroll
    for (int k = 0; k < DIM; ++k) { v[k] = w[1 + k] * ir; v2 += v[k] * v[k]; vs += v[k] * s[1 + k]; }
    const V E = w[DIM + 1];
    const V pr = p.gm1 * (E - (T(0.5) * p.eps2) * (w[0] * v2));
    const V dp = p.gm1 * (s[DIM + 1] - p.eps2 * vs + (T(0.5) * p.eps2) * (v2 * s[0]));
    const V dpe = dp * p.inv_eps2;
#pragma unroll
    for (int m = 0; m < DIM; ++m) {
      J[m][0] = s[1 + m];
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        const V t = v[m] * s[1 + k] + v[k] * s[1 + m] - v[m] * (v[k] * s[0]);
        J[m][1 + k] = (k == m) ? t + dpe : t;
      }
      const V dvm = (s[1 + m] - v[m] * s[0]) * ir;
      J[m][DIM + 1] = dvm * (E + pr) + v[m] * (s[DIM + 1] + dp);
    }
  }
  template <class V>
  __device__ __forceinline__ static void jvp(const V* w, const V* s, int m, V* J, const DGParams<T>& p) {
    const V ir = V(T(1)) / w[0];
    V v[DIM], v2 = V(T(0)), vs = V(T(0));
#pragma unroll
    for (int k = 0; k < DIM; ++k) { v[k] = w[1 + k] * ir; v2 += v[k] * v[k]; vs += v[k] * s[1 + k]; }
    const V E = w[DIM + 1];
    const V pr = p.gm1 * (E - (T(0.5) * p.eps2) * (w[0] * v2));
    const V dp = p.gm1 * (s[DIM + 1] - p.eps2 * vs + (T(0.5) * p.eps2) * (v2 * s[0]));
    const V sm = pick<DIM>(s + 1, m), vm = pick<DIM>(v, m);
    J[0] = sm;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      const V t = vm * s[1 + k] + v[k] * sm - vm * (v[k] * s[0]);
      J[1 + k] = (k == m) ? t + dp * p.inv_eps2 : t;
    }
    const V dvm = (sm - vm * s[0]) * ir;
    J[DIM + 1] = dvm * (E + pr) + vm * (s[DIM + 1] + dp);
  }
  __device__ __forceinline__ static T speed(const T* w, int m, const DGParams<T>& p) {
    const T ir = T(1) / w[0];
    T v2 = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) { const T vk = w[1 + k] * ir; v2 += vk * vk; }
    const T pr = p.gm1 * (w[DIM + 1] - T(0.5) * p.eps2 * w[0] * v2);
    return fabs(pick<DIM>(w + 1, m) * ir) + sqrt(p.gamma * pr * ir) * p.inv_eps;
  }
};

// Navier-Stokes viscous flux (Sec. 5, Eq. 25) as a function of the gradient
// variables g = (v_1..v_d, T) of Eq. 26 and their gradient d[k][c] (derivative
// of channel c along x_k):
//   F^v_m = (0, tau_{k m}, sum_k tau_{m k} v_k + lambda dT/dx_m),
//   tau = mu (grad v + grad v^T - 2/3 div v I).
// tau depends on d only, so the linearisation (Eq. 32) in the direction
// (gs, ds) is (0, tau(ds)_{k m}, sum_k [tau(ds)_{m k} v_k + tau(d)_{m k} gs_k] + lambda ds[m][T]).
template <int DIM, typename T>
struct NSVisc {
  static constexpr int NG = DIM + 1;
  static constexpr int NV = DIM + 2;
  // g = (m / rho, p / (rho R))
  template <class V>
  __device__ __forceinline__ static void grad_vars(const V* w, V* g, const DGParams<T>& p) {
    const V ir = V(T(1)) / w[0];
    V v2 = V(T(0));
#pragma unroll
    for (int k = 0; k < DIM; ++k) { g[k] = w[1 + k] * ir; v2 += g[k] * g[k]; }
    const V pr = p.gm1 * (w[DIM + 1] - (T(0.5) * p.eps2) * (w[0] * v2));
    g[DIM] = (pr * ir) * p.invR;
  }
  // (dg/dw) s (the matrix of Eq. 31 applied to sigma)
  template <class V>
  __device__ __forceinline__ static void grad_vars_jvp(const V* w, const V* s, V* gs, const DGParams<T>& p) {
    const V ir = V(T(1)) / w[0];
    V v[DIM], v2 = V(T(0)), vs = V(T(0));
#pragma unroll
    for (int k = 0; k < DIM; ++k) { v[k] = w[1 + k] * ir; v2 += v[k] * v[k]; vs += v[k] * s[1 + k]; }
    const V pr = p.gm1 * (w[DIM + 1] - (T(0.5) * p.eps2) * (w[0] * v2));
    const V dp = p.gm1 * (s[DIM + 1] - p.eps2 * vs + (T(0.5) * p.eps2) * (v2 * s[0]));
#pragma unroll
    for (int k = 0; k < DIM; ++k) gs[k] = (s[1 + k] - v[k] * s[0]) * ir;
    gs[DIM] = ((dp - (pr * ir) * s[0]) * ir) * p.invR;
  }
  template <class V>
  __device__ __forceinline__ static V tau(const V (*d)[NG], int i, int j, T mu) {
    V t = d[i][j] + d[j][i];
    if (i == j) {
      V dv = V(T(0));
#pragma unroll
      for (int k = 0; k < DIM; ++k) dv += d[k][k];
      t -= T(2.0 / 3.0) * dv;
    }
    return mu * t;
  }
  // F^v along x_m; F[0] (mass) is zero and is not written
  template <class V>
  __device__ __forceinline__ static void flux(const V* g, const V (*d)[NG], int m, V* F, const DGParams<T>& p) {
    V e = p.kheat * d[m][DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      const V t = tau(d, k, m, p.mu);
      F[1 + k] = t;
      e += t * g[k];
    }
    F[DIM + 1] = e;
  }
  template <class V>
  __device__ __forceinline__ static void flux_lin(const V* g, const V (*d)[NG], const V* gs, const V (*ds)[NG], int m,
                                                  V* F, const DGParams<T>& p) {
    V e = p.kheat * ds[m][DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      const V ts = tau(ds, k, m, p.mu);
      F[1 + k] = ts;
      e += ts * g[k] + tau(d, m, k, p.mu) * gs[k];
    }
    F[DIM + 1] = e;
  }
};

template <int LAW, int DIM, typename T> struct LawOf;
template <int DIM, typename T> struct LawOf<LAW_ADV, DIM, T> { using type = Advection<DIM, T>; };
template <int DIM, typename T> struct LawOf<LAW_BURGERS, DIM, T> { using type = Burgers<DIM, T>; };
template <int DIM, typename T> struct LawOf<LAW_EULER, DIM, T> { using type = Euler<DIM, T>; };
// Navier-Stokes: the Euler flux; the viscous part is added by the operator kernel
template <int DIM, typename T> struct LawOf<LAW_NS, DIM, T> { using type = Euler<DIM, T>; };
template <int DIM, typename T> struct LawOf<LAW_ADV2, DIM, T> { using type = AdvectionPair<DIM, T>; };

}  // namespace hbpc
