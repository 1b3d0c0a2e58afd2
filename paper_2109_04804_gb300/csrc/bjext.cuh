// BJ_ext block preconditioner (Sec. 3.2.3) on the device.
//
//   J_i = dR1/dW restricted to element i with the neighbours' traces frozen
//   S_i = A_i - B_i C_i = I - c1 J_i + c2 J_i^2        (c1 = a1 dt, c2 = a2 dt^2/2)
//   M_i = S_i^-1
//   P^-1 (w, s) = (D w + E s, F w + G s) with D = M, E = -B M, F = -C M, G = A M,
//   A = I - c1 J, B = c2 J, C = -J; because J commutes with M this is applied as
//     u = M w, v = M s,  top = u - c2 J v,  bottom = J u + v - c1 J v.
//
// BJ^H_ext keeps the Hessian block H_i = dR2/dW|_i in A = I - c1 J + c2 H:
//   M_i = (I - c1 J_i + c2 H_i + c2 J_i^2)^-1,
//   D = M, E = -M B, F = -C M, G = I + C M B, applied as
//     t = w - c2 J s,  u = M t,  top = u,  bottom = J u + s.
//
// Storage: per element an n_b x n_b block, column-major (entry (r, c) at
// c * n_b + r), n_b = n_var (N+1)^dim, so that the threads of one element, one
// per row, read consecutive addresses.
#pragma once
#include "dg_common.cuh"
#include "krylov_common.cuh"

namespace hbpc {

// Assembly of J_i from the structure of Eq. 12: the column of node q, variable
// u has, for every direction m, the volume entries Dvol[m][r_m][q_m] A^m(w_q)
// along the line of q, and the face entries of the lifted numerical flux's
// derivative with respect to the element's own trace (the neighbour is frozen).
// A BR2 viscous term adds nu times its element-diagonal block along the line
// (a constant table, the same for every element).
//
// HESS = true assembles instead the Hessian block H_i = dR2/dW restricted to
// element i at fixed sigma (BJ^H_ext, Sec. 3.2.3): the same routine with the
// physical flux Jacobian A(w) e_u replaced by the flux Hessian H(w)[sigma, e_u]
// (Sec. 3.2.2), evaluated in dual numbers as the derivative of A(w + eps e_u)
// sigma; sigma is the element's own (volume node, or own face trace).  The
// dissipation coefficient is not differentiated and the viscous part of R2 is
// linear in sigma, so neither contributes.  Sg: sigma, same layout as W.
template <int LAW, int DIM, int P, bool LGL, typename T = double, bool HESS = false>
__global__ void __launch_bounds__(128) k_pc_assemble(const double* __restrict__ W, T* __restrict__ Jout,
                                                     const DGParams<T> prm, const double* __restrict__ Sg = nullptr) {
  using L = typename LawOf<LAW, DIM, T>::type;
  using D = Dual<T>;
  constexpr int NV = L::NV, NN = ipow(P, DIM), NB = NV * NN;
  const int e = blockIdx.x;
  if (e >= prm.nE) return;
  T* J = Jout + size_t(e) * NB * NB;
  __shared__ T sw[NB];
  __shared__ T ss[HESS ? NB : 1];
  for (int t = threadIdx.x; t < NB; t += blockDim.x) sw[t] = T(W[size_t(e) * NB + t]);
  if constexpr (HESS)
    for (int t = threadIdx.x; t < NB; t += blockDim.x) ss[t] = T(Sg[size_t(e) * NB + t]);
  for (size_t t = threadIdx.x; t < size_t(NB) * NB; t += blockDim.x) J[t] = T(0);
  __syncthreads();
  // the instance of this element (batches): its mesh and scales; padding
  // elements between instances keep J = 0
  const InstGeo<T> geo = inst_geo(prm, e / Geo<DIM, P>::EPB);
  const int el = e - geo.e0;
  if (el >= geo.nE) return;
  int ec[3];
  ec[0] = el % geo.n[0];
  ec[1] = (el / geo.n[0]) % geo.n[1];
  ec[2] = el / (geo.n[0] * geo.n[1]);
  for (int col = threadIdx.x; col < NB; col += blockDim.x) {
    const int u = col / NN, q = col - u * NN;
    T* Jc = J + size_t(col) * NB;
    int qi[3] = {q % P, (q / P) % P, q / (P * P)};
    T wq[NV], eu[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) { wq[v] = sw[v * NN + q]; eu[v] = (v == u) ? T(1) : T(0); }
#pragma unroll
    for (int m = 0; m < DIM; ++m) {
      const int st = (m == 0) ? 1 : (m == 1 ? P : P * P);
      const int b0 = q - qi[m] * st;
      T a[NV];
      if constexpr (HESS) {
        // H^m(w_q)[sigma_q, e_u]: eps part of A^m(w_q + eps e_u) sigma_q
        if constexpr (L::LINEAR) {
#pragma unroll
          for (int v = 0; v < NV; ++v) a[v] = T(0);
        } else {
          D wd[NV], sd[NV], hd[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) { wd[v] = D(wq[v], eu[v]); sd[v] = D(ss[v * NN + q]); }
          L::jvp(wd, sd, m, hd, prm);
#pragma unroll
          for (int v = 0; v < NV; ++v) a[v] = hd[v].d;
        }
      } else if constexpr (L::LINEAR) {
        // a_m is folded into Dvol unless a viscous term is present
        const T am = prm.visc ? prm.a[m] : T(1);
#pragma unroll
        for (int v = 0; v < NV; ++v) a[v] = am * eu[v];
      } else {
        L::jvp(wq, eu, m, a, prm);
      }
      const T hs = geo.hs[m];
      // volume: output node r = b0 + l*st receives Dvol[m][l][q_m] * a
      for (int l = 0; l < P; ++l)
#pragma unroll
        for (int v = 0; v < NV; ++v) Jc[v * NN + b0 + l * st] += hs * prm.Dvol[m][l][qi[m]] * a[v];
      // BR2 viscous term (scalar laws): its element-diagonal block along the line
      // (a second-derivative operator: two factors 2/h)
      if constexpr (NV == 1 && !HESS) {
        if (prm.visc)
          for (int l = 0; l < P; ++l) Jc[b0 + l * st] += geo.nu * hs * hs * T(prm.vloc[(m * P + l) * P + qi[m]]);
      }
      // faces: own traces at the - and + face of the line through q
      T Ap[NV];
      if constexpr (HESS) {
#pragma unroll
        for (int v = 0; v < NV; ++v) Ap[v] = a[v];   // the node's Hessian term (Lobatto)
      } else {
        L::jvp(wq, eu, m, Ap, prm);   // dF^m/dw at w_q applied to e_u (used for Lobatto)
      }
      for (int side = 0; side < 2; ++side) {
        const T lq = side ? prm.lp[qi[m]] : prm.lm[qi[m]];   // d(own trace)/d(w_q)
        if (lq == T(0)) continue;
        // own trace t_o and neighbour trace t_n at this face point
        T to[NV], tn[NV], so[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) { to[v] = T(0); tn[v] = T(0); so[v] = T(0); }
        int nc[3] = {ec[0], ec[1], ec[2]};
        nc[m] += side ? 1 : -1;
        // a boundary face: the exterior state depends only on the own trace
        const bool bnd = (nc[m] < 0 || nc[m] >= geo.n[m]) && prm.bck[m][side] != BC_PERIODIC;
        const bool wall = bnd && prm.bck[m][side] == BC_WALL;
        if (nc[m] < 0) nc[m] += geo.n[m];
        if (nc[m] >= geo.n[m]) nc[m] -= geo.n[m];
        const int en = geo.e0 + nc[0] + geo.n[0] * (nc[1] + geo.n[1] * nc[2]);
        for (int i = 0; i < P; ++i) {
          const T lo = side ? prm.lp[i] : prm.lm[i];
          const T ln = side ? prm.lm[i] : prm.lp[i];
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            to[v] += lo * sw[v * NN + b0 + i * st];
            if constexpr (HESS) so[v] += lo * ss[v * NN + b0 + i * st];
            else if (!bnd) tn[v] += ln * T(W[(size_t(en) * NV + v) * NN + b0 + i * st]);
          }
        }
        if (bnd) exterior_state<NV>(prm, m, side, to, tn);
        // wall: the exterior trace M t_o (momentum along m reversed) moves with
        // the own trace, d(M t_o)/d(w_q) e_u = lq M e_u, and contributes
        // 1/2 A(M t_o) M e_u (Hessian form: 1/2 H(M t_o)[M s_o, M e_u]) and
        // -kappa M e_u to the derivative of the face flux
        T Aw[NV], meu[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) { Aw[v] = T(0); meu[v] = (v == 1 + m) ? -eu[v] : eu[v]; }
        if constexpr (!L::LINEAR) {
          if (wall) {
            if constexpr (HESS) {
              D td[NV], sd[NV], hd[NV];
#pragma unroll
              for (int v = 0; v < NV; ++v) {
                td[v] = D(tn[v], meu[v]);
                sd[v] = D((v == 1 + m) ? -so[v] : so[v]);
              }
              L::jvp(td, sd, m, hd, prm);
#pragma unroll
              for (int v = 0; v < NV; ++v) Aw[v] = hd[v].d;
            } else {
              L::jvp(tn, meu, m, Aw, prm);
            }
          }
        }
        T A[NV], kap[NV];
        if (LGL) {
#pragma unroll
          for (int v = 0; v < NV; ++v) A[v] = Ap[v];
        } else if constexpr (HESS) {
          if constexpr (L::LINEAR) {
#pragma unroll
            for (int v = 0; v < NV; ++v) A[v] = T(0);
          } else {
            D td[NV], sd[NV], hd[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) { td[v] = D(to[v], eu[v]); sd[v] = D(so[v]); }
            L::jvp(td, sd, m, hd, prm);
#pragma unroll
            for (int v = 0; v < NV; ++v) A[v] = hd[v].d;
          }
        } else {
          L::jvp(to, eu, m, A, prm);
        }
        if (HESS) {
          // sigma's jump does not depend on W and kappa is not differentiated
#pragma unroll
          for (int v = 0; v < NV; ++v) kap[v] = T(0);
        } else if (prm.rusanov) {
          const T c = T(0.5) * fmax(L::speed(to, m, prm), L::speed(tn, m, prm));
#pragma unroll
          for (int v = 0; v < NV; ++v) kap[v] = c;
        } else {
#pragma unroll
          for (int v = 0; v < NV; ++v) kap[v] = prm.lam[m][v];
        }
        // + face: f = 1/2 (F(t_o) + F(t_n)) + kap (t_o - t_n)      -> df/dt_o = A/2 + kap
        // - face: f = -(1/2 (F(t_n) + F(t_o)) + kap (t_n - t_o))  -> df/dt_o = -A/2 + kap
        for (int l = 0; l < P; ++l) {
          const T lift = hs * (side ? prm.sp[m][l] : prm.sm[m][l]);
          if (lift == T(0)) continue;
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            T d = (side ? T(0.5) : T(-0.5)) * A[v] + kap[v] * eu[v];
            if (wall) d += (side ? T(0.5) : T(-0.5)) * Aw[v] - kap[v] * meu[v];
            Jc[v * NN + b0 + l * st] += lift * lq * d;
          }
        }
      }
    }
  }
}

// Apply P^-1 to x = scale * (xW, xS) (element blocks of n_b values), result to
// (oW, oS) (added when accumulate != 0), and the norms of the result's halves
// (unscaled, square-rooted) to zn[0..2] (total, W, S) through the last block.
// EPB elements per block, one thread per row.  S: storage and arithmetic type
// of the blocks and vectors (FP64, or FP32 in the mixed-precision mode).
template <typename S>
struct PcApplyT {
  const S* M; const S* J;
  const S* xW; const S* xS;
  const double* scale;          // device scalar or null (1)
  const int* jidx;              // column index for xW/xS (stride ld), null -> 0
  size_t ld;
  S* oW; S* oS;
  const double* c12;            // device c1, c2
  const int* skip;
  int accumulate;
  double* zn;
  int nb, nE;
  int shared;                   // 1: every element uses block 0 (a state- and
                                // element-independent J_i, see pc_build)
  // shared block only: J_0 as a Kronecker sum of 1-D p x p factors
  // (kron[m][i][l], row-major, direction m), valid when *kron_ok != 0
  const S* kron; const int* kron_ok;
  int P, dim;
  // BJ^H_ext (M = (I - c1 J + c2 H + c2 J^2)^-1): A no longer commutes with B,
  // and P^-1 (w, s) is applied as t = w - c2 J s, u = M t, (u, J u + s)
  int hess;
};
using PcApply = PcApplyT<double>;

}  // namespace hbpc
