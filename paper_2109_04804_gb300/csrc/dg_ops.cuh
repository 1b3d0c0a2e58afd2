// Element-batched DGSEM operator kernel (Eq. 12 for R1, Eq. 16 for R2).
//
// One thread per volume node; EPB elements per block.  Per operator evaluation:
//   1. every node loads its state (and direction for R2), evaluates the nodal
//      flux F^m(w) (R1) or (dF^m/dw) s (R2) for all directions and stores it in
//      shared memory;
//   2. the element's 2*DIM*P^(DIM-1) face points compute the numerical flux of
//      Eq. 13 (R1) or the flux f~* of Sec. 3.1.2 (R2) from the element's own
//      trace (shared memory) and the neighbour's trace (global memory, L2) and
//      store it in shared memory -- each face is evaluated by both of its
//      elements, which keeps the pass free of any grid-wide dependency;
//   3. every node contracts the fluxes with Dvol along each direction and adds
//      the lifted face fluxes.
// With a BR2 viscous term (scalar laws, Sec. 5.1.1) pass 2 also forms, per face
// point, the common value u* and the average of the two face-local lifted
// gradients (the neighbour's line is read in full for its derivative at the
// face); a pass 2b then forms the lifted gradient d at every node and folds
// -nu d into the nodal flux, and the viscous face flux into the face flux, so
// pass 3 is unchanged.  The Navier-Stokes law (Sec. 5) does the same for the
// d + 1 gradient variables (v, T): pass 1 converts the nodes to them, pass 2
// stores the face traces of both sides (stage A), and after the barrier the
// face-local gradients (with tangential components from the stored traces) give
// the central viscous face flux (stage B) while every node forms its lifted
// gradient and F^v (Eq. 25), or their linearisations for R2 (Eq. 31-33).
// A Job supplies how node values are loaded (so that perturbed states W + eps dW
// are formed on the fly) and what is done with the results (the epilogue), so
// Jacobian-vector products and residuals are single passes over memory.
#pragma once
#include <type_traits>

#include "dg_common.cuh"

namespace hbpc {

enum EvalKind { EV_R1 = 0, EV_R2 = 1 };

// A job with kFrozenNb = true evaluates R2 with the neighbours' direction taken
// as zero (the element-diagonal block of the preconditioner, Sec. 3.2.3); every
// load of a neighbour's direction goes through load_nb_dir.
template <class Job, class = void> struct FrozenNb { static constexpr bool value = false; };
template <class Job> struct FrozenNb<Job, std::void_t<decltype(Job::kFrozenNb)>> {
  static constexpr bool value = Job::kFrozenNb;
};
// A job with kDirectionState = true loads directions where the operator
// expects states (the linear Jv of Eq. 24 applies R1 to Krylov vectors): a
// boundary's exterior is then the exterior direction, not the exterior state.
template <class Job, class = void> struct DirectionState { static constexpr bool value = false; };
template <class Job> struct DirectionState<Job, std::void_t<decltype(Job::kDirectionState)>> {
  static constexpr bool value = Job::kDirectionState;
};

template <int NV, class Job, typename V>
__device__ __forceinline__ void load_nb_dir(const Job& job, int k, int en, int node, V* x) {
  if constexpr (FrozenNb<Job>::value) {
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] = V(0);
  } else {
    job.load_dir(k, en, node, x);
  }
}


template <int LAW, int DIM, int P>
struct KernelShape {
  static constexpr int NV = (LAW == LAW_EULER || LAW == LAW_NS) ? DIM + 2 : (LAW == LAW_ADV2 ? 2 : 1);
  static constexpr bool NSV = LAW == LAW_NS;     // Navier-Stokes viscous flux (system BR2)
  static constexpr bool VISC = NV == 1 || NSV;   // BR2 viscous term available
  static constexpr int NN = Geo<DIM, P>::NN, NF = Geo<DIM, P>::NF, EPB = Geo<DIM, P>::EPB;
  // gradient channels of the system path: g = (v, T) and, for R2, gs = (dg/dw) s
  static constexpr int NCH = NSV ? 2 * (DIM + 1) : 0;
  // resident blocks per SM the register allocation must allow (shared memory
  // admits two blocks of the 3-D Navier-Stokes kernel)
  static constexpr int MIN_BLOCKS = (NSV && DIM == 3) ? 2 : 1;
  // shared values per element: state + direction + DIM fluxes + 2*DIM faces
  // (+ 2*DIM faces of u* - u for the scalar viscous term; + the nodal channels
  // and, per face, the own trace, the neighbour's trace and the neighbour's
  // normal derivative of every channel for the system)
  static constexpr int PER_ELEM = 2 * NV * NN + DIM * NV * NN + 2 * DIM * NV * NF + (NV == 1 ? 2 * DIM * NF : 0) +
                                  (NSV ? NCH * NN + 3 * 2 * DIM * NCH * NF : 0);
  // Dvol, sp, sm (+ Dg, gp, gm)
  static constexpr int MATS = DIM * P * P + 2 * DIM * P + (VISC ? DIM * P * P + 2 * DIM * P : 0);
  // operator matrices (base type B, padded to 16 bytes) then element data (V)
  template <typename V, typename B>
  static constexpr size_t mats_bytes() { return ((MATS * sizeof(B) + 15) / 16) * 16; }
  template <typename V, typename B = V>
  static constexpr size_t smem_bytes() { return mats_bytes<V, B>() + size_t(EPB) * PER_ELEM * sizeof(V); }
};

// Numerical flux at one face point of direction M and side SIDE (0: -, 1: +)
// of the thread's element: Eq. 13 for R1, the flux f~* of Sec. 3.1.2 for R2.
// Direction and side are compile-time so that every array stays in registers.
template <int LAW, int DIM, int P, bool LGL, typename V, class Job>
struct FaceFlux {
  using T = typename BaseOf<V>::type;
  using L = typename LawOf<LAW, DIM, T>::type;
  static constexpr int NV = L::NV, NN = Geo<DIM, P>::NN, NF = Geo<DIM, P>::NF;
  // Face M (direction) / SIDE of the element: compile-time constants where
  // the caller dispatches on the face (one inlined copy per face), runtime
  // values where one copy serves every face (the large Navier-Stokes kernels,
  // whose instruction footprint otherwise stalls issue).
  template <int M, int SIDE>
  __device__ __forceinline__ static void run(const Job& job, const DGParams<T>& prm, const InstGeo<T>& g,
                                             int k, bool r2, const int* ec, int pt, const V* sst,
                                             const V* sdir, V* sface) {
    run_face(M, SIDE, job, prm, g, k, r2, ec, pt, sst, sdir, sface);
  }
  __device__ __forceinline__ static void run_face(const int M, const int SIDE, const Job& job,
                                                  const DGParams<T>& prm, const InstGeo<T>& g, int k, bool r2,
                                                  const int* ec, int pt, const V* sst, const V* sdir, V* sface) {
    const int st = (M == 0) ? 1 : (M == 1 ? P : P * P);
    const int base = (pt % st) + (pt / st) * st * P;   // face point -> node with idx_M = 0
    // neighbour element across this face (periodic within the instance), or
    // a boundary face of a non-periodic direction
    const int gnM = M == 0 ? g.n[0] : (M == 1 ? g.n[1] : g.n[2]);
    int c = M == 0 ? ec[0] : (M == 1 ? ec[1] : ec[2]);
    c += SIDE ? 1 : -1;
    const bool bnd = (c < 0 || c >= gnM) && bc_kind(prm, M, SIDE) != BC_PERIODIC;
    if (c < 0) c += gnM;
    if (c >= gnM) c -= gnM;
    const int nc0 = M == 0 ? c : ec[0], nc1 = M == 1 ? c : ec[1], nc2 = M == 2 ? c : ec[2];
    const int en = g.e0 + nc0 + g.n[0] * (nc1 + g.n[1] * nc2);
    V wo[NV], wn[NV], so[NV], sn[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) { wo[v] = V(T(0)); wn[v] = V(T(0)); so[v] = V(T(0)); sn[v] = V(T(0)); }
    if constexpr (LGL) {
      const int own_node = base + (SIDE ? (P - 1) * st : 0);
      const int nb_node = base + (SIDE ? 0 : (P - 1) * st);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        wo[v] = sst[v * NN + own_node];
        if (r2) so[v] = sdir[v * NN + own_node];
      }
      if (!bnd) {
        job.load_state(k, en, nb_node, wn);
        if (r2) load_nb_dir<NV>(job, k, en, nb_node, sn);
      }
    } else {
#pragma unroll
      for (int i = 0; i < P; ++i) {
        const int node = base + i * st;
        const T lo = SIDE ? prm.lp[i] : prm.lm[i];   // own trace at this face
        const T ln = SIDE ? prm.lm[i] : prm.lp[i];   // neighbour's trace at this face
        V tw[NV], ts[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) { tw[v] = V(T(0)); ts[v] = V(T(0)); }
        if (!bnd) {
          job.load_state(k, en, node, tw);
          if (r2) load_nb_dir<NV>(job, k, en, node, ts);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          wo[v] += lo * sst[v * NN + node];
          wn[v] += ln * tw[v];
          if (r2) { so[v] += lo * sdir[v * NN + node]; sn[v] += ln * ts[v]; }
        }
      }
    }
    if (bnd) {
      // exterior of the boundary face from the element's own traces
      if constexpr (DirectionState<Job>::value) exterior_dir<NV>(prm, M, SIDE, wo, wn);
      else exterior_state<NV>(prm, M, SIDE, wo, wn);
      if (r2) exterior_dir<NV>(prm, M, SIDE, so, sn);
    }
    // (L, R) = (own, neighbour) on the + face, (neighbour, own) on the - face
    V wL[NV], wR[NV], sL[NV], sR[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      wL[v] = SIDE ? wo[v] : wn[v];
      wR[v] = SIDE ? wn[v] : wo[v];
      sL[v] = SIDE ? so[v] : sn[v];
      sR[v] = SIDE ? sn[v] : so[v];
    }
    V FL[NV], FR[NV];
    T kap[NV];
    if (prm.rusanov) {
      // dissipation from the real parts of the traces: frozen in derivatives
      T wLr[NV], wRr[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) { wLr[v] = real_part(wL[v]); wRr[v] = real_part(wR[v]); }
      const T cmax = T(0.5) * fmax(L::speed(wLr, M, prm), L::speed(wRr, M, prm));
#pragma unroll
      for (int v = 0; v < NV; ++v) kap[v] = cmax;
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) kap[v] = M == 0 ? prm.lam[0][v] : (M == 1 ? prm.lam[1][v] : prm.lam[2][v]);
    }
    if (r2) { L::jvp(wL, sL, M, FL, prm); L::jvp(wR, sR, M, FR, prm); }
    else { L::flux(wL, M, FL, prm); L::flux(wR, M, FR, prm); }
    const T sgn = SIDE ? T(1) : T(-1);     // outward normal of the element
    const int f = 2 * M + SIDE;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const V jump = r2 ? (sL[v] - sR[v]) : (wL[v] - wR[v]);
      sface[(f * NV + v) * NF + pt] = sgn * (T(0.5) * (FL[v] + FR[v]) + kap[v] * jump);
    }
  }
};

// BR2 viscous part at one face point (scalar law): the common value
// u* = (u_own + u_nb)/2 (Eq. 30) and the face-local lifted gradients
//   element left of the face:  d^L = u'(+1) + eta c_+ (u* - u^L(+1)),
//   element right of the face: d^R = u'(-1) + eta c_- (u^R(-1) - u*)   (times 2/h),
// (strong-form liftings keeping only this face's surface term, scaled by eta).
// The viscous face flux nu (d^L + d^R)/2 along +e_M enters sface with the sign
// that makes pass 3 add +(2/h)[lhat(+1) F^v*_+ - lhat(-1) F^v*_-]; u* - u_own is
// kept for the lifted volume gradient of pass 2b.  u: the element's values of
// the viscous input (state for R1, direction for R2) in shared memory.
template <int DIM, int P, typename V, class Job>
struct FaceVisc {
  using T = typename BaseOf<V>::type;
  static constexpr int NF = Geo<DIM, P>::NF;
  template <int M, int SIDE>
  __device__ __forceinline__ static void run(const Job& job, const DGParams<T>& prm, const InstGeo<T>& g,
                                             int k, bool r2, const int* ec, int pt, const V* u,
                                             const T* sgp, const T* sgm, V* sface, V* sjump) {
    constexpr int st = (M == 0) ? 1 : (M == 1 ? P : P * P);
    const int base = (pt % st) + (pt / st) * st * P;
    int nc0 = ec[0], nc1 = ec[1], nc2 = ec[2];
    int& c = (M == 0) ? nc0 : (M == 1 ? nc1 : nc2);
    c += SIDE ? 1 : -1;
    if (c < 0) c += g.n[M];
    if (c >= g.n[M]) c -= g.n[M];
    const int en = g.e0 + nc0 + g.n[0] * (nc1 + g.n[1] * nc2);
    V uo = V(T(0)), go = V(T(0)), un = V(T(0)), gn = V(T(0));
#pragma unroll
    for (int i = 0; i < P; ++i) {
      const int node = base + i * st;
      V y[1];
      if (r2) load_nb_dir<1>(job, k, en, node, y); else job.load_state(k, en, node, y);
      const V x = u[node];
      uo += (SIDE ? prm.lp[i] : prm.lm[i]) * x;
      go += (SIDE ? sgp[M * P + i] : sgm[M * P + i]) * x;
      un += (SIDE ? prm.lm[i] : prm.lp[i]) * y[0];
      gn += (SIDE ? sgm[M * P + i] : sgp[M * P + i]) * y[0];
    }
    const V us = T(0.5) * (uo + un);
    V dL, dR;
    if (SIDE) {
      dL = go + prm.bp[M] * (us - uo);
      dR = gn + prm.bm[M] * (un - us);
    } else {
      dL = gn + prm.bp[M] * (us - un);
      dR = go + prm.bm[M] * (uo - us);
    }
    const int f = 2 * M + SIDE;
    const T sg = SIDE ? T(-0.5) : T(0.5);
    sface[f * NF + pt] += (sg * g.nu * g.hs[M]) * (dL + dR);
    sjump[f * NF + pt] = us - uo;
  }
};

// Navier-Stokes BR2 (Sec. 5.1.1-5.1.2), stage A at one face point: the own
// trace of every gradient channel (from the element's nodal channels in shared
// memory) and the neighbour's trace and normal derivative (its line of nodes
// through this face point is read from global memory and converted to g, and
// for R2 to gs = (dg/dw) s).  Stored per face for stage B, which needs the
// traces of neighbouring face points for the tangential derivatives.
// Channel layout: [0, NG) g, [NG, 2 NG) gs (R2 only).  The face direction M and
// side are runtime values (one copy of the code for all 2 DIM faces keeps the
// kernel inside the instruction cache); register arrays are indexed only by
// unrolled loop counters.
template <int DIM, int P, typename V, class Job>
struct FaceViscSysA {
  using T = typename BaseOf<V>::type;
  using NS = NSVisc<DIM, T>;
  static constexpr int NV = DIM + 2, NG = DIM + 1, NCH = 2 * NG;
  static constexpr int NN = Geo<DIM, P>::NN, NF = Geo<DIM, P>::NF;
  __device__ __forceinline__ static void run(const Job& job, const DGParams<T>& prm, const InstGeo<T>& g, int k,
                                             bool r2, const int* ec, int f, int pt, const V* sgc, const T* sgp,
                                             const T* sgm, V* sfo, V* sfn, V* sfd) {
    const int M = f >> 1, side = f & 1;
    const int st = (M == 0) ? 1 : (M == 1 ? P : P * P);
    const int base = (pt % st) + (pt / st) * st * P;
    const int nch = r2 ? NCH : NG;
    // a boundary face: the exterior channels from the own ones (adiabatic
    // no-slip wall: the velocity reversed, T kept, the own normal derivative
    // with dT/dn reversed; Dirichlet: the state's channels, zero for the
    // linearised ones, the own normal derivative); the exterior's tangential
    // derivatives are the own ones (stage B)
    {
      const int ecM = M == 0 ? ec[0] : (M == 1 ? ec[1] : ec[2]);
      const int gnM = M == 0 ? g.n[0] : (M == 1 ? g.n[1] : g.n[2]);
      const int kind = bc_kind(prm, M, side);
      if (kind != BC_PERIODIC && (side ? ecM == gnM - 1 : ecM == 0)) {
        V gbc[NG];
        if (kind == BC_DIRICHLET) {
          V sb[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) sb[v] = V(bc_value(prm, M, side, v));
          NS::grad_vars(sb, gbc, prm);
        }
        const T* gown = (side ? sgp : sgm) + M * P;   // shared-memory table
#pragma unroll
        for (int q = 0; q < NCH; ++q) {
          if (q >= nch) continue;
          const int cq = q % NG;
          V uo = V(T(0)), go = V(T(0));
#pragma unroll
          for (int i = 0; i < P; ++i) {
            uo += (side ? prm.lp[i] : prm.lm[i]) * sgc[q * NN + base + i * st];
            go += gown[i] * sgc[q * NN + base + i * st];
          }
          V ux, gx;
          if (kind == BC_DIRICHLET) {
            ux = q < NG ? gbc[cq] : V(T(0));
            gx = go;
          } else {
            ux = cq < DIM ? -uo : uo;
            gx = cq == DIM ? -go : go;
          }
          sfo[(f * NCH + q) * NF + pt] = uo;
          sfn[(f * NCH + q) * NF + pt] = ux;
          sfd[(f * NCH + q) * NF + pt] = gx;
        }
        return;
      }
    }
    // neighbour element across this face (periodic within the instance)
    const int dlt = side ? 1 : -1;
    int nc0 = ec[0] + (M == 0 ? dlt : 0), nc1 = ec[1] + (M == 1 ? dlt : 0), nc2 = ec[2] + (M == 2 ? dlt : 0);
    nc0 = nc0 < 0 ? nc0 + g.n[0] : (nc0 >= g.n[0] ? nc0 - g.n[0] : nc0);
    nc1 = nc1 < 0 ? nc1 + g.n[1] : (nc1 >= g.n[1] ? nc1 - g.n[1] : nc1);
    nc2 = nc2 < 0 ? nc2 + g.n[2] : (nc2 >= g.n[2] ? nc2 - g.n[2] : nc2);
    const int en = g.e0 + nc0 + g.n[0] * (nc1 + g.n[1] * nc2);
    const T* dnb = (side ? sgm : sgp) + M * P;             // neighbour's normal-derivative weights
    V un[NCH], gn[NCH];
#pragma unroll
    for (int q = 0; q < NCH; ++q) { un[q] = V(T(0)); gn[q] = V(T(0)); }
#pragma unroll
    for (int i = 0; i < P; ++i) {
      const int node = base + i * st;
      V x[NV], ch[NCH];
      job.load_state(k, en, node, x);
      NS::grad_vars(x, ch, prm);
      if (r2) {
        V y[NV];
        load_nb_dir<NV>(job, k, en, node, y);
        NS::grad_vars_jvp(x, y, ch + NG, prm);
      }
      // the neighbour's trace weights at this face (parameters read by value:
      // no pointer into the parameter space)
      const T ln = side ? prm.lm[i] : prm.lp[i], dn = dnb[i];
#pragma unroll
      for (int q = 0; q < NCH; ++q)
        if (q < nch) { un[q] += ln * ch[q]; gn[q] += dn * ch[q]; }
    }
#pragma unroll
    for (int q = 0; q < NCH; ++q) {
      if (q < nch) {
        V uo = V(T(0));
#pragma unroll
        for (int i = 0; i < P; ++i) uo += (side ? prm.lp[i] : prm.lm[i]) * sgc[q * NN + base + i * st];
        sfo[(f * NCH + q) * NF + pt] = uo;
        sfn[(f * NCH + q) * NF + pt] = un[q];
        sfd[(f * NCH + q) * NF + pt] = gn[q];
      }
    }
  }
};

// Stage B at one face point: the face-local BR2 gradients of both sides, all
// directions -- the normal component from the normal derivative plus eta times
// the face's own lifting, the tangential ones from the traces of the face
// points along that direction -- and the central viscous flux of Eq. 30 (R1)
// or its linearisation (R2, Eq. 32), added to sface with the sign convention
// of the inviscid flux (outward normal).  Runtime face as in stage A.
template <int DIM, int P, typename V>
struct FaceViscSysB {
  using T = typename BaseOf<V>::type;
  using NS = NSVisc<DIM, T>;
  static constexpr int NV = DIM + 2, NG = DIM + 1, NCH = 2 * NG;
  static constexpr int NN = Geo<DIM, P>::NN, NF = Geo<DIM, P>::NF;
  // bnd: a boundary face, whose exterior side takes the own tangential
  // derivatives (stage A's exterior gradient)
  __device__ __forceinline__ static void run(const DGParams<T>& prm, const InstGeo<T>& g, bool r2, int f, int pt,
                                             const V* sgc, const T* sDg, const T* sgp, const T* sgm, const V* sfo,
                                             const V* sfn, const V* sfd, V* sface, bool bnd) {
    const int M = f >> 1, side = f & 1;
    const int st = (M == 0) ? 1 : (M == 1 ? P : P * P);
    const int base = (pt % st) + (pt / st) * st * P;
    const int nch = r2 ? NCH : NG;
    const T* gown = (side ? sgp : sgm) + M * P;            // own normal-derivative weights
    // lower tangential direction is fastest in the face numbering
    // (pt = j + P k on x faces, i + P k on y faces, i + P j on z faces)
    const int lo_t = (M == 0) ? 1 : 0;
    // gradients of the own (o) and neighbour (n) side: [channel set][direction][channel]
    V dO[2][DIM][NG], dN[2][DIM][NG], gO[NCH], gN[NCH];
#pragma unroll
    for (int q = 0; q < NCH; ++q) {
      const int set = q / NG, cq = q - set * NG;
      if (q >= nch) {
        gO[q] = V(T(0)); gN[q] = V(T(0));
#pragma unroll
        for (int kk = 0; kk < DIM; ++kk) { dO[set][kk][cq] = V(T(0)); dN[set][kk][cq] = V(T(0)); }
        continue;
      }
      const V* fo = sfo + (f * NCH + q) * NF;
      const V* fn = sfn + (f * NCH + q) * NF;
      const V uo = fo[pt], un = fn[pt];
      gO[q] = uo; gN[q] = un;
#pragma unroll
      for (int kk = 0; kk < DIM; ++kk) {
        if (kk == M) {
          // normal component: + face (own = L): d^L = go + bp (u* - uo), d^R = gn + bm (un - u*);
          //                   - face (own = R): d^L = gn + bp (u* - un), d^R = go + bm (uo - u*)
          V go = V(T(0));
#pragma unroll
          for (int i = 0; i < P; ++i) go += gown[i] * sgc[q * NN + base + i * st];
          const V gn = sfd[(f * NCH + q) * NF + pt];
          const V us = T(0.5) * (uo + un);
          const V lo_ = side ? prm.bp[kk] * (us - uo) : prm.bm[kk] * (uo - us);
          const V ln_ = side ? prm.bm[kk] * (un - us) : prm.bp[kk] * (us - un);
          dO[set][kk][cq] = g.hs[kk] * (go + lo_);
          dN[set][kk][cq] = g.hs[kk] * (gn + ln_);
        } else {
          // tangential component: derivative of the face traces along x_kk
          const int tstride = (kk == lo_t) ? 1 : P;
          const int it = (pt / tstride) % P;
          const int p0 = pt - it * tstride;
          const T* Drow = sDg + (kk * P + it) * P;
          V a = V(T(0)), b = V(T(0));
#pragma unroll
          for (int j = 0; j < P; ++j) {
            a += Drow[j] * fo[p0 + j * tstride];
            b += Drow[j] * fn[p0 + j * tstride];
          }
          dO[set][kk][cq] = g.hs[kk] * a;
          dN[set][kk][cq] = g.hs[kk] * (bnd ? a : b);
        }
      }
    }
    // flux along x_M: the direction is expanded over the unrolled m so that the
    // register arrays keep compile-time indices
    V FO[NV], FN[NV];
#pragma unroll
    for (int m = 0; m < DIM; ++m) {
      if (m != M) continue;
      if (r2) {
        NS::flux_lin(gO, dO[0], gO + NG, dO[1], m, FO, prm);
        NS::flux_lin(gN, dN[0], gN + NG, dN[1], m, FN, prm);
      } else {
        NS::flux(gO, dO[0], m, FO, prm);
        NS::flux(gN, dN[0], m, FN, prm);
      }
    }
    const T sg = side ? T(-0.5) : T(0.5);
#pragma unroll
    for (int v = 1; v < NV; ++v) sface[(f * NV + v) * NF + pt] += sg * (FO[v] + FN[v]);
  }
};

template <int LAW, int DIM, int P, bool LGL, typename V, class Job>
__global__ void __launch_bounds__(Geo<DIM, P>::THREADS, KernelShape<LAW, DIM, P>::MIN_BLOCKS)
dg_operator_kernel(const Job job, const DGParams<typename BaseOf<V>::type> prm) {
  using T = typename BaseOf<V>::type;
  using L = typename LawOf<LAW, DIM, T>::type;
  using G = Geo<DIM, P>;
  constexpr int NV = L::NV, NN = G::NN, NF = G::NF, EPB = G::EPB;
  constexpr int PER_ELEM = KernelShape<LAW, DIM, P>::PER_ELEM;
  constexpr bool VISC = KernelShape<LAW, DIM, P>::VISC;
  constexpr bool NSV = KernelShape<LAW, DIM, P>::NSV;
  constexpr int NCH = KernelShape<LAW, DIM, P>::NCH;
  constexpr int NG = DIM + 1;

  if (!job.active()) return;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  // operator matrices first (indexed by node, so kept out of the constant bank)
  T* const sD = reinterpret_cast<T*>(smem_raw);              // [DIM][P][P]
  T* const sSp = sD + DIM * P * P;                           // [DIM][P]
  T* const sSm = sSp + DIM * P;                              // [DIM][P]
  for (int t = threadIdx.x; t < DIM * P * P; t += blockDim.x) {
    const int m = t / (P * P), r = t - m * P * P;
    sD[t] = prm.Dvol[m][r / P][r % P];
  }
  for (int t = threadIdx.x; t < DIM * P; t += blockDim.x) {
    sSp[t] = prm.sp[t / P][t % P];
    sSm[t] = prm.sm[t / P][t % P];
  }
  const bool visc = VISC && prm.visc;
  T* const sDg = sSm + DIM * P;                              // [DIM][P][P] (viscous)
  T* const sgp = sDg + DIM * P * P;                          // [DIM][P]
  T* const sgm = sgp + DIM * P;                              // [DIM][P]
  if (visc) {
    for (int t = threadIdx.x; t < DIM * P * P + 2 * DIM * P; t += blockDim.x) sDg[t] = prm.vtab[t];
  }
  V* const smem = reinterpret_cast<V*>(smem_raw + KernelShape<LAW, DIM, P>::template mats_bytes<V, T>());
  const int le = threadIdx.x / NN;
  const int n = threadIdx.x - le * NN;
  const int e = blockIdx.x * EPB + le;               // element in the (batch) numbering
  const InstGeo<T> geo = inst_geo(prm, blockIdx.x);  // its instance's mesh and scales
  const int el = e - geo.e0;                         // element within the instance
  const bool live = e < prm.nE && el < geo.nE;
  V* const sst = smem + le * PER_ELEM;     // [NV][NN] state
  V* const sdir = sst + NV * NN;           // [NV][NN] direction (R2)
  V* const sG = sdir + NV * NN;            // [DIM][NV][NN] nodal fluxes
  V* const sface = sG + DIM * NV * NN;     // [2*DIM][NV][NF] face fluxes
  V* const sjump = sface + 2 * DIM * NV * NF;   // [2*DIM][NF] u* - u_own (scalar viscous)
  // system viscous: nodal channels [NCH][NN]; per face [2*DIM][NCH][NF] the own
  // trace, the neighbour's trace and the neighbour's normal derivative
  V* const sgc = sjump + (NV == 1 ? 2 * DIM * NF : 0);
  V* const sfo = sgc + NCH * NN;
  V* const sfn = sfo + 2 * DIM * NCH * NF;
  V* const sfd = sfn + 2 * DIM * NCH * NF;

  int ec[3] = {0, 0, 0};
  if (live) {
    ec[0] = el % geo.n[0];
    ec[1] = (el / geo.n[0]) % geo.n[1];
    ec[2] = el / (geo.n[0] * geo.n[1]);
  }
  int idx[3] = {0, 0, 0};
  idx[0] = n % P;
  if (DIM > 1) idx[1] = (n / P) % P;
  if (DIM > 2) idx[2] = n / (P * P);

  V res[Job::K][NV];

#pragma unroll
  for (int k = 0; k < Job::K; ++k) {
    const bool r2 = Job::kind(k) == EV_R2;
    // -- 1. node values and nodal fluxes --------------------------------
    if (live) {
      V w[NV], s[NV];
      job.load_state(k, e, n, w);
      if (r2) job.load_dir(k, e, n, s);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        sst[v * NN + n] = w[v];
        if (r2) sdir[v * NN + n] = s[v];
      }
      if (!L::LINEAR || visc) {
        V F[DIM][NV];
        if (r2) L::jvp_all(w, s, F, prm); else L::flux_all(w, F, prm);
#pragma unroll
        for (int m = 0; m < DIM; ++m)
#pragma unroll
          for (int v = 0; v < NV; ++v) sG[(m * NV + v) * NN + n] = F[m][v];
      }
      if constexpr (NSV) {
        if (visc) {   // gradient variables g = (v, T) (Eq. 26) and, for R2, gs = (dg/dw) s
          V ch[NCH];
          NSVisc<DIM, T>::grad_vars(w, ch, prm);
          if (r2) NSVisc<DIM, T>::grad_vars_jvp(w, s, ch + NG, prm);
#pragma unroll
          for (int q = 0; q < NCH; ++q)
            if (q < NG || r2) sgc[q * NN + n] = ch[q];
        }
      }
    }
    __syncthreads();
    // -- 2. face fluxes ------------------------------------------------------
    // The block's face points are spread over all its threads in face-major
    // order (face direction and side, then element, then point): the threads of
    // a warp mostly run the same face's code, with all lanes active, which on
    // GB300's narrow FP64 pipe matters (a partially masked FP64 warp
    // instruction occupies the pipe as long as a full one).
    for (int wi = threadIdx.x; wi < EPB * 2 * DIM * NF; wi += blockDim.x) {
      const int f = wi / (EPB * NF);
      const int rem = wi - f * (EPB * NF);
      const int fle = rem / NF, pt = rem - fle * NF;
      const int fe = blockIdx.x * EPB + fle, fel = fe - geo.e0;
      if (fe >= prm.nE || fel >= geo.nE) continue;
      int ec[3];
      ec[0] = fel % geo.n[0];
      ec[1] = (fel / geo.n[0]) % geo.n[1];
      ec[2] = fel / (geo.n[0] * geo.n[1]);
      V* const sst = smem + fle * PER_ELEM;
      V* const sdir = sst + NV * NN;
      V* const sface = sdir + NV * NN + DIM * NV * NN;
      V* const sjump = sface + 2 * DIM * NV * NF;
      V* const sgc = sjump + (NV == 1 ? 2 * DIM * NF : 0);
      V* const sfo = sgc + NCH * NN;
      V* const sfn = sfo + 2 * DIM * NCH * NF;
      V* const sfd = sfn + 2 * DIM * NCH * NF;
      {
        using FF = FaceFlux<LAW, DIM, P, LGL, V, Job>;
        if constexpr (NSV) {
          FF::run_face(f >> 1, f & 1, job, prm, geo, k, r2, ec, pt, sst, sdir, sface);
        } else switch (f) {
          case 0: FF::template run<0, 0>(job, prm, geo, k, r2, ec, pt, sst, sdir, sface); break;
          case 1: FF::template run<0, 1>(job, prm, geo, k, r2, ec, pt, sst, sdir, sface); break;
          case 2: if constexpr (DIM > 1) FF::template run<1, 0>(job, prm, geo, k, r2, ec, pt, sst, sdir, sface); break;
          case 3: if constexpr (DIM > 1) FF::template run<1, 1>(job, prm, geo, k, r2, ec, pt, sst, sdir, sface); break;
          case 4: if constexpr (DIM > 2) FF::template run<2, 0>(job, prm, geo, k, r2, ec, pt, sst, sdir, sface); break;
          case 5: if constexpr (DIM > 2) FF::template run<2, 1>(job, prm, geo, k, r2, ec, pt, sst, sdir, sface); break;
          default: break;
        }
        if constexpr (NSV) {
          if (visc) FaceViscSysA<DIM, P, V, Job>::run(job, prm, geo, k, r2, ec, f, pt, sgc, sgp, sgm, sfo, sfn, sfd);
        } else if constexpr (VISC) {
          if (visc) {
            using FV = FaceVisc<DIM, P, V, Job>;
            const V* u = r2 ? sdir : sst;
            switch (f) {
              case 0: FV::template run<0, 0>(job, prm, geo, k, r2, ec, pt, u, sgp, sgm, sface, sjump); break;
              case 1: FV::template run<0, 1>(job, prm, geo, k, r2, ec, pt, u, sgp, sgm, sface, sjump); break;
              case 2: if constexpr (DIM > 1) FV::template run<1, 0>(job, prm, geo, k, r2, ec, pt, u, sgp, sgm, sface, sjump); break;
              case 3: if constexpr (DIM > 1) FV::template run<1, 1>(job, prm, geo, k, r2, ec, pt, u, sgp, sgm, sface, sjump); break;
              case 4: if constexpr (DIM > 2) FV::template run<2, 0>(job, prm, geo, k, r2, ec, pt, u, sgp, sgm, sface, sjump); break;
              case 5: if constexpr (DIM > 2) FV::template run<2, 1>(job, prm, geo, k, r2, ec, pt, u, sgp, sgm, sface, sjump); break;
              default: break;
            }
          }
        }
      }
    }
    __syncthreads();
    // -- 2b (system). Navier-Stokes: the viscous face fluxes (stage B) and, per
    // node, the lifted gradient of every channel (Eq. 29 / Eq. 33, strong form)
    // and the viscous flux F^v (R1) or its linearisation (R2), folded into sG --
    if constexpr (NSV) {
      if (visc) {
        // stage B over the block's face points in face-major order (as pass 2)
        for (int wi = threadIdx.x; wi < EPB * 2 * DIM * NF; wi += blockDim.x) {
          const int f = wi / (EPB * NF);
          const int rem = wi - f * (EPB * NF);
          const int fle = rem / NF, pt = rem - fle * NF;
          const int fe = blockIdx.x * EPB + fle, fel = fe - geo.e0;
          if (fe >= prm.nE || fel >= geo.nE) continue;
          V* const fst = smem + fle * PER_ELEM;
          V* const fface = fst + 2 * NV * NN + DIM * NV * NN;
          V* const fgc = fface + 2 * DIM * NV * NF + (NV == 1 ? 2 * DIM * NF : 0);
          V* const ffo = fgc + NCH * NN;
          V* const ffn = ffo + 2 * DIM * NCH * NF;
          V* const ffd = ffn + 2 * DIM * NCH * NF;
          const int M = f >> 1, side = f & 1;
          const int ecM = M == 0 ? fel % geo.n[0] : (M == 1 ? (fel / geo.n[0]) % geo.n[1] : fel / (geo.n[0] * geo.n[1]));
          const int gnM = M == 0 ? geo.n[0] : (M == 1 ? geo.n[1] : geo.n[2]);
          const bool bnd = bc_kind(prm, M, side) != BC_PERIODIC && (side ? ecM == gnM - 1 : ecM == 0);
          FaceViscSysB<DIM, P, V>::run(prm, geo, r2, f, pt, fgc, sDg, sgp, sgm, ffo, ffn, ffd, fface, bnd);
        }
        if (live) {
          const int nch = r2 ? NCH : NG;
          V d[2][DIM][NG], gch[NCH];
#pragma unroll
          for (int q = 0; q < NCH; ++q) {
            const int set = q / NG, cq = q - set * NG;
            if (q >= nch) {
              gch[q] = V(T(0));
#pragma unroll
              for (int kk = 0; kk < DIM; ++kk) d[set][kk][cq] = V(T(0));
              continue;
            }
            gch[q] = sgc[q * NN + n];
#pragma unroll
            for (int kk = 0; kk < DIM; ++kk) {
              const int st = (kk == 0) ? 1 : (kk == 1 ? P : P * P);
              const int i = idx[kk];
              const int b0 = n - i * st;
              const T* Grow = sDg + (kk * P + i) * P;
              V a = V(T(0));
#pragma unroll
              for (int l = 0; l < P; ++l) a += Grow[l] * sgc[q * NN + b0 + l * st];
              const int pt = (n % st) + (n / (st * P)) * st;
              // u* - u_own at the + and - faces of direction kk
              const V jp = T(0.5) * (sfn[((2 * kk + 1) * NCH + q) * NF + pt] - sfo[((2 * kk + 1) * NCH + q) * NF + pt]);
              const V jm = T(0.5) * (sfn[((2 * kk) * NCH + q) * NF + pt] - sfo[((2 * kk) * NCH + q) * NF + pt]);
              if constexpr (LGL) {
                if (i == P - 1) a -= sSp[kk * P + P - 1] * jp;
                if (i == 0) a += sSm[kk * P] * jm;
              } else {
                a += sSm[kk * P + i] * jm - sSp[kk * P + i] * jp;
              }
              d[set][kk][cq] = geo.hs[kk] * a;
            }
          }
#pragma unroll
          for (int m = 0; m < DIM; ++m) {
            V F[NV];
            if (r2) NSVisc<DIM, T>::flux_lin(gch, d[0], gch + NG, d[1], m, F, prm);
            else NSVisc<DIM, T>::flux(gch, d[0], m, F, prm);
#pragma unroll
            for (int v = 1; v < NV; ++v) sG[(m * NV + v) * NN + n] -= F[v];
          }
        }
        __syncthreads();
      }
    }
    // -- 2b. viscous: lifted gradient (Eq. 29, strong form) folded into sG -----
    //   d^m_i = (2/h)(D u)_i + (2/h) lhat_i(+1)(u*_+ - u_+) - (2/h) lhat_i(-1)(u*_- - u_-)
    if constexpr (VISC && !NSV) {
      if (visc) {
        if (live) {
          const V* u = r2 ? sdir : sst;
#pragma unroll
          for (int m = 0; m < DIM; ++m) {
            const int st = (m == 0) ? 1 : (m == 1 ? P : P * P);
            const int i = idx[m];
            const int b0 = n - i * st;
            const T* Grow = sDg + (m * P + i) * P;
            V d = V(T(0));
#pragma unroll
            for (int l = 0; l < P; ++l) d += Grow[l] * u[b0 + l * st];
            const int pt = (n % st) + (n / (st * P)) * st;
            const V jp = sjump[(2 * m + 1) * NF + pt], jm = sjump[(2 * m) * NF + pt];
            // sp = -(2/h) lhat(+1), sm = -(2/h) lhat(-1)
            if constexpr (LGL) {
              if (i == P - 1) d -= sSp[m * P + P - 1] * jp;
              if (i == 0) d += sSm[m * P] * jm;
            } else {
              d += sSm[m * P + i] * jm - sSp[m * P + i] * jp;
            }
            sG[m * NN + n] -= (geo.nu * geo.hs[m]) * d;
          }
        }
        __syncthreads();
      }
    }
    // -- 3. volume contraction + lifting ---------------------------------------
    if (live) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        V acc = V(T(0));
#pragma unroll
        for (int m = 0; m < DIM; ++m) {
          const int st = (m == 0) ? 1 : (m == 1 ? P : P * P);
          const int i = idx[m];
          const int b0 = n - i * st;
          const V* g;
          if (L::LINEAR && !visc) g = (r2 ? sdir : sst) + v * NN;
          else g = sG + (m * NV + v) * NN;
          const T* Drow = sD + (m * P + i) * P;
          V am = V(T(0));
#pragma unroll
          for (int l = 0; l < P; ++l) am += Drow[l] * g[b0 + l * st];
          const int pt = (n % st) + (n / (st * P)) * st;
          const V* fm = sface + ((2 * m) * NV + v) * NF;
          const V* fpl = sface + ((2 * m + 1) * NV + v) * NF;
          if constexpr (LGL) {
            if (i == P - 1) am += sSp[m * P + P - 1] * fpl[pt];
            if (i == 0) am += sSm[m * P] * fm[pt];
          } else {
            am += sSp[m * P + i] * fpl[pt] + sSm[m * P + i] * fm[pt];
          }
          acc += geo.hs[m] * am;
        }
        res[k][v] = acc;
      }
    }
    if (k + 1 < Job::K) __syncthreads();
  }
  if (live) job.epilogue(e, n, res);
}

// ---------------------------------------------------------------------------
// Jobs.  Index of (element e, variable v, node n): (e * NV + v) * NN + n.
// ---------------------------------------------------------------------------
template <int NV, int NN, typename T>
struct JobR1 {
  static constexpr int K = 1;
  const double* w; double* out;
  __device__ static constexpr int kind(int) { return EV_R1; }
  __device__ bool active() const { return true; }
  __device__ void load_state(int, int e, int n, T* x) const {
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] = T(w[(size_t(e) * NV + v) * NN + n]);
  }
  __device__ void load_dir(int, int, int, T*) const {}
  __device__ void epilogue(int e, int n, const T (*r)[NV]) const {
#pragma unroll
    for (int v = 0; v < NV; ++v) out[(size_t(e) * NV + v) * NN + n] = double(r[0][v]);
  }
};

template <int NV, int NN, typename T>
struct JobR2 {
  static constexpr int K = 1;
  const double* w; const double* s; double* out;
  __device__ static constexpr int kind(int) { return EV_R2; }
  __device__ bool active() const { return true; }
  __device__ void load_state(int, int e, int n, T* x) const {
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] = T(w[(size_t(e) * NV + v) * NN + n]);
  }
  __device__ void load_dir(int, int e, int n, T* x) const {
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] = T(s[(size_t(e) * NV + v) * NN + n]);
  }
  __device__ void epilogue(int e, int n, const T (*r)[NV]) const {
#pragma unroll
    for (int v = 0; v < NV; ++v) out[(size_t(e) * NV + v) * NN + n] = double(r[0][v]);
  }
};

// Extended residual of a stage (Sec. 3.2.1) from X = (W, S):
//   r1 = R1(W), r2 = R2(W, S), G1 = W - b - c1 r1 + c2 r2, G2 = S - r1.
template <int NV, int NN>
struct JobResidual {
  static constexpr int K = 2;
  const double* W; const double* S; const double* b;
  double c1, c2;
  double* G1; double* G2; double* r1; double* r2;
  __device__ static constexpr int kind(int k) { return k == 0 ? EV_R1 : EV_R2; }
  __device__ bool active() const { return true; }
  __device__ void load_state(int, int e, int n, double* x) const {
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] = W[(size_t(e) * NV + v) * NN + n];
  }
  __device__ void load_dir(int, int e, int n, double* x) const {
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] = S[(size_t(e) * NV + v) * NN + n];
  }
  __device__ void epilogue(int e, int n, const double (*r)[NV]) const {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const size_t i = (size_t(e) * NV + v) * NN + n;
      const double a = r[0][v], c = r[1][v];
      r1[i] = a;
      r2[i] = c;
      G1[i] = W[i] - b[i] - c1 * a + c2 * c;
      G2[i] = S[i] - a;
    }
  }
};

// Device-side description of the vector z a Jacobian-vector product acts on:
// z = scale * V[:, col] where col = *jidx (device scalar; 0 if jidx is null),
// scale = vscale[col] (1 if vscale is null) and nrmW[col], nrmS[col] are the
// Euclidean norms of the unscaled W and sigma halves.  The output goes to
// column *out_jidx + out_offset of `out` (same layout).  S is the storage type.
template <typename S>
struct JvInputT {
  const S* V; size_t ld, half;
  const int* jidx;
  const double* vscale;
  const double* nrmW; const double* nrmS;
  const int* skip;              // device flag: nonzero -> nothing to do
  S* out; size_t out_ld; int out_offset;
  const int* out_jidx;          // output column = *out_jidx + out_offset (null -> out_offset)
  __device__ __forceinline__ int col() const { return jidx ? *jidx : 0; }
  __device__ __forceinline__ const S* zW() const { return V + size_t(col()) * ld; }
  __device__ __forceinline__ const S* zS() const { return zW() + half; }
  __device__ __forceinline__ double scale() const { return vscale ? vscale[col()] : 1.0; }
  __device__ __forceinline__ double nW() const { return fabs(scale()) * nrmW[col()]; }
  __device__ __forceinline__ double nS() const { return fabs(scale()) * nrmS[col()]; }
  __device__ __forceinline__ S* oW() const {
    return out + size_t((out_jidx ? *out_jidx : 0) + out_offset) * out_ld;
  }
  __device__ __forceinline__ S* oS() const { return oW() + half; }
  __device__ __forceinline__ bool skipped() const { return skip && *skip; }
};
using JvInput = JvInputT<double>;

struct JvCoef {
  const double* c1;        // device scalars alpha1 dt and alpha2 dt^2 / 2
  const double* c2;
  double sqrt_eps_machine; // sqrt(2^-52)
  double eps_ref;          // reference Mach number in eps_FD
};

// Eq. 23, first part: the two quotients taken at W + eps_w dW,
//   eps_w = sqrt(eps_machine) / (eps ||dW||),
//   t1 = (R1(W + eps_w dW) - R1(W)) / eps_w,  t2 = (R2(W + eps_w dW, S) - R2(W, S)) / eps_w,
//   out = (dW - c1 t1 + c2 t2,  dS - t1).   (||dW|| = 0: t1 = t2 = 0.)
template <int NV, int NN>
struct JobJvFD_A {
  static constexpr int K = 2;
  const double* W; const double* S; const double* r1; const double* r2;
  JvInput z; JvCoef c;
  __device__ static constexpr int kind(int k) { return k == 0 ? EV_R1 : EV_R2; }
  __device__ bool active() const { return !z.skipped(); }
  __device__ double eps_w() const {
    const double nw = z.nW();
    return nw > 0.0 ? c.sqrt_eps_machine / (c.eps_ref * nw) : 0.0;
  }
  __device__ void load_state(int, int e, int n, double* x) const {
    const double ew = eps_w() * z.scale();
    const double* zw = z.zW();
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const size_t i = (size_t(e) * NV + v) * NN + n;
      x[v] = W[i] + ew * zw[i];
    }
  }
  __device__ void load_dir(int, int e, int n, double* x) const {
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] = S[(size_t(e) * NV + v) * NN + n];
  }
  __device__ void epilogue(int e, int n, const double (*r)[NV]) const {
    const double ew = eps_w(), sc = z.scale();
    const double iew = ew > 0.0 ? 1.0 / ew : 0.0;
    const double c1 = *c.c1, c2 = *c.c2;
    const double* zw = z.zW(); const double* zs = z.zS();
    double* ow = z.oW(); double* os = z.oS();
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const size_t i = (size_t(e) * NV + v) * NN + n;
      const double t1 = (r[0][v] - r1[i]) * iew;
      const double t2 = (r[1][v] - r2[i]) * iew;
      ow[i] = sc * zw[i] - c1 * t1 + c2 * t2;
      os[i] = sc * zs[i] - t1;
    }
  }
};

// Eq. 23, second part: out_W += c2 (R2(W, S + eps_s dS) - R2(W, S)) / eps_s.
template <int NV, int NN>
struct JobJvFD_B {
  static constexpr int K = 1;
  const double* W; const double* S; const double* r2;
  JvInput z; JvCoef c;
  __device__ static constexpr int kind(int) { return EV_R2; }
  __device__ bool active() const { return !z.skipped() && z.nS() > 0.0; }
  __device__ double eps_s() const { return c.sqrt_eps_machine / (c.eps_ref * z.nS()); }
  __device__ void load_state(int, int e, int n, double* x) const {
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] = W[(size_t(e) * NV + v) * NN + n];
  }
  __device__ void load_dir(int, int e, int n, double* x) const {
    const double es = eps_s() * z.scale();
    const double* zs = z.zS();
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const size_t i = (size_t(e) * NV + v) * NN + n;
      x[v] = S[i] + es * zs[i];
    }
  }
  __device__ void epilogue(int e, int n, const double (*r)[NV]) const {
    const double ies = 1.0 / eps_s(), c2 = *c.c2;
    double* ow = z.oW();
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const size_t i = (size_t(e) * NV + v) * NN + n;
      ow[i] += c2 * (r[0][v] - r2[i]) * ies;
    }
  }
};

// Eq. 24 (linear flux): out = (dW - c1 R1(dW) + c2 R1(dS), dS - R1(dW)),
// arithmetic in T, vectors stored as S (FP64, or FP32 in the mixed mode).
template <int NV, int NN, typename T = double, typename S = double>
struct JobJvLinear {
  static constexpr int K = 2;
  static constexpr bool kDirectionState = true;   // R1 of Krylov vectors: the derivative
  JvInputT<S> z; JvCoef c;
  __device__ static constexpr int kind(int) { return EV_R1; }
  __device__ bool active() const { return !z.skipped(); }
  __device__ void load_state(int k, int e, int n, T* x) const {
    const S* src = k == 0 ? z.zW() : z.zS();
    const T sc = T(z.scale());
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] = sc * T(src[(size_t(e) * NV + v) * NN + n]);
  }
  __device__ void load_dir(int, int, int, T*) const {}
  __device__ void epilogue(int e, int n, const T (*r)[NV]) const {
    const T c1 = T(*c.c1), c2 = T(*c.c2), sc = T(z.scale());
    const S* zw = z.zW(); const S* zs = z.zS();
    S* ow = z.oW(); S* os = z.oS();
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const size_t i = (size_t(e) * NV + v) * NN + n;
      const T a = r[0][v], b = r[1][v];
      ow[i] = S(sc * T(zw[i]) - c1 * a + c2 * b);
      os[i] = S(sc * T(zs[i]) - a);
    }
  }
};

// Eq. 24 with both operator passes in one: the two halves (dW, dS) of the input
// are the two components of an AdvectionPair evaluation,
//   out = (dW - c1 R1(dW) + c2 R1(dS), dS - R1(dW))   (inviscid linear advection).
template <int NN, typename T = double, typename S = double>
struct JobJvLinearPair {
  static constexpr int K = 1;
  static constexpr bool kDirectionState = true;
  JvInputT<S> z; JvCoef c;
  __device__ static constexpr int kind(int) { return EV_R1; }
  __device__ bool active() const { return !z.skipped(); }
  __device__ void load_state(int, int e, int n, T* x) const {
    const T sc = T(z.scale());
    const size_t i = size_t(e) * NN + n;
    x[0] = sc * T(z.zW()[i]);
    x[1] = sc * T(z.zS()[i]);
  }
  __device__ void load_dir(int, int, int, T*) const {}
  __device__ void epilogue(int e, int n, const T (*r)[2]) const {
    const T c1 = T(*c.c1), c2 = T(*c.c2), sc = T(z.scale());
    const size_t i = size_t(e) * NN + n;
    const T a = r[0][0], b = r[0][1];
    z.oW()[i] = S(sc * T(z.zW()[i]) - c1 * a + c2 * b);
    z.oS()[i] = S(sc * T(z.zS()[i]) - a);
  }
};

// Analytic Jacobian-vector product of the stage system (Eq. 18) in FP32 with
// dual numbers, used by the mixed-precision mode for a nonlinear flux:
//   eval 0: R1 at the dual state W + eps dW          -> eps part R2(W, dW)
//   eval 1: R2 at (W + eps dW, S + eps dS)            -> eps part R2(W, dS) + dR2/dW[dW]
//   out = (dW - c1 R2(W, dW) + c2 (R2(W, dS) + dR2/dW[dW]),  dS - R2(W, dW)),
// i.e. Eq. 18 with dR1/dW = R2(W, .) (Sec. 3.2.1) and the Hessian block taken
// exactly (the dissipation coefficient of a Rusanov flux is frozen).
template <int NV, int NN>
struct JobJvMixed {
  static constexpr int K = 2;
  using V = Dual<float>;
  const float* W; const float* Sg;   // FP32 copies of the linearisation point (W, sigma)
  JvInputT<float> z; JvCoef c;
  __device__ static constexpr int kind(int k) { return k == 0 ? EV_R1 : EV_R2; }
  __device__ bool active() const { return !z.skipped(); }
  __device__ void load_state(int, int e, int n, V* x) const {
    const float sc = float(z.scale());
    const float* zw = z.zW();
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const size_t i = (size_t(e) * NV + v) * NN + n;
      x[v] = V(W[i], sc * zw[i]);
    }
  }
  __device__ void load_dir(int, int e, int n, V* x) const {
    const float sc = float(z.scale());
    const float* zs = z.zS();
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const size_t i = (size_t(e) * NV + v) * NN + n;
      x[v] = V(Sg[i], sc * zs[i]);
    }
  }
  __device__ void epilogue(int e, int n, const V (*r)[NV]) const {
    const float c1 = float(*c.c1), c2 = float(*c.c2), sc = float(z.scale());
    const float* zw = z.zW(); const float* zs = z.zS();
    float* ow = z.oW(); float* os = z.oS();
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const size_t i = (size_t(e) * NV + v) * NN + n;
      const float d0 = r[0][v].d, d1 = r[1][v].d;
      ow[i] = sc * zw[i] - c1 * d0 + c2 * d1;
      os[i] = sc * zs[i] - d0;
    }
  }
};

// Element-diagonal block J_i of the BJ_ext preconditioner (Sec. 3.2.3) by
// columns: column c = blockIdx.y of every element's block is R2(W, e_c) on that
// element with the neighbours' direction zero (kFrozenNb), i.e. dR1/dW
// restricted to the element with the neighbours' values frozen -- for a law
// whose viscous Jacobian has no compact closed form (Navier-Stokes).  Blocks
// are column-major, entry (r, c) at c * n_b + r, as the analytic assembly.
template <int NV, int NN, typename T>
struct JobPcCols {
  static constexpr int K = 1;
  static constexpr bool kFrozenNb = true;
  static constexpr int NB = NV * NN;
  const double* w; T* J;
  __device__ static constexpr int kind(int) { return EV_R2; }
  __device__ bool active() const { return true; }
  __device__ void load_state(int, int e, int n, T* x) const {
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] = T(w[(size_t(e) * NV + v) * NN + n]);
  }
  // only the element's own nodes (neighbours go through load_nb_dir -> 0)
  __device__ void load_dir(int, int, int n, T* x) const {
    const int col = blockIdx.y;
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] = (v * NN + n == col) ? T(1) : T(0);
  }
  __device__ void epilogue(int e, int n, const T (*r)[NV]) const {
    T* Jc = J + (size_t(e) * NB + blockIdx.y) * NB;
#pragma unroll
    for (int v = 0; v < NV; ++v) Jc[v * NN + n] = r[0][v];
  }
};

}  // namespace hbpc
