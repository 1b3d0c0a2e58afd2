// GMRES building blocks on the device: Arnoldi orthogonalisation (classical
// Gram-Schmidt with one conditional re-orthogonalisation, Daniel-Gragg-Kaufman-
// Stewart criterion), Givens rotations, the small triangular solve and the
// solution update.  The iteration state lives in device memory, so one GMRES
// iteration is a fixed sequence of launches that needs no host round trip and
// can be replayed from a CUDA graph; every kernel returns at once when the
// cycle is finished.  Included by exactly one translation unit.
#pragma once
#include "krylov_common.cuh"

namespace hbpc {

// Squared norms (total, first `half`, rest) of x; result in st->nrm and, if
// given, written to out3.  One launch of nblocks blocks.
__global__ void k_norms(const double* x, size_t n, size_t half, Krylov K, double* out3) {
  size_t lo, hi;
  chunk_range(n, K.nblocks, lo, hi);
  double a = 0.0, b = 0.0;
  for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const double v = x[i];
    if (i < half) a += v * v; else b += v * v;
  }
  __shared__ double s[2][kVecWarps];
  a = warp_sum(a); b = warp_sum(b);
  if ((threadIdx.x & 31) == 0) { s[0][threadIdx.x >> 5] = a; s[1][threadIdx.x >> 5] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int w = 0; w < kVecWarps; ++w) { ta += s[0][w]; tb += s[1][w]; }
    K.partial[size_t(blockIdx.x) * (K.m + 3) + 0] = ta;
    K.partial[size_t(blockIdx.x) * (K.m + 3) + 1] = tb;
  }
  if (!last_block(K.ticket, K.nblocks)) return;
  __shared__ double r[2];
  reduce_partials(K.partial, K.m + 3, K.nblocks, 2, r);
  __syncthreads();
  if (threadIdx.x == 0) {
    K.st->nrm[0] = r[0] + r[1];
    K.st->nrm[1] = r[0];
    K.st->nrm[2] = r[1];
    if (out3) { out3[0] = r[0] + r[1]; out3[1] = r[0]; out3[2] = r[1]; }
  }
}

// Start a cycle from V_0 (already holding the unscaled residual r) with
// v_0 = sign * V_0 / ||V_0||.  Norms come from st->nrm (k_norms on V_0).
// first != 0 also fixes the target tol * ||rhs|| and clears the counters.
__global__ void k_cycle_init(Krylov K, double sign, double tol, int first, int max_its) {
  if (threadIdx.x != 0) return;
  GmresState* st = K.st;
  const double beta = sqrt(st->nrm[0]);
  if (first) { st->target = tol * beta; st->its = 0; st->max_its = max_its; }
  st->m = K.m;
  st->j = 0;
  st->reorth = 0;
  st->breakdown = 0;
  st->resid = beta;
  K.g[0] = beta;
  K.vscale[0] = beta > 0.0 ? sign / beta : 0.0;
  K.nrmW[0] = sqrt(st->nrm[1]);
  K.nrmS[0] = sqrt(st->nrm[2]);
  st->converged = beta <= st->target ? 1 : 0;
  st->done = (st->converged || st->its >= st->max_its) ? 1 : 0;
}

// Column finalisation (one thread): H(j+1, j) = ||q||, rotations, residual,
// stopping decision.  q = V_{j+1}; nq2/nw2/ns2 are its squared norms.
__device__ __forceinline__ void finalize_column(const Krylov& K, double nq2, double nw2, double ns2) {
  GmresState* st = K.st;
  const int j = st->j, ldh = K.m + 1;
  double* Hj = K.H + size_t(j) * ldh;
  const double hnext = sqrt(nq2);
  Hj[j + 1] = hnext;
  K.vscale[j + 1] = hnext > 0.0 ? 1.0 / hnext : 0.0;
  K.nrmW[j + 1] = sqrt(nw2);
  K.nrmS[j + 1] = sqrt(ns2);
  for (int i = 0; i < j; ++i) {           // previous rotations
    const double t = K.cs[i] * Hj[i] + K.sn[i] * Hj[i + 1];
    Hj[i + 1] = -K.sn[i] * Hj[i] + K.cs[i] * Hj[i + 1];
    Hj[i] = t;
  }
  const double den = hypot(Hj[j], Hj[j + 1]);
  const double c = den > 0.0 ? Hj[j] / den : 1.0, s = den > 0.0 ? Hj[j + 1] / den : 0.0;
  K.cs[j] = c; K.sn[j] = s;
  Hj[j] = den; Hj[j + 1] = 0.0;
  K.g[j + 1] = -s * K.g[j];
  K.g[j] = c * K.g[j];
  st->resid = fabs(K.g[j + 1]);
  st->its += 1;
  st->j = j + 1;
  st->reorth = 0;
  const bool ok = st->resid <= st->target;
  const bool brk = !(hnext > 0.0);
  st->breakdown = brk ? 1 : 0;
  st->converged = (ok || brk) ? 1 : 0;
  st->done = (ok || brk || st->j >= K.m || st->its >= st->max_its) ? 1 : 0;
}

// Dot products d_i = <q, V_i>, i = 0..j, with q = V_{j+1}; h_i = vscale_i d_i is
// stored in K.hc.  pass 0: first Gram-Schmidt pass, also ||q||^2 -> st->qq.
// pass 1: re-orthogonalisation pass, runs only if st->reorth.
__global__ void __launch_bounds__(kVecThreads) k_arnoldi_dot(Krylov K, int pass) {
  GmresState* st = K.st;
  if (st->done || (pass == 1 && !st->reorth)) return;
  const int j = st->j;
  const int cnt = j + 1 + (pass == 0 ? 1 : 0);     // + ||q||^2 in the first pass
  const double* q = K.V + size_t(j + 1) * K.ld;
  __shared__ double sq[kSub];
  extern __shared__ double s_acc[];                 // cnt accumulators
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) s_acc[i] = 0.0;
  size_t lo, hi;
  chunk_range(K.n2, K.nblocks, lo, hi);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (size_t c0 = lo; c0 < hi; c0 += kSub) {
    const int len = int(hi - c0 < size_t(kSub) ? hi - c0 : size_t(kSub));
    __syncthreads();
    for (int t = threadIdx.x; t < len; t += blockDim.x) sq[t] = q[c0 + t];
    __syncthreads();
    for (int i = warp; i < cnt; i += kVecWarps) {
      const double* Vi = (i <= j) ? K.V + size_t(i) * K.ld + c0 : nullptr;
      double a = 0.0;
      if (Vi) { for (int t = lane; t < len; t += 32) a += sq[t] * Vi[t]; }
      else { for (int t = lane; t < len; t += 32) a += sq[t] * sq[t]; }
      a = warp_sum(a);
      if (lane == 0) s_acc[i] += a;
    }
  }
  __syncthreads();
  const int stride = K.m + 3;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) K.partial[size_t(blockIdx.x) * stride + i] = s_acc[i];
  if (!last_block(K.ticket, K.nblocks)) return;
  reduce_partials(K.partial, stride, K.nblocks, cnt, K.hc);
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i <= j; ++i) K.hc[i] *= K.vscale[i];
    if (pass == 0) {
      st->qq = K.hc[j + 1];
      double* Hj = K.H + size_t(j) * (K.m + 1);
      for (int i = 0; i <= j; ++i) Hj[i] = K.hc[i];
    } else {
      double* Hj = K.H + size_t(j) * (K.m + 1);
      for (int i = 0; i <= j; ++i) Hj[i] += K.hc[i];
    }
  }
}

// q <- q - sum_i hc_i vscale_i V_i and the squared norms of q.  pass 0: decide
// on re-orthogonalisation (||q_new|| < ||q_old|| / sqrt(2)) or finalise the
// column; pass 1 (only if st->reorth): finalise.
__global__ void __launch_bounds__(kVecThreads) k_arnoldi_update(Krylov K, int pass) {
  GmresState* st = K.st;
  if (st->done || (pass == 1 && !st->reorth)) return;
  const int j = st->j;
  double* q = K.V + size_t(j + 1) * K.ld;
  extern __shared__ double s_coef[];
  for (int i = threadIdx.x; i <= j; i += blockDim.x) s_coef[i] = K.hc[i] * K.vscale[i];
  __syncthreads();
  size_t lo, hi;
  chunk_range(K.n2, K.nblocks, lo, hi);
  double aw = 0.0, as = 0.0;
  for (size_t t = lo + threadIdx.x; t < hi; t += blockDim.x) {
    double x = q[t];
    for (int i = 0; i <= j; ++i) x -= s_coef[i] * K.V[size_t(i) * K.ld + t];
    q[t] = x;
    if (t < K.half) aw += x * x; else as += x * x;
  }
  __shared__ double s[2][kVecWarps];
  aw = warp_sum(aw); as = warp_sum(as);
  if ((threadIdx.x & 31) == 0) { s[0][threadIdx.x >> 5] = aw; s[1][threadIdx.x >> 5] = as; }
  __syncthreads();
  const int stride = K.m + 3;
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int w = 0; w < kVecWarps; ++w) { ta += s[0][w]; tb += s[1][w]; }
    K.partial[size_t(blockIdx.x) * stride + 0] = ta;
    K.partial[size_t(blockIdx.x) * stride + 1] = tb;
  }
  if (!last_block(K.ticket, K.nblocks)) return;
  __shared__ double r[2];
  reduce_partials(K.partial, stride, K.nblocks, 2, r);
  __syncthreads();
  if (threadIdx.x == 0) {
    const double nq2 = r[0] + r[1];
    if (pass == 0 && nq2 < 0.5 * st->qq) {
      st->reorth = 1;
    } else {
      finalize_column(K, nq2, r[0], r[1]);
    }
  }
}

// y = R^-1 g over the j columns of the finished cycle; y_i *= vscale_i.
__global__ void k_solve_y(Krylov K) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int jn = K.st->j, ldh = K.m + 1;
  for (int i = jn - 1; i >= 0; --i) {
    double t = K.g[i];
    for (int k = i + 1; k < jn; ++k) t -= K.H[size_t(k) * ldh + i] * K.y[k];
    const double d = K.H[size_t(i) * ldh + i];
    K.y[i] = d != 0.0 ? t / d : 0.0;
  }
  for (int i = 0; i < jn; ++i) K.y[i] *= K.vscale[i];
}

// x (+)= sum_i y_i V_i over the cycle's columns (accumulate != 0 adds to x).
__global__ void __launch_bounds__(kVecThreads) k_combine(Krylov K, double* x, int accumulate) {
  const int jn = K.st->j;
  extern __shared__ double s_y[];
  for (int i = threadIdx.x; i < jn; i += blockDim.x) s_y[i] = K.y[i];
  __syncthreads();
  size_t lo, hi;
  chunk_range(K.n2, K.nblocks, lo, hi);
  for (size_t t = lo + threadIdx.x; t < hi; t += blockDim.x) {
    double a = accumulate ? x[t] : 0.0;
    for (int i = 0; i < jn; ++i) a += s_y[i] * K.V[size_t(i) * K.ld + t];
    x[t] = a;
  }
}

}  // namespace hbpc
