// GMRES building blocks on the device: Arnoldi orthogonalisation (classical
// Gram-Schmidt with one conditional re-orthogonalisation, Daniel-Gragg-Kaufman-
// Stewart criterion), Givens rotations, the small triangular solve and the
// solution update.  The iteration state lives in device memory, so one GMRES
// iteration is a fixed sequence of launches that needs no host round trip and
// can be replayed from a CUDA graph; every kernel returns at once when the
// cycle is finished.  Included by exactly one translation unit.
#pragma once
#include <cooperative_groups.h>

#include "krylov_common.cuh"

namespace hbpc {

// Squared norms (total, first `half`, rest) of x; result in st->nrm and, if
// given, written to out3.  One launch of nblocks blocks.
template <typename S, typename V>
__global__ void k_norms(const V* x, size_t n, size_t half, KrylovT<S> K, double* out3) {
  size_t lo, hi;
  chunk_range(n, K.nblocks, lo, hi);
  double a = 0.0, b = 0.0;
  for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const double v = double(x[i]);
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
template <typename S>
__global__ void k_cycle_init(KrylovT<S> K, double sign, double tol, int first, int max_its) {
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

// Column finalisation: H(j+1, j) = ||q||, rotations, residual, stopping
// decision.  q = V_{j+1}; nq2/nw2/ns2 are its squared norms.  Called by every
// thread of the last block: the column and the rotations are staged in shared
// memory in parallel, thread 0 applies the rotations there (the chain is
// sequential by nature) and the column is written back in parallel.
template <typename S>
__device__ __forceinline__ void finalize_column(const KrylovT<S>& K, double nq2, double nw2, double ns2,
                                                double* sh /* >= 3 (m+2) doubles */) {
  GmresState* st = K.st;
  const int j = st->j, ldh = K.m + 1;
  double* Hj = K.H + size_t(j) * ldh;
  double* hcol = sh;
  double* scs = sh + (K.m + 2);
  double* ssn = scs + (K.m + 2);
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    hcol[i] = Hj[i];
    scs[i] = K.cs[i];
    ssn[i] = K.sn[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double hnext = sqrt(nq2);
    hcol[j + 1] = hnext;
    K.vscale[j + 1] = hnext > 0.0 ? 1.0 / hnext : 0.0;
    K.nrmW[j + 1] = sqrt(nw2);
    K.nrmS[j + 1] = sqrt(ns2);
    for (int i = 0; i < j; ++i) {           // previous rotations
      const double t = scs[i] * hcol[i] + ssn[i] * hcol[i + 1];
      hcol[i + 1] = -ssn[i] * hcol[i] + scs[i] * hcol[i + 1];
      hcol[i] = t;
    }
    const double den = hypot(hcol[j], hcol[j + 1]);
    const double c = den > 0.0 ? hcol[j] / den : 1.0, s = den > 0.0 ? hcol[j + 1] / den : 0.0;
    K.cs[j] = c; K.sn[j] = s;
    hcol[j] = den; hcol[j + 1] = 0.0;
    const double gj = K.g[j];
    K.g[j + 1] = -s * gj;
    K.g[j] = c * gj;
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
  __syncthreads();
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) Hj[i] = hcol[i];
}

// ---------------------------------------------------------------------------
// Classical Gram-Schmidt with re-orthogonalisation (CGS2) in three passes and a
// finalisation, without single-block tails: every pass writes per-block partial
// sums; the next pass's blocks all reduce them redundantly in their prologue
// (same data, same order, hence the same value in every block).
//   pass A  k_cgs_dot:        P0[b][i]  = <q, V_i>_b                         i <= j
//   pass B  k_cgs_update_dot: h_i = vscale_i sum_b P0[b][i];  q1 = q - sum h_i v_i;
//                             P2[b][i]  = <q1, V_i>_b
//   pass C  k_cgs_update:     c_i = vscale_i sum_b P2[b][i];  q2 = q1 - sum c_i v_i;
//                             P3[b]     = (|q2_W|^2, |q2_S|^2)_b
//   k_cgs_finalize (1 block): H(:, j) = h + c, H(j+1, j) = |q2|, Givens rotation,
//                             residual and stopping decision.
// Partial layout: row b of K.partial holds P0 / P2 in columns [0, m+1) and
// [m+1, 2m+2), P3 in the two columns after.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int cgs_stride(int m) { return 2 * (m + 1) + 2; }

// Block-redundant reduction of partial columns [col0, col0 + cnt) into shared
// s_out (times vscale when given).  Warp w handles columns w, w + 8, ..
__device__ __forceinline__ void cgs_reduce_cols(const double* partial, int stride, int nb, int col0, int cnt,
                                                const double* vscale, double* s_out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = warp; c < cnt; c += kVecWarps) {
    const double t = strided_sum(partial + col0 + c, stride, lane, nb);
    if (lane == 0) s_out[c] = vscale ? t * vscale[c] : t;
  }
}

template <typename S>
__global__ void __launch_bounds__(kVecThreads) k_cgs_dot(KrylovT<S> K) {
  using A = typename AccOf<S>::type;
  GmresState* st = K.st;
  if (st->done) return;
  const int j = st->j, cnt = j + 1;
  const S* q = K.V + size_t(j + 1) * K.ld;
  extern __shared__ double s_red[];                 // [cnt][kVecWarps]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = threadIdx.x; t < cnt * kVecWarps; t += blockDim.x) s_red[t] = 0.0;
  __syncthreads();
  const size_t ntiles = (K.n2 + kTile - 1) / kTile;
  for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const size_t base = tile * kTile + threadIdx.x;
    A qv[kRows];
    bool in[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const size_t row = base + size_t(r) * kVecThreads;
      in[r] = row < K.n2;
      qv[r] = in[r] ? A(q[row]) : A(0);
    }
    col_dots<true>(K.V, K.ld, base, qv, in, cnt, s_red);
  }
  __syncthreads();
  const int stride = cgs_stride(K.m);
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < kVecWarps; ++w) s += s_red[i * kVecWarps + w];
    K.partial[size_t(blockIdx.x) * stride + i] = s;
  }
}

// q <- q - sum_i c_i vscale_i V_i for the rows of this block, with c from the
// partials at column col0 (prologue), then either the next pass's dot partials
// (with_dot) or the squared norms of the result.
template <typename S, bool WITH_DOT>
__device__ __forceinline__ void cgs_update_body(const KrylovT<S>& K, int j, int col_in, int col_out,
                                                double* s_h, double* s_red, bool reduce = true) {
  using A = typename AccOf<S>::type;
  const int cnt = j + 1;
  const int stride = cgs_stride(K.m);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  S* q = K.V + size_t(j + 1) * K.ld;
  // prologue: this pass's coefficients, reduced redundantly by every block
  // (unless the caller has them in s_h already)
  if (reduce) cgs_reduce_cols(K.partial, stride, K.nblocks, col_in, cnt, K.vscale, s_h);
  if (WITH_DOT)
    for (int t = threadIdx.x; t < cnt * kVecWarps; t += blockDim.x) s_red[t] = 0.0;
  __syncthreads();
  A aw = A(0), as = A(0);
  const size_t ntiles = (K.n2 + kTile - 1) / kTile;
  for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const size_t base = tile * kTile + threadIdx.x;
    A x[kRows];
    bool in[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const size_t row = base + size_t(r) * kVecThreads;
      in[r] = row < K.n2;
      x[r] = in[r] ? A(q[row]) : A(0);
    }
    col_axpy(K.V, K.ld, base, x, in, cnt, s_h, K.vscale);
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const size_t row = base + size_t(r) * kVecThreads;
      if (in[r]) {
        q[row] = S(x[r]);
        if (row < K.half) aw += x[r] * x[r]; else as += x[r] * x[r];
      }
    }
    if (WITH_DOT) col_dots<true>(K.V, K.ld, base, x, in, cnt, s_red);
  }
  if (WITH_DOT) {
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      double s = 0.0;
      for (int w = 0; w < kVecWarps; ++w) s += s_red[i * kVecWarps + w];
      K.partial[size_t(blockIdx.x) * stride + col_out + i] = s;
    }
  } else {
    __shared__ double s2[2][kVecWarps];
    aw = warp_sum(aw); as = warp_sum(as);
    if (lane == 0) { s2[0][warp] = double(aw); s2[1][warp] = double(as); }
    __syncthreads();
    if (threadIdx.x == 0) {
      double ta = 0.0, tb = 0.0;
      for (int w = 0; w < kVecWarps; ++w) { ta += s2[0][w]; tb += s2[1][w]; }
      K.partial[size_t(blockIdx.x) * stride + col_out] = ta;
      K.partial[size_t(blockIdx.x) * stride + col_out + 1] = tb;
    }
  }
  if (blockIdx.x == 0)   // the coefficients of this pass for the Hessenberg column
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) (WITH_DOT ? K.hc : K.hc + (K.m + 2))[i] = s_h[i];
}

template <typename S>
__global__ void __launch_bounds__(kVecThreads) k_cgs_update_dot(KrylovT<S> K) {
  if (K.st->done) return;
  extern __shared__ double sm[];          // s_h [m+1] | s_red [(m+1) kVecWarps]
  cgs_update_body<S, true>(K, K.st->j, 0, K.m + 1, sm, sm + (K.m + 1));
}

template <typename S>
__global__ void __launch_bounds__(kVecThreads) k_cgs_update(KrylovT<S> K) {
  if (K.st->done) return;
  extern __shared__ double sm[];
  cgs_update_body<S, false>(K, K.st->j, K.m + 1, 2 * (K.m + 1), sm, nullptr);
}

// One block: norms of q2, Hessenberg column h + c, rotation, stopping decision.
template <typename S>
__global__ void __launch_bounds__(kVecThreads) k_cgs_finalize(KrylovT<S> K) {
  GmresState* st = K.st;
  if (st->done) return;
  const int j = st->j;
  extern __shared__ double sm[];          // >= 3 (m+2) doubles
  __shared__ double nrm[2];
  cgs_reduce_cols(K.partial, cgs_stride(K.m), K.nblocks, 2 * (K.m + 1), 2, nullptr, nrm);
  double* Hj = K.H + size_t(j) * (K.m + 1);
  for (int i = threadIdx.x; i <= j; i += blockDim.x) Hj[i] = K.hc[i] + K.hc[(K.m + 2) + i];
  __syncthreads();
  finalize_column(K, nrm[0] + nrm[1], nrm[0], nrm[1], sm);
}

// The CGS2 passes and the finalisation in one cooperative launch, the kernel
// boundaries replaced by grid-wide barriers; the second Gram-Schmidt pass runs
// only when the DGKS test asks for it (the four-kernel form always runs it).
// Launched with cudaLaunchCooperativeKernel, which refuses a grid whose blocks
// cannot all be resident, so every barrier is reached by every block.  The
// early exit reads st->done before any block writes the state (the state is
// written only by block 0 after the last barrier), so it is grid-uniform.
// Dynamic shared memory: max((m+1)(kVecWarps+1), 3(m+2)) doubles.
template <typename S>
__global__ void __launch_bounds__(kVecThreads) k_cgs_coop(KrylovT<S> K) {
  using A = typename AccOf<S>::type;
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  GmresState* st = K.st;
  if (st->done) return;
  const int j = st->j, cnt = j + 1;
  const int stride = cgs_stride(K.m);
  extern __shared__ double sm[];
  __shared__ double s_qq[kVecWarps];
  __shared__ int s_flag;
  {   // pass A: partial dots <q, V_i>_b and |q|^2
    const S* q = K.V + size_t(j + 1) * K.ld;
    double* s_red = sm;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double qq_b = 0.0;
    for (int t = threadIdx.x; t < cnt * kVecWarps; t += blockDim.x) s_red[t] = 0.0;
    __syncthreads();
    const size_t ntiles = (K.n2 + kTile - 1) / kTile;
    for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      const size_t base = tile * kTile + threadIdx.x;
      A qv[kRows];
      bool in[kRows];
#pragma unroll
      for (int r = 0; r < kRows; ++r) {
        const size_t row = base + size_t(r) * kVecThreads;
        in[r] = row < K.n2;
        qv[r] = in[r] ? A(q[row]) : A(0);
      }
      col_dots<true>(K.V, K.ld, base, qv, in, cnt, s_red);
      A qq = A(0);
#pragma unroll
      for (int r = 0; r < kRows; ++r) qq += qv[r] * qv[r];
      qq_b += double(warp_sum(qq));
    }
    if (lane == 0) s_qq[warp] = qq_b;
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      double t = 0.0;
      for (int w = 0; w < kVecWarps; ++w) t += s_red[i * kVecWarps + w];
      K.partial[size_t(blockIdx.x) * stride + i] = t;
    }
    if (threadIdx.x == 0) {   // |q|^2 of this block's rows; column 2m+1 is free until pass C
      double t = 0.0;
      for (int w = 0; w < kVecWarps; ++w) t += s_qq[w];
      K.partial[size_t(blockIdx.x) * stride + 2 * K.m + 1] = t;
    }
  }
  __threadfence();
  grid.sync();
  // first-pass coefficients h_i = <q, v_i> and |q|^2, reduced redundantly (and
  // identically) by every block; a second Gram-Schmidt pass only when the
  // projection removed more than half of |q|^2 (the DGKS criterion
  // |q - sum h_i v_i| < |q| / sqrt 2), decided identically in every block
  cgs_reduce_cols(K.partial, stride, K.nblocks, 0, cnt, K.vscale, sm);
  if ((threadIdx.x >> 5) == 0) {
    const double t = strided_sum(K.partial + 2 * K.m + 1, stride, threadIdx.x & 31, K.nblocks);
    if (threadIdx.x == 0) s_qq[0] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double hh = 0.0;
    for (int i = 0; i < cnt; ++i) hh += sm[i] * sm[i];
    s_flag = (s_qq[0] - hh) < 0.5 * s_qq[0] ? 1 : 0;
  }
  __syncthreads();
  if (s_flag) {
    cgs_update_body<S, true>(K, j, 0, K.m + 1, sm, sm + (K.m + 1), false);      // pass B
    __threadfence();
    grid.sync();
    cgs_update_body<S, false>(K, j, K.m + 1, 2 * (K.m + 1), sm, nullptr);      // pass C
  } else {
    cgs_update_body<S, false>(K, j, 0, 2 * (K.m + 1), sm, nullptr, false);     // the only update
    if (blockIdx.x == 0)   // its coefficients went to the second slot: the first is zero
      for (int i = threadIdx.x; i <= j; i += blockDim.x) K.hc[i] = 0.0;
  }
  __threadfence();
  grid.sync();
  if (blockIdx.x != 0) return;
  __shared__ double nrm[2];
  cgs_reduce_cols(K.partial, stride, K.nblocks, 2 * (K.m + 1), 2, nullptr, nrm);
  double* Hj = K.H + size_t(j) * (K.m + 1);
  for (int i = threadIdx.x; i <= j; i += blockDim.x) Hj[i] = K.hc[i] + K.hc[(K.m + 2) + i];
  __syncthreads();
  finalize_column(K, nrm[0] + nrm[1], nrm[0], nrm[1], sm);
}

// y = R^-1 g over the j columns of the finished cycle; y_i *= vscale_i.  One
// warp, column-oriented back substitution (lane k owns y_k).
template <typename S>
__global__ void k_solve_y(KrylovT<S> K) {
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  const int jn = K.st->j, ldh = K.m + 1, lane = threadIdx.x;
  for (int i = lane; i < jn; i += 32) K.y[i] = K.g[i];
  __syncwarp();
  for (int i = jn - 1; i >= 0; --i) {
    const double d = K.H[size_t(i) * ldh + i];
    const double yi = d != 0.0 ? K.y[i] / d : 0.0;
    __syncwarp();
    if (lane == 0) K.y[i] = yi;
    for (int k2 = lane; k2 < i; k2 += 32) K.y[k2] -= K.H[size_t(i) * ldh + k2] * yi;
    __syncwarp();
  }
  for (int i = lane; i < jn; i += 32) K.y[i] *= K.vscale[i];
}

// x (+)= sum_i y_i V_i over the cycle's columns (accumulate != 0 adds to x).
template <typename S, typename X>
__global__ void __launch_bounds__(kVecThreads) k_combine(KrylovT<S> K, X* x, int accumulate) {
  using A = typename AccOf<S>::type;
  const int jn = K.st->j;
  extern __shared__ double s_y[];
  for (int i = threadIdx.x; i < jn; i += blockDim.x) s_y[i] = K.y[i];
  __syncthreads();
  const size_t ntiles = (K.n2 + kTile - 1) / kTile;
  for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const size_t base = tile * kTile + threadIdx.x;
    A a[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) a[r] = A(0);
    for (int i = 0; i < jn; ++i) {
      const S* Vi = K.V + size_t(i) * K.ld;
      const A y = A(s_y[i]);
#pragma unroll
      for (int r = 0; r < kRows; ++r) {
        const size_t row = base + size_t(r) * kVecThreads;
        if (row < K.n2) a[r] += y * A(Vi[row]);
      }
    }
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const size_t row = base + size_t(r) * kVecThreads;
      if (row < K.n2) x[row] = accumulate ? X(double(x[row]) + double(a[r])) : X(a[r]);
    }
  }
}

}  // namespace hbpc
