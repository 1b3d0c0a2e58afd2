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

// One pass of the cooperative CGS2 kernel over the block's tiles of the new
// vector q = V_{j+1}: q -= sum_i c_i V_i (UPDATE, coefficients c already in the
// accumulation type), then either the dot products with V_0..V_{cnt-1} (DOTS,
// to partial[b][col_out + i]) or the squared norms of the W and sigma halves
// (to partial[b][col_out], [col_out + 1]); QQ adds |q|^2 to partial[b][qq_col].
// The hot loop has no FP64 instruction for an FP32 basis (GB300 runs FP64 at
// 1/64 of the FP32 rate); only the cross-warp sums are FP64.
template <typename S, bool UPDATE, bool DOTS, bool QQ>
__device__ __forceinline__ void coop_pass(const KrylovT<S>& K, S* q, int cnt, const typename AccOf<S>::type* s_c,
                                          typename AccOf<S>::type* s_red, int col_out, int qq_col) {
  using A = typename AccOf<S>::type;
  const int stride = cgs_stride(K.m);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ double s_w[3][kVecWarps];
  if (DOTS)
    for (int t = threadIdx.x; t < cnt * kVecWarps; t += blockDim.x) s_red[t] = A(0);
  __syncthreads();
  A aw = A(0), as = A(0), qq = A(0);
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
    if (UPDATE) {
      col_axpy_c(K.V, K.ld, base, x, in, cnt, s_c);
#pragma unroll
      for (int r = 0; r < kRows; ++r) {
        const size_t row = base + size_t(r) * kVecThreads;
        if (in[r]) {
          q[row] = S(x[r]);
          if (row < K.half) aw += x[r] * x[r]; else as += x[r] * x[r];
        }
      }
    }
    if (QQ)
#pragma unroll
      for (int r = 0; r < kRows; ++r) qq += x[r] * x[r];
    if (DOTS) col_dots<true>(K.V, K.ld, base, x, in, cnt, s_red);
  }
  aw = warp_sum(aw); as = warp_sum(as); qq = warp_sum(qq);
  if (lane == 0) { s_w[0][warp] = double(aw); s_w[1][warp] = double(as); s_w[2][warp] = double(qq); }
  __syncthreads();
  double* prow = K.partial + size_t(blockIdx.x) * stride;
  if (DOTS) {
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      double t = 0.0;
      for (int w = 0; w < kVecWarps; ++w) t += double(s_red[i * kVecWarps + w]);
      prow[col_out + i] = t;
    }
  } else if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int w = 0; w < kVecWarps; ++w) { ta += s_w[0][w]; tb += s_w[1][w]; }
    prow[col_out] = ta;
    prow[col_out + 1] = tb;
  }
  if (QQ && threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kVecWarps; ++w) t += s_w[2][w];
    prow[qq_col] = t;
  }
}

// Sum of the blocks' partials of columns [col0, col0 + cnt) into out[c] (times
// scale[c] when given), one warp per column spread over the blocks (the
// reduction is done once, not redundantly by every block).
template <typename S>
__device__ __forceinline__ void coop_reduce(const KrylovT<S>& K, int col0, int cnt, const double* scale,
                                            double* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int stride = cgs_stride(K.m);
  for (int c = blockIdx.x * kVecWarps + warp; c < cnt; c += gridDim.x * kVecWarps) {
    const double t = strided_sum(K.partial + col0 + c, stride, lane, K.nblocks);
    if (lane == 0) out[c] = scale ? t * scale[c] : t;
  }
}

// One Arnoldi column in one cooperative launch (kernel boundaries replaced by
// grid-wide barriers): classical Gram-Schmidt, a second pass only when the DGKS
// test asks for it (|q - sum h_i v_i| < |q| / sqrt 2; the four-kernel form
// always runs it), the Hessenberg column, Givens rotation and stopping test.
// Every reduction across blocks is done once by one warp per column (written to
// hc) and read back by all after a barrier.  Launched with
// cudaLaunchCooperativeKernel, which refuses a grid that cannot be resident.
// The early exit and the column index are read before any block writes the
// state (block 0 writes it after the last barrier), so they are grid-uniform,
// and so is the DGKS decision (every block reads the same reduced values).
// Dynamic shared memory: max((m + 1) doubles + (m + 1)(kVecWarps + 1)
// accumulation values, 3 (m + 2) doubles).
template <typename S>
__global__ void __launch_bounds__(kVecThreads) k_cgs_coop(KrylovT<S> K) {
  using A = typename AccOf<S>::type;
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  GmresState* st = K.st;
  if (st->done) return;
  const int j = st->j, cnt = j + 1, m = K.m;
  extern __shared__ double sm[];
  double* s_h = sm;                                   // [m + 1] reduced coefficients
  A* s_red = reinterpret_cast<A*>(s_h + (m + 1));     // [m + 1][kVecWarps]
  A* s_c = s_red + size_t(m + 1) * kVecWarps;         // [m + 1] update coefficients
  __shared__ int s_flag;
  __shared__ double s_qq;
  S* q = K.V + size_t(j + 1) * K.ld;
  // pass 1: <q, V_i> and |q|^2
  coop_pass<S, false, true, true>(K, q, cnt, s_c, s_red, 0, 2 * m + 1);
  grid.sync();
  // h_i = vscale_i <q, V_i> into hc[0..cnt), |q|^2 into hc[m + 1]
  coop_reduce(K, 0, cnt, K.vscale, K.hc);
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x < 32) {
    const double t = strided_sum(K.partial + 2 * m + 1, cgs_stride(m), threadIdx.x, K.nblocks);
    if (threadIdx.x == 0) K.hc[m + 1] = t;
  }
  grid.sync();
  // the reduced values into shared memory in one parallel round trip
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) s_h[i] = __ldcg(K.hc + i);
  if (threadIdx.x == 0) s_qq = __ldcg(K.hc + m + 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    double hh = 0.0;
    for (int i = 0; i < cnt; ++i) hh += s_h[i] * s_h[i];
    s_flag = (s_qq - hh) < 0.5 * s_qq ? 1 : 0;
  }
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) s_c[i] = A(s_h[i] * K.vscale[i]);
  __syncthreads();
  if (!s_flag) {
    coop_pass<S, true, false, false>(K, q, cnt, s_c, s_red, 2 * (m + 1), 0);   // the only update
    if (blockIdx.x == 0)
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) K.hc[(m + 2) + i] = 0.0;
    grid.sync();
  } else {
    coop_pass<S, true, true, false>(K, q, cnt, s_c, s_red, m + 1, 0);          // update + second dots
    grid.sync();
    coop_reduce(K, m + 1, cnt, K.vscale, K.hc + (m + 2));
    grid.sync();
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) s_c[i] = A(__ldcg(K.hc + (m + 2) + i) * K.vscale[i]);
    __syncthreads();
    coop_pass<S, true, false, false>(K, q, cnt, s_c, s_red, 2 * (m + 1), 0);   // second update + norms
    grid.sync();
  }
  if (blockIdx.x != 0) return;
  __shared__ double nrm[2];
  if (threadIdx.x < 64) {
    const int w = threadIdx.x >> 5;
    const double t = strided_sum(K.partial + 2 * (m + 1) + w, cgs_stride(m), threadIdx.x & 31, K.nblocks);
    if ((threadIdx.x & 31) == 0) nrm[w] = t;
  }
  double* Hj = K.H + size_t(j) * (m + 1);
  for (int i = threadIdx.x; i <= j; i += blockDim.x) Hj[i] = __ldcg(K.hc + i) + __ldcg(K.hc + (m + 2) + i);
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
