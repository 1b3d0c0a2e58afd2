// Per-instance GMRES for a batch of independent instances sharing one context
// (hbpc_batch_*): every instance keeps its own Krylov space, Hessenberg matrix,
// Givens rotations, residual and convergence test, while all instances advance
// in lock step (the same column index j), so one launch per kernel serves the
// whole group.  The Jacobian and the block preconditioner are block diagonal
// over instances, so the Jacobian-vector product and the preconditioner apply
// act on all instances' columns at once; only the reductions of the
// Gram-Schmidt process are segmented by instance.
//
// Vectors are cut into tiles of at most kTile rows, each inside one instance's
// W or sigma range (tile table built on the host); the tiles of an instance
// are consecutive.  Columns are normalised explicitly per instance (no lazy
// scale), so the preconditioner apply and the Jacobian-vector product read
// them unscaled.  FP32 basis (the mixed-precision mode); every cross-thread,
// cross-tile and per-instance sum in FP64, in a fixed order.
#pragma once
#include <cooperative_groups.h>

#include "krylov_common.cuh"

namespace hbpc {

template <typename S>
struct BKrylovT {
  S* V; size_t ld, half;
  int m, ninst, ntiles;
  const long long* trow;   // first row of every tile (in the 2 n_dof vector)
  const int* tcnt;         // rows of every tile (<= kTile)
  const int* tinst;        // instance of every tile
  const int* itile;        // tiles of instance i: [itile[i], itile[i + 1])
  double* H;               // per instance (m+1) x m, column-major
  double* cs; double* sn;  // per instance m
  double* g; double* y;    // per instance m + 1
  double* hc;              // per instance 2 (m + 2): coefficients of the two passes
  double* part;            // per tile m + 3 partial sums
  double* inv;             // per instance: scale of the new column
  double* resid; double* target;
  int* conv;               // per instance: 1 once its target is met
  int* jn;                 // per instance: columns of its solution (fixed at convergence)
  GmresState* st;          // the group's column index, iteration count, done flag
};

// Dot products of rows [r0, r0 + cnt) of q with columns 0..j of V into
// part[tile * stride + i] (one tile per block iteration; fixed-order sums).
template <typename S>
__device__ __forceinline__ void bk_tile_dots(const BKrylovT<S>& K, const S* q, long long r0, int cnt, int j,
                                             double* part_row, typename AccOf<S>::type* s_red) {
  using A = typename AccOf<S>::type;
  A qv[kRows];
  bool in[kRows];
#pragma unroll
  for (int r = 0; r < kRows; ++r) {
    const int row = threadIdx.x + r * kVecThreads;
    in[r] = row < cnt;
    qv[r] = in[r] ? A(q[r0 + row]) : A(0);
  }
  col_dots<false>(K.V, K.ld, size_t(r0) + threadIdx.x, qv, in, j + 1, s_red);
  __syncthreads();
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < kVecWarps; ++w) t += double(s_red[i * kVecWarps + w]);
    part_row[i] = t;
  }
  __syncthreads();
}

// Per-instance sums of the tile partials of columns [0, cnt) into
// out[inst * ostride + col] (one warp per (instance, column) pair).
template <typename S>
__device__ __forceinline__ void bk_reduce(const BKrylovT<S>& K, int cnt, int stride, double* out, int ostride) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kVecWarps + warp, nw = gridDim.x * kVecWarps;
  for (int p = gw; p < K.ninst * cnt; p += nw) {
    const int inst = p / cnt, col = p - inst * cnt;
    if (K.conv[inst]) continue;
    const int t0 = K.itile[inst];
    const double s = strided_sum(K.part + size_t(t0) * stride + col, stride, lane, K.itile[inst + 1] - t0);
    if (lane == 0) out[size_t(inst) * ostride + col] = s;
  }
}

// One Arnoldi column of every active instance: CGS2 (two passes) with the
// per-instance reductions, the Hessenberg column, Givens rotation and residual
// of every instance, and the explicit normalisation of the new column.  One
// cooperative launch (grid-wide barriers between the phases; the launch is
// refused if the grid cannot be resident).  The early exit and the column
// index are read before any block writes the state, so they are grid-uniform.
// Dynamic shared memory: (m + 1)(kVecWarps + 1) doubles (covers the
// accumulation arrays and the 3 m + 2 doubles of the per-instance finalisation).
template <typename S>
__global__ void __launch_bounds__(kVecThreads) k_bcgs_coop(BKrylovT<S> K) {
  using A = typename AccOf<S>::type;
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  GmresState* st = K.st;
  if (st->done) return;
  const int j = st->j, cnt = j + 1, m = K.m;
  const int stride = m + 3, hstride = 2 * (m + 2);
  S* q = K.V + size_t(j + 1) * K.ld;
  extern __shared__ double sm_raw[];
  A* s_red = reinterpret_cast<A*>(sm_raw);            // [m + 1][kVecWarps]
  A* s_c = s_red + size_t(m + 1) * kVecWarps;          // [m + 1] coefficients of the tile's instance
  __shared__ double s_w[kVecWarps];
  // pass 1: dots
  for (int t = blockIdx.x; t < K.ntiles; t += gridDim.x) {
    if (K.conv[K.tinst[t]]) continue;
    bk_tile_dots(K, q, K.trow[t], K.tcnt[t], j, K.part + size_t(t) * stride, s_red);
  }
  grid.sync();
  bk_reduce(K, cnt, stride, K.hc, hstride);
  grid.sync();
  // pass 2 (twice): q -= sum h_i V_i; then the second dots, or the squared norm
  for (int pass = 0; pass < 2; ++pass) {
    for (int t = blockIdx.x; t < K.ntiles; t += gridDim.x) {
      const int inst = K.tinst[t];
      if (K.conv[inst]) continue;
      const double* h = K.hc + size_t(inst) * hstride + (pass ? (m + 2) : 0);
      const long long r0 = K.trow[t];
      const int rows = K.tcnt[t];
      for (int i = threadIdx.x; i <= j; i += blockDim.x) s_c[i] = A(__ldcg(h + i));
      __syncthreads();
      A x[kRows];
      bool in[kRows];
#pragma unroll
      for (int r = 0; r < kRows; ++r) {
        const int row = threadIdx.x + r * kVecThreads;
        in[r] = row < rows;
        x[r] = in[r] ? A(q[r0 + row]) : A(0);
      }
      col_axpy_c(K.V, K.ld, size_t(r0) + threadIdx.x, x, in, j + 1, s_c);
      A sq = A(0);
#pragma unroll
      for (int r = 0; r < kRows; ++r) {
        const int row = threadIdx.x + r * kVecThreads;
        if (row < rows) { q[r0 + row] = S(x[r]); sq += x[r] * x[r]; }
      }
      __syncthreads();
      if (pass == 0) {
        bk_tile_dots(K, q, r0, rows, j, K.part + size_t(t) * stride, s_red);
      } else {
        sq = warp_sum(sq);
        if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = double(sq);
        __syncthreads();
        if (threadIdx.x == 0) {
          double tt = 0.0;
          for (int w = 0; w < kVecWarps; ++w) tt += s_w[w];
          K.part[size_t(t) * stride] = tt;
        }
        __syncthreads();
      }
    }
    grid.sync();
    if (pass == 0) {
      bk_reduce(K, cnt, stride, K.hc + (m + 2), hstride);
      grid.sync();
    }
  }
  // per instance (one block each): norm, Hessenberg column h + c, rotations,
  // residual; the column and the rotations are staged in shared memory in one
  // parallel round trip, thread 0 runs the sequential rotation chain there
  {
    double* hcol = reinterpret_cast<double*>(sm_raw);     // [m + 2]
    double* scs = hcol + (m + 2);                         // [m]
    double* ssn = scs + m;                                // [m]
    __shared__ double s_nq;
    for (int inst = blockIdx.x; inst < K.ninst; inst += gridDim.x) {
      if (K.conv[inst]) continue;                         // block-uniform
      const int t0 = K.itile[inst];
      if (threadIdx.x < 32) {
        const double sq = strided_sum(K.part + size_t(t0) * stride, stride, threadIdx.x, K.itile[inst + 1] - t0);
        if (threadIdx.x == 0) s_nq = sq;
      }
      const double* hh = K.hc + size_t(inst) * hstride;
      double* Hj = K.H + size_t(inst) * (m + 1) * m + size_t(j) * (m + 1);
      double* cs = K.cs + size_t(inst) * m;
      double* sn = K.sn + size_t(inst) * m;
      for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        hcol[i] = __ldcg(hh + i) + __ldcg(hh + (m + 2) + i);
        if (i < j) { scs[i] = cs[i]; ssn[i] = sn[i]; }
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double* gg = K.g + size_t(inst) * (m + 1);
        const double hnext = sqrt(s_nq);
        hcol[j + 1] = hnext;
        K.inv[inst] = hnext > 0.0 ? 1.0 / hnext : 0.0;
        for (int i = 0; i < j; ++i) {
          const double a = scs[i] * hcol[i] + ssn[i] * hcol[i + 1];
          hcol[i + 1] = -ssn[i] * hcol[i] + scs[i] * hcol[i + 1];
          hcol[i] = a;
        }
        const double den = hypot(hcol[j], hcol[j + 1]);
        const double c = den > 0.0 ? hcol[j] / den : 1.0, sv = den > 0.0 ? hcol[j + 1] / den : 0.0;
        cs[j] = c; sn[j] = sv;
        hcol[j] = den; hcol[j + 1] = 0.0;
        const double gj = gg[j];
        gg[j + 1] = -sv * gj;
        gg[j] = c * gj;
        K.resid[inst] = fabs(gg[j + 1]);
        K.jn[inst] = j + 1;
        if (K.resid[inst] <= K.target[inst] || !(hnext > 0.0)) K.conv[inst] = 1;
      }
      __syncthreads();
      for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) Hj[i] = hcol[i];
      __syncthreads();
    }
  }
  grid.sync();
  // normalise the new column of every instance that computed it
  for (int t = blockIdx.x; t < K.ntiles; t += gridDim.x) {
    const int inst = K.tinst[t];
    if (K.jn[inst] != j + 1) continue;   // converged before this column
    const S sc = S(K.inv[inst]);
    const long long r0 = K.trow[t];
    const int rows = K.tcnt[t];
    for (int row = threadIdx.x; row < rows; row += blockDim.x) q[r0 + row] *= sc;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int all = 1;
    for (int i = 0; i < K.ninst; ++i) all &= K.conv[i];
    st->its += 1;
    st->j = j + 1;
    st->converged = all;
    st->done = (all || st->j >= m || st->its >= st->max_its) ? 1 : 0;
  }
}

// Squared norm of every tile of column 0 into part[tile * stride].
template <typename S>
__global__ void __launch_bounds__(kVecThreads) k_btile_sqnorm(BKrylovT<S> K) {
  using A = typename AccOf<S>::type;
  __shared__ double s[kVecWarps];
  const int stride = K.m + 3;
  for (int t = blockIdx.x; t < K.ntiles; t += gridDim.x) {
    const long long r0 = K.trow[t];
    A a = A(0);
    for (int row = threadIdx.x; row < K.tcnt[t]; row += blockDim.x) {
      const A v = A(K.V[r0 + row]);
      a += v * v;
    }
    a = warp_sum(a);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = double(a);
    __syncthreads();
    if (threadIdx.x == 0) {
      double tt = 0.0;
      for (int w = 0; w < kVecWarps; ++w) tt += s[w];
      K.part[size_t(t) * stride] = tt;
    }
    __syncthreads();
  }
}

// Start a cycle of every instance from column 0 (the unscaled residual r):
// beta_i = |r_i|, g_i = beta_i e_1, v_0 = sign r_i / beta_i (scale stored in
// inv for k_bscale0); first != 0 fixes target_i = tol beta_i and clears the
// iteration count.  One block; warp w handles instances w, w + 8, ..
template <typename S>
__global__ void k_bcycle_init(BKrylovT<S> K, double sign, double tol, int first, int max_its) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int stride = K.m + 3;
  __shared__ int s_all;
  if (threadIdx.x == 0) s_all = 1;
  __syncthreads();
  for (int inst = warp; inst < K.ninst; inst += blockDim.x >> 5) {
    double s = 0.0;
    for (int t = K.itile[inst] + lane; t < K.itile[inst + 1]; t += 32) s += K.part[size_t(t) * stride];
    s = warp_sum(s);
    if (lane == 0) {
      const double beta = sqrt(s);
      if (first) K.target[inst] = tol * beta;
      K.g[size_t(inst) * (K.m + 1)] = beta;
      K.inv[inst] = beta > 0.0 ? sign / beta : 0.0;
      K.resid[inst] = beta;
      K.jn[inst] = 0;
      // an instance already within its target (or with a zero residual) takes no step
      K.conv[inst] = (beta <= K.target[inst]) ? 1 : 0;
      if (!K.conv[inst]) atomicAnd(&s_all, 0);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    GmresState* st = K.st;
    if (first) { st->its = 0; st->max_its = max_its; }
    st->m = K.m;
    st->j = 0;
    st->converged = s_all;
    st->done = (s_all || st->its >= st->max_its) ? 1 : 0;
  }
}

// Column 0 times the per-instance scale inv.
template <typename S>
__global__ void __launch_bounds__(kVecThreads) k_bscale0(BKrylovT<S> K) {
  for (int t = blockIdx.x; t < K.ntiles; t += gridDim.x) {
    const S sc = S(K.inv[K.tinst[t]]);
    const long long r0 = K.trow[t];
    for (int row = threadIdx.x; row < K.tcnt[t]; row += blockDim.x) K.V[r0 + row] *= sc;
  }
}

// y_i = R_i^-1 g_i over the jn_i columns of every instance (one warp each).
template <typename S>
__global__ void k_bsolve_y(BKrylovT<S> K) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ldh = K.m + 1;
  for (int inst = blockIdx.x * (blockDim.x >> 5) + warp; inst < K.ninst; inst += gridDim.x * (blockDim.x >> 5)) {
    const int jn = K.jn[inst];
    const double* H = K.H + size_t(inst) * ldh * K.m;
    double* y = K.y + size_t(inst) * (K.m + 1);
    const double* g = K.g + size_t(inst) * (K.m + 1);
    for (int i = lane; i < jn; i += 32) y[i] = g[i];
    __syncwarp();
    for (int i = jn - 1; i >= 0; --i) {
      const double d = H[size_t(i) * ldh + i];
      const double yi = d != 0.0 ? y[i] / d : 0.0;
      __syncwarp();
      if (lane == 0) y[i] = yi;
      for (int k2 = lane; k2 < i; k2 += 32) y[k2] -= H[size_t(i) * ldh + k2] * yi;
      __syncwarp();
    }
  }
}

// x (+)= sum_{i < jn_inst} y_inst,i V_i on every tile (accumulate != 0 adds).
template <typename S, typename X>
__global__ void __launch_bounds__(kVecThreads) k_bcombine(BKrylovT<S> K, X* x, int accumulate) {
  using A = typename AccOf<S>::type;
  for (int t = blockIdx.x; t < K.ntiles; t += gridDim.x) {
    const int inst = K.tinst[t];
    const int jn = K.jn[inst];
    const double* y = K.y + size_t(inst) * (K.m + 1);
    const long long r0 = K.trow[t];
    const int rows = K.tcnt[t];
    A a[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) a[r] = A(0);
    for (int i = 0; i < jn; ++i) {
      const S* Vi = K.V + size_t(i) * K.ld;
      const A yi = A(y[i]);
#pragma unroll
      for (int r = 0; r < kRows; ++r) {
        const int row = threadIdx.x + r * kVecThreads;
        if (row < rows) a[r] += yi * A(Vi[r0 + row]);
      }
    }
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const int row = threadIdx.x + r * kVecThreads;
      if (row < rows) x[r0 + row] = accumulate ? X(double(x[r0 + row]) + double(a[r])) : X(a[r]);
    }
  }
}

}  // namespace hbpc
