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
__device__ __host__ __forceinline__ int cgs_stride(int m) { return 2 * (m + 1) + 4; }

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

// ---------------------------------------------------------------------------
// One Arnoldi column with two grid-wide barriers in the common case.
//
// Classical Gram-Schmidt needs <q, V_i> for i <= j and, for the Hessenberg
// entry H(j+1, j), the norm of q - sum h_i v_i.  With an orthonormal basis that
// norm follows from |q|^2 and the coefficients (Pythagoras):
//     |q - V h|^2 = |q|^2 - |h|^2,
// accurate to rounding whenever no cancellation has happened, i.e. exactly when
// the DGKS test |q|^2 - |h|^2 >= |q|^2 / 2 says that no second pass is needed.
// So the column is
//   pass 1: block partials of <q, V_i> and |q|^2                 grid barrier
//   the sums over the blocks, one warp per sum over the grid      grid barrier
//   every block reads h and |q|^2 back and takes the DGKS test (grid-uniform)
//   common case:  the last block closes the column (H(:, j) = h, H(j+1, j) from
//                 Pythagoras, Givens rotation, residual, stopping test) while
//                 every block applies q -= sum h_i v_i to its rows
//   re-orthogonalisation (DGKS): q -= V h with second-pass partials of
//                 <q', V_i> and |q'|^2, summed the same way   two grid barriers
//                 the last block closes the column with H(:, j) = h + c and
//                 H(j+1, j)^2 = |q'|^2 - |c|^2; every block applies q' -= V c.
// The norms of the two halves of the new vector (needed only by the
// difference-quotient Jv without a preconditioner, half_norms != 0) are summed
// by the last block to finish (ticket, no waiting).
// Partial layout per block row (stride cgs_stride(m) = 2 m + 6): pass-1 dots
// [0, m + 1), |q|^2 at m + 1, pass-2 dots [m + 2, 2 m + 3), |q'|^2 at 2 m + 3,
// half norms at 2 m + 4 and 2 m + 5.
// Dot products are summed per thread over the block's rows for chunks of C
// columns, then across the warp with a transposed butterfly (C - 1 + 5 -
// log2 C exchanges per lane instead of 5 C), then across warps and blocks in
// FP64 in a fixed order.
// ---------------------------------------------------------------------------

// Transposed warp sum of C per-lane partials a[0..C): afterwards a[0] of lane
// l holds the warp total of column l / (32 / C) (the same value in the 32 / C
// lanes of that column).  C is a power of two, 1 <= C <= 32.
template <int K, int O, typename A>
struct TransposeSum {
  __device__ __forceinline__ static void run(A* a, int lane) {
    const bool up = (lane & O) != 0;
#pragma unroll
    for (int i = 0; i < K / 2; ++i) {
      const A send = up ? a[i] : a[i + K / 2];
      const A keep = up ? a[i + K / 2] : a[i];
      a[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
    }
    TransposeSum<K / 2, O / 2, A>::run(a, lane);
  }
};
template <int O, typename A>
struct TransposeSum<1, O, A> {
  __device__ __forceinline__ static void run(A* a, int) {
#pragma unroll
    for (int o = O; o > 0; o >>= 1) a[0] += __shfl_xor_sync(0xffffffffu, a[0], o);
  }
};

constexpr int kCgsChunk = 16;   // columns per transposed reduction

// Block partials of <q, V_i> for i in [0, cnt) into s_w[warp * ldw + i]
// (per-warp totals), and of |q|^2 into s_qq[warp] when QQ.
template <typename S, bool QQ>
__device__ __forceinline__ void lowsync_dots(const KrylovT<S>& K, const S* q, int cnt, double* s_w, int ldw,
                                             double* s_qq) {
  using A = typename AccOf<S>::type;
  constexpr int C = kCgsChunk, L = 32 / C;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t ntiles = (K.n2 + kTile - 1) / kTile;
  A qq = A(0);
  for (int c0 = 0; c0 < cnt; c0 += C) {
    const int nc = cnt - c0 < C ? cnt - c0 : C;
    A acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = A(0);
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
      if (QQ && c0 == 0)
#pragma unroll
        for (int r = 0; r < kRows; ++r) qq += x[r] * x[r];
      const S* V0 = K.V + size_t(c0) * K.ld + base;
      if (nc == C) {
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
          for (int r = 0; r < kRows; ++r)
            if (in[r]) acc[c] += x[r] * A(V0[size_t(c) * K.ld + size_t(r) * kVecThreads]);
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c)
          if (c < nc)
#pragma unroll
            for (int r = 0; r < kRows; ++r)
              if (in[r]) acc[c] += x[r] * A(V0[size_t(c) * K.ld + size_t(r) * kVecThreads]);
      }
    }
    TransposeSum<C, 16, A>::run(acc, lane);
    if ((lane % L) == 0) {
      const int c = c0 + lane / L;
      if (c < cnt) s_w[warp * ldw + c] = double(acc[0]);
    }
  }
  if (QQ) {
    qq = warp_sum(qq);
    if (lane == 0) s_qq[warp] = double(qq);
  }
}

// q -= sum_{i < cnt} s_c[i] V_i over the block's rows (coefficients already in
// the accumulation type and scaled for the unscaled columns); with HALF the
// squared norms of the two halves of the result into s_n[0][warp], s_n[1][warp].
template <typename S, bool HALF>
__device__ __forceinline__ void lowsync_update(const KrylovT<S>& K, S* q, int cnt,
                                               const typename AccOf<S>::type* s_c, double (*s_n)[kVecWarps]) {
  using A = typename AccOf<S>::type;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t ntiles = (K.n2 + kTile - 1) / kTile;
  A aw = A(0), as = A(0);
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
    col_axpy_c(K.V, K.ld, base, x, in, cnt, s_c);
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const size_t row = base + size_t(r) * kVecThreads;
      if (in[r]) {
        q[row] = S(x[r]);
        if (HALF) { if (row < K.half) aw += x[r] * x[r]; else as += x[r] * x[r]; }
      }
    }
  }
  if (HALF) {
    aw = warp_sum(aw);
    as = warp_sum(as);
    if (lane == 0) { s_n[0][warp] = double(aw); s_n[1][warp] = double(as); }
  }
}

// One block closes column j: H(0..j, j) = hcol[0..j] (in shared memory),
// H(j+1, j) = hnext, vscale[j+1] = 1 / hnext, previous rotations, the new
// rotation, residual and stopping decision.  hcol has m + 2 entries; scs,
// ssn m + 1 each (shared).
template <typename S>
__device__ __forceinline__ void lowsync_close(const KrylovT<S>& K, int j, double* hcol, double hnext, double* scs,
                                              double* ssn) {
  GmresState* st = K.st;
  const int ldh = K.m + 1;
  double* Hj = K.H + size_t(j) * ldh;
  for (int i = threadIdx.x; i < j; i += blockDim.x) { scs[i] = K.cs[i]; ssn[i] = K.sn[i]; }
  __syncthreads();
  if (threadIdx.x == 0) {
    hcol[j + 1] = hnext;
    K.vscale[j + 1] = hnext > 0.0 ? 1.0 / hnext : 0.0;
    for (int i = 0; i < j; ++i) {
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

// Half norms of the new vector: block partials, the last block sums them into
// nrmW[j + 1], nrmS[j + 1].
template <typename S>
__device__ __forceinline__ void lowsync_half_norms(const KrylovT<S>& K, int j, double (*s_n)[kVecWarps]) {
  const int stride = cgs_stride(K.m);
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int w = 0; w < kVecWarps; ++w) { ta += s_n[0][w]; tb += s_n[1][w]; }
    K.partial[size_t(blockIdx.x) * stride + 2 * K.m + 4] = ta;
    K.partial[size_t(blockIdx.x) * stride + 2 * K.m + 5] = tb;
  }
  if (!last_block(K.ticket, K.nblocks)) return;
  if (threadIdx.x < 64) {
    const int w = threadIdx.x >> 5;
    const double t = strided_sum(K.partial + 2 * K.m + 4 + w, stride, threadIdx.x & 31, K.nblocks);
    if ((threadIdx.x & 31) == 0) (w == 0 ? K.nrmW : K.nrmS)[j + 1] = sqrt(t);
  }
}

// Sums over the blocks of partial columns [col0, col0 + cnt) and of column
// colq, one warp per sum, the warps of the whole grid sharing the work; the
// results go to hc at the same column indices (hc[col0 + i], hc[colq]).
template <typename S>
__device__ __forceinline__ void lowsync_reduce(const KrylovT<S>& K, int col0, int cnt, int colq) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int stride = cgs_stride(K.m);
  for (int c = blockIdx.x * kVecWarps + warp; c <= cnt; c += gridDim.x * kVecWarps) {
    const int col = c < cnt ? col0 + c : colq;
    const double t = strided_sum(K.partial + col, stride, lane, K.nblocks);
    if (lane == 0) K.hc[col] = t;
  }
}

// Dynamic shared memory of k_cgs_lowsync: per-warp dot totals [kVecWarps][m+1],
// coefficients h [m + 2] and c [m + 1] (FP64), update coefficients [m + 1] (A),
// rotation scratch 2 (m + 1).
template <typename S>
constexpr size_t cgs_lowsync_smem(int m) {
  return (size_t(kVecWarps) * (m + 1) + (m + 2) + (m + 1) + 2 * (m + 1)) * sizeof(double) +
         size_t(m + 1) * sizeof(typename AccOf<S>::type);
}

template <typename S>
__global__ void __launch_bounds__(kVecThreads, 2) k_cgs_lowsync(KrylovT<S> K, int half_norms) {
  using A = typename AccOf<S>::type;
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  GmresState* st = K.st;
  if (st->done) return;                     // read by every block before the closer writes it
  const int j = st->j, cnt = j + 1, m = K.m;
  const int stride = cgs_stride(m);
  extern __shared__ double sm[];
  double* s_w = sm;                                   // [kVecWarps][m + 1]
  double* s_h = s_w + size_t(kVecWarps) * (m + 1);    // [m + 2]
  double* s_c2 = s_h + (m + 2);                       // [m + 1]
  double* scs = s_c2 + (m + 1);                       // [m + 1]
  double* ssn = scs + (m + 1);                        // [m + 1]
  A* s_c = reinterpret_cast<A*>(ssn + (m + 1));       // [m + 1]
  __shared__ double s_qq[kVecWarps];
  __shared__ double s_n[2][kVecWarps];
  __shared__ double s_tot[2];                         // |q|^2 (or |q'|^2), |h|^2 (or |c|^2)
  __shared__ int s_reorth;
  S* q = K.V + size_t(j + 1) * K.ld;
  double* prow = K.partial + size_t(blockIdx.x) * stride;

  auto dots = [&]() { lowsync_dots<S, true>(K, q, cnt, s_w, m + 1, s_qq); };
  auto update = [&](bool half) {
    if (half) {
      lowsync_update<S, true>(K, q, cnt, s_c, s_n);
      lowsync_half_norms(K, j, s_n);
    } else {
      lowsync_update<S, false>(K, q, cnt, s_c, s_n);
    }
  };
  // pass 1: <q, V_i>, |q|^2
  dots();
  __syncthreads();
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < kVecWarps; ++w) t += s_w[w * (m + 1) + i];
    prow[i] = t;
  }
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kVecWarps; ++w) t += s_qq[w];
    prow[m + 1] = t;
  }
  grid.sync();
  // the cnt + 1 sums over the blocks, one warp each, spread over the grid,
  // into hc[0, cnt) and hc[m + 1]; then every block reads them back
  lowsync_reduce(K, 0, cnt, m + 1);
  grid.sync();
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) s_h[i] = __ldcg(K.hc + i) * K.vscale[i];
  if (threadIdx.x == 0) s_tot[0] = __ldcg(K.hc + m + 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    double hh = 0.0;
    for (int i = 0; i < cnt; ++i) hh += s_h[i] * s_h[i];
    s_tot[1] = hh;
    s_reorth = (s_tot[0] - hh) < 0.5 * s_tot[0] ? 1 : 0;
  }
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) s_c[i] = A(s_h[i] * K.vscale[i]);
  __syncthreads();
  // the last block closes the column (it has no rows, or as many as the
  // others, depending on the grid the autotuner picked)
  const bool closer = blockIdx.x == gridDim.x - 1;
  if (!s_reorth) {
    if (closer) lowsync_close(K, j, s_h, sqrt(s_tot[0] - s_tot[1]), scs, ssn);
    update(half_norms != 0);
    return;
  }
  // second pass (DGKS): q' = q - V h, then <q', V_i>, |q'|^2
  update(false);
  dots();
  __syncthreads();
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < kVecWarps; ++w) t += s_w[w * (m + 1) + i];
    prow[m + 2 + i] = t;
  }
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kVecWarps; ++w) t += s_qq[w];
    prow[2 * m + 3] = t;
  }
  grid.sync();
  lowsync_reduce(K, m + 2, cnt, 2 * m + 3);
  grid.sync();
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) s_c2[i] = __ldcg(K.hc + m + 2 + i) * K.vscale[i];
  if (threadIdx.x == 0) s_tot[0] = __ldcg(K.hc + 2 * m + 3);
  __syncthreads();
  if (threadIdx.x == 0) {
    double cc = 0.0;
    for (int i = 0; i < cnt; ++i) cc += s_c2[i] * s_c2[i];
    s_tot[1] = cc;
  }
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) s_c[i] = A(s_c2[i] * K.vscale[i]);
  __syncthreads();
  if (closer) {
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) s_h[i] += s_c2[i];
    __syncthreads();
    const double r2 = s_tot[0] - s_tot[1];
    lowsync_close(K, j, s_h, r2 > 0.0 ? sqrt(r2) : 0.0, scs, ssn);
  }
  update(half_norms != 0);
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
