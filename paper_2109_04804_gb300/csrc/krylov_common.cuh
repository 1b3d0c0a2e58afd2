// Device-side GMRES state, Krylov basis description and the deterministic
// reduction helpers shared by the Krylov and preconditioner kernels.
//
// Reductions are deterministic: every block writes its partial sums, the last
// block to finish (atomic ticket, no waiting) adds them in block order with a
// fixed shuffle tree.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace hbpc {

constexpr int kVecThreads = 256;
constexpr int kVecWarps = kVecThreads / 32;
constexpr int kRows = 4;            // rows of a vector per thread and tile
constexpr int kTile = kVecThreads * kRows;

struct GmresState {
  int j;             // columns built in this cycle
  int done;          // cycle finished
  int converged;     // residual target met
  int reorth;        // current column needs a second Gram-Schmidt pass
  int its;           // iterations of this solve
  int max_its;
  int m;             // restart length
  int breakdown;
  double target;     // absolute target on the residual norm
  double resid;      // current residual norm estimate |g_j|
  double qq;         // ||q||^2 before orthogonalisation
  double nrm[3];     // scratch norms of the last norm-producing kernel (total, W, S)
};

// All pointers are device memory.  V holds m+1 columns of length n2 at stride
// ld; column i represents v_i = vscale[i] * V_i.  nrmW/nrmS are the norms of the
// unscaled halves of V_i (first `half` entries are W, the rest sigma).  S is the
// storage type of the basis (double, or float in the mixed-precision mode).
template <typename S>
struct KrylovT {
  S* V; size_t ld, n2, half;
  int m;
  double* H;        // (m+1) x m, column-major, ldh = m+1
  double* cs; double* sn; double* g;
  double* vscale; double* nrmW; double* nrmS;
  double* hc;       // Gram-Schmidt coefficients of the two passes: [0, m+2) and [m+2, 2m+4)
  double* y;        // solution coefficients (times vscale), length m
  GmresState* st;
  double* partial;  // nblocks x (m+3)
  unsigned* ticket;
  int nblocks;
};
using Krylov = KrylovT<double>;

// Accumulation type of per-thread sums over a basis of storage type S: FP64
// for an FP64 basis; FP32 for an FP32 basis (the per-warp sums are then added
// in FP64 across warps and blocks).
template <typename S> struct AccOf { using type = double; };
template <> struct AccOf<float> { using type = float; };

template <typename A>
__device__ __forceinline__ A warp_sum(A x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Warp-wide sum of p[b * stride] for b = 0 .. n-1 (lane handles b = lane,
// lane + 32, ..; four independent accumulators keep four loads in flight);
// every lane returns the total.  The order is fixed, so every block that
// reduces the same data gets the same value.
__device__ __forceinline__ double strided_sum(const double* p, int stride, int lane, int n) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int b = lane;
  for (; b + 96 < n; b += 128) {
    a0 += __ldcg(p + size_t(b) * stride);
    a1 += __ldcg(p + size_t(b + 32) * stride);
    a2 += __ldcg(p + size_t(b + 64) * stride);
    a3 += __ldcg(p + size_t(b + 96) * stride);
  }
  for (; b < n; b += 32) a0 += __ldcg(p + size_t(b) * stride);
  return warp_sum((a0 + a1) + (a2 + a3));
}

// Dot products of this thread's kRows values x (rows base + r kVecThreads,
// valid where in[r]) with columns [0, cnt) of V (stride ld), warp-reduced;
// lane 0 stores (ACC: adds) the warp's sum of column i at s_red[i kVecWarps +
// warp].  Four columns per step, so that 4 kRows independent loads are in
// flight (the sums of every column keep their order).
template <bool ACC, typename S, typename A, typename R>
__device__ __forceinline__ void col_dots(const S* V, size_t ld, size_t base, const A* x, const bool* in, int cnt,
                                         R* s_red) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int i = 0;
  for (; i + 3 < cnt; i += 4) {
    A v[4][kRows];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int r = 0; r < kRows; ++r)
        v[c][r] = in[r] ? A(V[size_t(i + c) * ld + base + size_t(r) * kVecThreads]) : A(0);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      A a = A(0);
#pragma unroll
      for (int r = 0; r < kRows; ++r) a += x[r] * v[c][r];
      a = warp_sum(a);
      if (lane == 0) {
        if (ACC) s_red[(i + c) * kVecWarps + warp] += R(a);
        else s_red[(i + c) * kVecWarps + warp] = R(a);
      }
    }
  }
  for (; i < cnt; ++i) {
    A a = A(0);
#pragma unroll
    for (int r = 0; r < kRows; ++r)
      if (in[r]) a += x[r] * A(V[size_t(i) * ld + base + size_t(r) * kVecThreads]);
    a = warp_sum(a);
    if (lane == 0) {
      if (ACC) s_red[i * kVecWarps + warp] += R(a);
      else s_red[i * kVecWarps + warp] = R(a);
    }
  }
}

// x[r] -= sum_i c[i] V_i(row) over columns [0, cnt) with coefficients already
// in the accumulation type (no FP64 work in the loop), ascending i.
template <typename S, typename A>
__device__ __forceinline__ void col_axpy_c(const S* V, size_t ld, size_t base, A* x, const bool* in, int cnt,
                                           const A* c) {
  int i = 0;
  for (; i + 3 < cnt; i += 4) {
    A v[4][kRows];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int r = 0; r < kRows; ++r)
        v[k][r] = in[r] ? A(V[size_t(i + k) * ld + base + size_t(r) * kVecThreads]) : A(0);
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int r = 0; r < kRows; ++r) x[r] -= c[i + k] * v[k][r];
  }
  for (; i < cnt; ++i)
#pragma unroll
    for (int r = 0; r < kRows; ++r)
      if (in[r]) x[r] -= c[i] * A(V[size_t(i) * ld + base + size_t(r) * kVecThreads]);
}

// x[r] -= sum_i c_i V_i(row) over columns [0, cnt), c_i = coef[i] (times
// scale[i] when scale is given), in ascending i; four columns' loads per step.
template <typename S, typename A>
__device__ __forceinline__ void col_axpy(const S* V, size_t ld, size_t base, A* x, const bool* in, int cnt,
                                         const double* coef, const double* scale) {
  int i = 0;
  for (; i + 3 < cnt; i += 4) {
    A v[4][kRows];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int r = 0; r < kRows; ++r)
        v[c][r] = in[r] ? A(V[size_t(i + c) * ld + base + size_t(r) * kVecThreads]) : A(0);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const A cc = A(scale ? coef[i + c] * scale[i + c] : coef[i + c]);
#pragma unroll
      for (int r = 0; r < kRows; ++r) x[r] -= cc * v[c][r];
    }
  }
  for (; i < cnt; ++i) {
    const A cc = A(scale ? coef[i] * scale[i] : coef[i]);
#pragma unroll
    for (int r = 0; r < kRows; ++r)
      if (in[r]) x[r] -= cc * A(V[size_t(i) * ld + base + size_t(r) * kVecThreads]);
  }
}

// Last-block election: returns true in every thread of the last block to
// arrive.  Partials written before must be visible (threadfence first).
__device__ __forceinline__ bool last_block(unsigned* ticket, int nblocks) {
  __shared__ unsigned s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(ticket, 1u);
    s_last = (t == unsigned(nblocks - 1)) ? 1u : 0u;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    if (threadIdx.x == 0) *ticket = 0u;   // reset for the next reduction
  }
  return s_last != 0u;
}

// Deterministic cross-block sum of partial[b * stride + c] for c in [0, cnt):
// warp w of the block's warps sums columns c = w, w + warps, ..; lanes stride
// over blocks.  The block may have any whole number of warps (the block
// preconditioner's apply runs with as few as one).
__device__ __forceinline__ void reduce_partials(const double* partial, int stride, int nblocks,
                                                int cnt, double* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int warps = int(blockDim.x >> 5);
  for (int c = warp; c < cnt; c += warps) {
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += __ldcg(partial + size_t(b) * stride + c);
    s = warp_sum(s);
    if (lane == 0) out[c] = s;
  }
}

__device__ __forceinline__ void chunk_range(size_t n, int nblocks, size_t& lo, size_t& hi) {
  const size_t chunk = ((n + nblocks - 1) / nblocks + 31) & ~size_t(31);
  lo = size_t(blockIdx.x) * chunk;
  hi = lo + chunk < n ? lo + chunk : n;
  if (lo > n) lo = n;
}

}  // namespace hbpc
