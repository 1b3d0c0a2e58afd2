// BJ_ext kernels that do not depend on the conservation law: S = I - c1 J +
// c2 J^2, the batched Gauss-Jordan inverse and the apply P^-1 (Sec. 3.2.3).
// Included by exactly one translation unit.
#pragma once
#include "bjext.cuh"

namespace hbpc {

// S = I - c1 J + c2 J^2 for one element per block (J staged in shared memory),
// written to `S` (same layout), in T (FP64, or FP32 for the mixed-precision
// mode, where the blocks only precondition).  Dynamic shared memory: nb * nb T.
//
// Hall (BJ^H_ext): the Hessian blocks, S = I - c1 J + c2 (H + J^2); may be
// the same buffer as Sall (each entry is read once, before it is written).
template <typename T>
__global__ void __launch_bounds__(256) k_pc_form_S(const T* __restrict__ Jall, T* Sall, int nb,
                                                   int nE, const double* c12, const int* only = nullptr,
                                                   const T* Hall = nullptr) {
  const int e = blockIdx.x;
  if (e >= nE || (only && !only[e])) return;   // only: the elements flagged for an exact block
  extern __shared__ __align__(16) unsigned char sJ_raw[];
  T* sJ = reinterpret_cast<T*>(sJ_raw);
  const T* J = Jall + size_t(e) * nb * nb;
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) sJ[t] = J[t];
  __syncthreads();
  const T c1 = T(c12[0]), c2 = T(c12[1]);
  T* S = Sall + size_t(e) * nb * nb;
  const T* H = Hall ? Hall + size_t(e) * nb * nb : nullptr;
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int c = t / nb, r = t - c * nb;          // entry (r, c)
    T jj = H ? H[t] : T(0);
    for (int k = 0; k < nb; ++k) jj += sJ[k * nb + r] * sJ[c * nb + k];   // (J J)(r, c)
    S[t] = (r == c ? T(1) : T(0)) - c1 * sJ[t] + c2 * jj;
  }
}

// In-place inverse of one n_b x n_b block per thread block by Gauss-Jordan
// elimination with partial (row) pivoting; the column exchanges implied by the
// row pivots are undone at the end.  A zero pivot leaves the block unchanged and
// sets *singular (the preconditioner is then skipped by the host).
// Dynamic shared memory: (nb * nb + nb) T + nb ints.
template <typename T>
__global__ void __launch_bounds__(256) k_pc_invert(T* __restrict__ Mall, int nb, int nE, int* singular,
                                                   const int* only = nullptr) {
  const int e = blockIdx.x;
  if (e >= nE || (only && !only[e])) return;
  extern __shared__ __align__(16) unsigned char inv_raw[];
  T* A = reinterpret_cast<T*>(inv_raw);   // column-major nb x nb
  T* colk = A + nb * nb;                  // copy of the pivot column
  int* perm = reinterpret_cast<int*>(colk + nb);
  __shared__ int s_piv;
  __shared__ int s_bad;
  T* M = Mall + size_t(e) * nb * nb;
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) A[t] = M[t];
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  for (int k = 0; k < nb; ++k) {
    // pivot: largest |A(i, k)|, i >= k (warp 0)
    if (threadIdx.x < 32) {
      T best = T(-1);
      int bi = k;
      for (int i = k + threadIdx.x; i < nb; i += 32) {
        const T a = fabs(A[k * nb + i]);
        if (a > best) { best = a; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) {
        s_piv = bi;
        perm[k] = bi;
        if (!(best > T(0))) s_bad = 1;
      }
    }
    __syncthreads();
    if (s_bad) break;
    const int p = s_piv;
    if (p != k)
      for (int c = threadIdx.x; c < nb; c += blockDim.x) {
        const T t = A[c * nb + k];
        A[c * nb + k] = A[c * nb + p];
        A[c * nb + p] = t;
      }
    __syncthreads();
    const T inv = T(1) / A[k * nb + k];
    for (int i = threadIdx.x; i < nb; i += blockDim.x) colk[i] = A[k * nb + i];
    __syncthreads();
    // row k scaled; column k becomes e_k scaled
    for (int c = threadIdx.x; c < nb; c += blockDim.x) A[c * nb + k] = (c == k ? T(1) : A[c * nb + k]) * inv;
    __syncthreads();
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
      const int c = t / nb, i = t - c * nb;
      if (i == k) continue;
      const T f = colk[i];
      const T rk = A[c * nb + k];
      A[t] = (c == k ? T(0) : A[t]) - f * rk;
    }
    __syncthreads();
  }
  if (s_bad) {
    if (threadIdx.x == 0) atomicExch(singular, 1);
    return;
  }
  // undo the column interchanges in reverse order
  for (int k = nb - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k)
      for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const T t = A[k * nb + i];
        A[k * nb + i] = A[p * nb + i];
        A[p * nb + i] = t;
      }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) M[t] = A[t];
}

// Verification of learned blocks: for every element, one Rademacher probe x
// (SplitMix64 of seed and row), u = S x = x - c1 J x + c2 J (J x), and
// r = M~ u - x.  flag[e] = |r|^2 > tau^2 |x|^2: the block does not map S x
// near x and gets the exact inverse instead; count += flagged elements.
// EPB elements per block, one thread per row (the apply's layout).
// Dynamic shared memory: epb * 3 * nb values of S.
__device__ __forceinline__ unsigned long long pc_mix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

template <typename S>
__global__ void __launch_bounds__(256) k_pc_verify(const S* __restrict__ M, const S* __restrict__ J, int nb, int nE,
                                                   const double* c12, unsigned long long seed, double tau,
                                                   int* __restrict__ flag, int* __restrict__ count) {
  const int epb = blockDim.x / nb;
  const int le = threadIdx.x / nb, r = threadIdx.x - le * nb;
  const int e = blockIdx.x * epb + le;
  const bool live = le < epb && e < nE;
  extern __shared__ double vf_raw[];
  S* sm = reinterpret_cast<S*>(vf_raw);
  S* sx = sm + le * 3 * nb;
  S* sy = sx + nb;
  S* su = sy + nb;
  if (live) sx[r] = (pc_mix64(seed * 0x100000001B3ull + size_t(e) * nb + r) >> 63) ? S(1) : S(-1);
  __syncthreads();
  const S* Je = J + size_t(live ? e : 0) * nb * nb;
  if (live) {
    S y = S(0);
    for (int c = 0; c < nb; ++c) y += Je[size_t(c) * nb + r] * sx[c];
    sy[r] = y;
  }
  __syncthreads();
  if (live) {
    S z = S(0);
    for (int c = 0; c < nb; ++c) z += Je[size_t(c) * nb + r] * sy[c];
    su[r] = sx[r] - S(c12[0]) * sy[r] + S(c12[1]) * z;
  }
  __syncthreads();
  double rr = 0.0;
  if (live) {
    const S* Me = M + size_t(e) * nb * nb;
    S t = S(0);
    for (int c = 0; c < nb; ++c) t += Me[size_t(c) * nb + r] * su[c];
    const double d = double(t) - double(sx[r]);
    rr = d * d;
  }
  // per-element sum over its nb rows (the rows of one element are consecutive threads)
  __shared__ double s_rows[256];
  s_rows[threadIdx.x] = rr;
  __syncthreads();
  if (live && r == 0) {
    double tt = 0.0;
    for (int k = 0; k < nb; ++k) tt += s_rows[le * nb + k];
    const int bad = tt > tau * tau * double(nb) ? 1 : 0;
    flag[e] = bad;
    if (bad) atomicAdd(count, 1);
  }
}

// Row r of the column-major n_b x n_b block A times x (shared memory): four
// columns' loads in flight, the sum in column order.
template <typename S>
__device__ __forceinline__ S pc_row_dot(const S* __restrict__ A, int nb, int r, const S* x) {
  S y = S(0);
  int c = 0;
  for (; c + 3 < nb; c += 4) {
    const S a0 = A[size_t(c) * nb + r], a1 = A[size_t(c + 1) * nb + r];
    const S a2 = A[size_t(c + 2) * nb + r], a3 = A[size_t(c + 3) * nb + r];
    y += a0 * x[c];
    y += a1 * x[c + 1];
    y += a2 * x[c + 2];
    y += a3 * x[c + 3];
  }
  for (; c < nb; ++c) y += A[size_t(c) * nb + r] * x[c];
  return y;
}

// The norms of the apply's result (total, W half, S half) through the last
// block, when the caller asked for them (a.zn); aw, as: this thread's squares.
template <typename S>
__device__ __forceinline__ void pc_apply_norms(const PcApplyT<S>& a, const Krylov& K, double aw, double as) {
  if (!a.zn) return;   // norms only needed by the difference-quotient Jv
  __shared__ double s2[2][kVecWarps];
  aw = warp_sum(aw);
  as = warp_sum(as);
  if ((threadIdx.x & 31) == 0) { s2[0][threadIdx.x >> 5] = aw; s2[1][threadIdx.x >> 5] = as; }
  __syncthreads();
  const int stride = K.m + 3;
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) { ta += s2[0][w]; tb += s2[1][w]; }
    K.partial[size_t(blockIdx.x) * stride + 0] = ta;
    K.partial[size_t(blockIdx.x) * stride + 1] = tb;
  }
  if (!last_block(K.ticket, gridDim.x)) return;
  __shared__ double rr[2];
  reduce_partials(K.partial, stride, gridDim.x, 2, rr);
  __syncthreads();
  if (threadIdx.x == 0 && a.zn) {
    a.zn[0] = sqrt(rr[0] + rr[1]);
    a.zn[1] = sqrt(rr[0]);
    a.zn[2] = sqrt(rr[1]);
  }
}

template <typename S>
__global__ void __launch_bounds__(256) k_pc_apply(PcApplyT<S> a, Krylov K) {
  if (a.skip && *a.skip) return;
  const int nb = a.nb;
  const int epb = blockDim.x / nb;
  const int le = threadIdx.x / nb, r = threadIdx.x - le * nb;
  const int e = blockIdx.x * epb + le;
  const bool live = le < epb && e < a.nE;
  extern __shared__ double sm_raw[];
  S* sm = reinterpret_cast<S*>(sm_raw);
  S* xw = sm + le * 4 * nb;
  S* xs = xw + nb;
  S* su = xs + nb;
  S* sv = su + nb;
  const size_t off = (a.jidx ? size_t(*a.jidx) * a.ld : 0) + size_t(e) * nb;
  const S sc = S(a.scale ? (a.jidx ? a.scale[*a.jidx] : *a.scale) : 1.0);
  if (live) {
    xw[r] = sc * a.xW[off + r];
    xs[r] = sc * a.xS[off + r];
  }
  __syncthreads();
  if (a.hess) {   // BJ^H_ext (uniform over the block): t = w - c2 J s, u = M t
    const S* Me = a.M + size_t(live ? e : 0) * nb * nb;
    const S* Je = a.J + size_t(live ? e : 0) * nb * nb;
    if (live) sv[r] = xw[r] - S(a.c12[1]) * pc_row_dot(Je, nb, r, xs);
    __syncthreads();
    if (live) su[r] = pc_row_dot(Me, nb, r, sv);
    __syncthreads();
    double aw = 0.0, as = 0.0;
    if (live) {
      S top = su[r];
      S bot = pc_row_dot(Je, nb, r, su) + xs[r];
      const size_t o = size_t(e) * nb + r;
      if (a.accumulate) { top += a.oW[o]; bot += a.oS[o]; }
      a.oW[o] = top;
      a.oS[o] = bot;
      aw = double(top * top);
      as = double(bot * bot);
    }
    pc_apply_norms(a, K, aw, as);
    return;
  }
  S u = S(0), v = S(0);
  if (live) {
    const S* Me = a.M + (a.shared ? size_t(0) : size_t(e) * nb * nb);
    int c = 0;
    for (; c + 3 < nb; c += 4) {   // four columns' loads in flight, sums in column order
      const S m0 = Me[size_t(c) * nb + r], m1 = Me[size_t(c + 1) * nb + r];
      const S m2 = Me[size_t(c + 2) * nb + r], m3 = Me[size_t(c + 3) * nb + r];
      u += m0 * xw[c]; v += m0 * xs[c];
      u += m1 * xw[c + 1]; v += m1 * xs[c + 1];
      u += m2 * xw[c + 2]; v += m2 * xs[c + 2];
      u += m3 * xw[c + 3]; v += m3 * xs[c + 3];
    }
    for (; c < nb; ++c) {
      const S m = Me[size_t(c) * nb + r];
      u += m * xw[c];
      v += m * xs[c];
    }
    su[r] = u;
    sv[r] = v;
  }
  __syncthreads();
  double aw = 0.0, as = 0.0;
  if (live) {
    const S* Je = a.J + (a.shared ? size_t(0) : size_t(e) * nb * nb);
    S ju = S(0), jv = S(0);
    int c = 0;
    for (; c + 3 < nb; c += 4) {
      const S j0 = Je[size_t(c) * nb + r], j1 = Je[size_t(c + 1) * nb + r];
      const S j2 = Je[size_t(c + 2) * nb + r], j3 = Je[size_t(c + 3) * nb + r];
      ju += j0 * su[c]; jv += j0 * sv[c];
      ju += j1 * su[c + 1]; jv += j1 * sv[c + 1];
      ju += j2 * su[c + 2]; jv += j2 * sv[c + 2];
      ju += j3 * su[c + 3]; jv += j3 * sv[c + 3];
    }
    for (; c < nb; ++c) {
      const S j = Je[size_t(c) * nb + r];
      ju += j * su[c];
      jv += j * sv[c];
    }
    const S c1 = S(a.c12[0]), c2 = S(a.c12[1]);
    S top = u - c2 * jv;
    S bot = ju + v - c1 * jv;
    const size_t o = size_t(e) * nb + r;
    if (a.accumulate) { top += a.oW[o]; bot += a.oS[o]; }
    a.oW[o] = top;
    a.oS[o] = bot;
    aw = double(top * top);
    as = double(bot * bot);
  }
  pc_apply_norms(a, K, aw, as);
}

// The element Jacobian of linear advection (with or without its viscous term)
// on a Cartesian element acts along each direction separately: J = sum_m
// I (x) .. (x) A_m (x) .. (x) I, one p x p factor A_m per direction m (the 1-D
// operator of Eq. 12 along x_m, its own-trace face terms included).  This
// kernel (one block) reads the factors off the assembled dense J_0 (column-
// major, node index i_0 + p i_1 + p^2 i_2): off-diagonal entries of A_m from
// the line through node 0 along x_m, diagonals split as A_0(i, i) = J(i, i)
// and A_m(i, i) = J(i p^m, i p^m) - J(0, 0) for m > 0.  It then rebuilds every
// entry of J_0 from the factors and sets *ok only if all agree with the
// assembled block to rounding (tol times max |J_0|), so the apply falls back
// to the dense J_0 for anything that is not a Kronecker sum.
template <typename T>
__global__ void __launch_bounds__(256) k_pc_kron_factors(const T* __restrict__ J, int nb, int P, int dim, T tol,
                                                         T* __restrict__ A, int* ok) {
  __shared__ T sA[3 * 8 * 8];
  __shared__ T s_red[2][256 / 32];
  const int pp = P * P;
  for (int t = threadIdx.x; t < dim * pp; t += blockDim.x) {
    const int m = t / pp, i = (t / P) % P, l = t % P;
    int st = 1;
    for (int k = 0; k < m; ++k) st *= P;
    T a = J[size_t(l * st) * nb + size_t(i * st)];
    if (i == l && m > 0) a -= J[0];
    sA[t] = a;
    A[t] = a;
  }
  __syncthreads();
  T dmax = T(0), jmax = T(0);
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int c = t / nb, r = t - c * nb;
    int rr = r, cc = c;
    int rd[3] = {0, 0, 0}, cd[3] = {0, 0, 0};
    for (int m = 0; m < dim; ++m) { rd[m] = rr % P; rr /= P; cd[m] = cc % P; cc /= P; }
    T rec = T(0);
    for (int m = 0; m < dim; ++m) {
      bool same = true;
      for (int k = 0; k < dim; ++k)
        if (k != m && rd[k] != cd[k]) same = false;
      if (same) rec += sA[m * pp + rd[m] * P + cd[m]];
    }
    const T jv = J[t];
    dmax = fmax(dmax, fabs(rec - jv));
    jmax = fmax(jmax, fabs(jv));
  }
  for (int o = 16; o > 0; o >>= 1) {
    dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    jmax = fmax(jmax, __shfl_xor_sync(0xffffffffu, jmax, o));
  }
  if ((threadIdx.x & 31) == 0) { s_red[0][threadIdx.x >> 5] = dmax; s_red[1][threadIdx.x >> 5] = jmax; }
  __syncthreads();
  if (threadIdx.x == 0) {
    T d = T(0), jm = T(0);
    for (int w = 0; w < int(blockDim.x >> 5); ++w) { d = fmax(d, s_red[0][w]); jm = fmax(jm, s_red[1][w]); }
    *ok = (d <= tol * jm) ? 1 : 0;
  }
}

// P^-1 with one block for all elements (PcApplyT::shared): the same algebra as
// k_pc_apply, organised as the small dense products they are.  M and J live in
// shared memory; a thread owns row r of EG elements, so every loaded entry of M
// and J is used for 2 EG multiply-adds, and the elements' inputs are staged with
// the EG elements of a group interleaved (one vector load per column).  The
// block covers (blockDim.x / n_b) groups.  No norms (callers with a.zn use
// k_pc_apply).  Dynamic shared memory: (2 n_b^2 + 4 EG n_b groups) S.
template <typename S, int EG>
__global__ void __launch_bounds__(256) k_pc_apply_shared(PcApplyT<S> a) {
  if (a.skip && *a.skip) return;
  const int nb = a.nb;
  const int groups = blockDim.x / nb;
  const int g = threadIdx.x / nb, r = threadIdx.x - g * nb;
  const bool live_t = g < groups;
  extern __shared__ double sh_raw[];
  S* sM = reinterpret_cast<S*>(sh_raw);
  S* sJ = sM + nb * nb;
  S* X = sJ + nb * nb;                        // [groups][nb][EG] xw, then xs, u, v
  const int gsz = nb * EG;
  S* Xw = X;
  S* Xs = Xw + groups * gsz;
  S* U = Xs + groups * gsz;
  S* Vv = U + groups * gsz;
  // J as Kronecker factors when they reproduce it (k_pc_kron_factors), kept
  // in the sJ slot
  const bool kron = a.kron && *a.kron_ok;
  S* const sK = sJ;
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) sM[t] = a.M[t];
  if (kron)
    for (int t = threadIdx.x; t < a.dim * a.P * a.P; t += blockDim.x) sK[t] = a.kron[t];
  else
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) sJ[t] = a.J[t];
  const long long e0 = (long long)blockIdx.x * groups * EG;   // first element of the block
  const size_t off = (a.jidx ? size_t(*a.jidx) * a.ld : 0);
  const S sc = S(a.scale ? (a.jidx ? a.scale[*a.jidx] : *a.scale) : 1.0);
  // stage the block's inputs (contiguous in memory), interleaving the EG
  // elements of each group
  const int nvals = groups * EG * nb;
  for (int t = threadIdx.x; t < nvals; t += blockDim.x) {
    const long long e = e0 + t / nb;
    const int c = t % nb;
    const int le = t / nb, gg = le / EG, k = le - gg * EG;
    S w = S(0), z = S(0);
    if (e < a.nE) {
      w = sc * a.xW[off + size_t(e) * nb + c];
      z = sc * a.xS[off + size_t(e) * nb + c];
    }
    Xw[gg * gsz + c * EG + k] = w;
    Xs[gg * gsz + c * EG + k] = z;
  }
  __syncthreads();
  S u[EG], v[EG];
#pragma unroll
  for (int k = 0; k < EG; ++k) { u[k] = S(0); v[k] = S(0); }
  if (live_t) {
    const S* xw = Xw + g * gsz;
    const S* xs = Xs + g * gsz;
    for (int c = 0; c < nb; ++c) {
      const S m = sM[c * nb + r];
#pragma unroll
      for (int k = 0; k < EG; ++k) { u[k] += m * xw[c * EG + k]; v[k] += m * xs[c * EG + k]; }
    }
#pragma unroll
    for (int k = 0; k < EG; ++k) { U[g * gsz + r * EG + k] = u[k]; Vv[g * gsz + r * EG + k] = v[k]; }
  }
  __syncthreads();
  if (!live_t) return;
  S ju[EG], jv[EG];
#pragma unroll
  for (int k = 0; k < EG; ++k) { ju[k] = S(0); jv[k] = S(0); }
  const S* su = U + g * gsz;
  const S* sv = Vv + g * gsz;
  if (kron) {
    // J as a Kronecker sum: along each direction m the p values of row r's
    // line through x_m (d p multiply-adds per row instead of n_b)
    const int P = a.P;
    int st = 1, rr = r;
    for (int m = 0; m < a.dim; ++m) {
      const int im = rr % P;
      rr /= P;
      const int b0 = r - im * st;
      const S* Arow = sK + (m * P + im) * P;
      for (int l = 0; l < P; ++l) {
        const S am = Arow[l];
        const int c = b0 + l * st;
#pragma unroll
        for (int k = 0; k < EG; ++k) { ju[k] += am * su[c * EG + k]; jv[k] += am * sv[c * EG + k]; }
      }
      st *= P;
    }
  } else {
    for (int c = 0; c < nb; ++c) {
      const S j = sJ[c * nb + r];
#pragma unroll
      for (int k = 0; k < EG; ++k) { ju[k] += j * su[c * EG + k]; jv[k] += j * sv[c * EG + k]; }
    }
  }
  const S c1 = S(a.c12[0]), c2 = S(a.c12[1]);
#pragma unroll
  for (int k = 0; k < EG; ++k) {
    const long long e = e0 + g * EG + k;
    if (e >= a.nE) break;
    S top = u[k] - c2 * jv[k];
    S bot = ju[k] + v[k] - c1 * jv[k];
    const size_t o = size_t(e) * nb + r;
    if (a.accumulate) { top += a.oW[o]; bot += a.oS[o]; }
    a.oW[o] = top;
    a.oS[o] = bot;
  }
}

// FP64 -> FP32 copy (mixed precision: basis, linearisation point, PC blocks)
__global__ void k_to_float(const double* __restrict__ x, float* __restrict__ y, size_t n, double scale) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    y[i] = float(scale * x[i]);
}

// y (FP64) += x (FP32)
__global__ void k_add_float(const float* __restrict__ x, double* __restrict__ y, size_t n) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    y[i] += double(x[i]);
}

// out (FP32) = -g (FP64) - jx (FP32): restart residual of the mixed mode
__global__ void k_neg_sum_f(const double* __restrict__ g, const float* __restrict__ jx, float* __restrict__ out,
                            size_t n) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    out[i] = float(-g[i]) - jx[i];
}

}  // namespace hbpc
