// BJ_ext apply of the shared block in FP64 on the tensor cores.
//
// For a state- and element-independent element Jacobian (linear advection on
// one uniform mesh) every element's BJ_ext inverse (Sec. 3.2.3) is the same
// 2 n_b x 2 n_b matrix acting on the element's (w, sigma):
//   [top; bot] = P [w; sigma],  P = [[M, -c2 J M], [J M, M - c1 J M]],
//   M = (I - c1 J + c2 J^2)^-1,
// i.e. the apply is one dense product P X with X holding one element per
// column.  GB300 executes FP64 at 1/64 of the FP32 rate, and the CUDA-core
// apply spends ~3,500 FP64 multiply-adds per element; here the product runs
// on the BF16 tensor cores with FP32 accumulation, exactly, by splitting
// both operands into integer digit planes (the error-free splitting of Ozaki,
// Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59, 2012):
//
//   * every row p of P and every column e of X is scaled by a power of two
//     taken from its largest entry and truncated to a signed integer of at
//     most 62 bits (x = T 2^(E - 1084), E the largest biased exponent of the
//     column; entries within 2^-9 of the largest are represented exactly);
//   * each integer is written as eight balanced base-256 digits in
//     [-128, 127] (top digit |d_0| <= 65), each exact in BF16;
//   * the products of digit planes a, b are summed per level L = a + b in one
//     FP32 tensor-memory accumulator: a level holds at most 8 plane pairs, so
//     its sum is bounded by 8 * 80 * 2^14 < 2^24 for 2 n_b <= 80 (2^24 for
//     2 n_b = 128) and is an exact integer;
//   * levels 0..8 are kept (the dropped pairs weigh below 2^-69 of
//     max|P_p| max|x_e| 2 n_b) and combined in 64-bit integers,
//     Q = Qhi 2^40 + Qlo, y = Q 2^(E_P + E_X - 2120) times the input's
//     scale factor, rounded once, all in integer operations (no FP64
//     instruction per output, instead of 2 n_b multiply-adds).
//
// The result differs from the FP64 CUDA-core product by rounding only (one
// rounding of the exact integer sum plus the truncation of entries more than
// 2^9 below their column's or row's largest).  A column or row holding Inf or
// NaN gives NaN outputs.
//
// P's digit planes are formed once per preconditioner build
// (k_pc_tc_planes), already in the shared-memory image of the tensor-core
// operand: no-swizzle K-major core matrices (8 rows x 16 bytes), 128 bytes
// apart along the rows and R * 16 bytes apart along K (R = 2 n_b rounded up
// to 8).  The apply (k_pc_apply_tc) stages them with one bulk copy per CTA
// (cp.async.bulk, completing on an mbarrier) while its 512 threads load 32
// elements' inputs with coalesced loads and split them into X's digit
// planes; four threads issue the 43 plane-pair products (tcgen05.mma,
// M = 128 rows of P, N = 32 elements, K = 16 per instruction; the levels
// split between them) into 9 x 32 tensor-memory columns, and 16 warps read
// them back (tcgen05.ld; a warp's rows are its quarter of the lanes, its
// columns 8 of the 32 elements) and combine the levels.  Every wait is
// bounded; a wait that runs out writes NaN outputs (the Krylov loop then
// stops with a non-finite residual) and sets *err.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "gemm_tc.cuh"

namespace hbpc {

constexpr int kPtcDigits = 8;      // balanced base-256 digits per value
constexpr int kPtcLevels = 9;      // levels a + b = 0..8 kept
constexpr int kPtcElems = 32;      // elements per CTA (the MMA's N)
constexpr int kPtcThreads = 512;   // 16 warps: warp w reads lanes 32 (w % 4) .. of columns 8 (w / 4) ..
constexpr uint32_t kPtcCols = 512; // tensor-memory columns allocated (9 x 32 used)
constexpr int kPtcIssuers = 4;     // threads issuing the tensor-core products
constexpr int kPtcPad = 2048;      // the M = 128 operand reads rows up to 127 past the last plane

// Sizes of the digit planes for n_b: K = 2 n_b rounded up to 16 (the MMA's K
// step), R = 2 n_b rounded up to 8 (rows of P stored).
struct PtcDims {
  int nb, K, R;
  __host__ __device__ PtcDims(int nb_) : nb(nb_), K(((2 * nb_ + 15) / 16) * 16), R(((2 * nb_ + 7) / 8) * 8) {}
  __host__ __device__ size_t a_plane() const { return size_t(K / 8) * R * 16; }
  __host__ __device__ size_t b_plane() const { return size_t(K / 8) * kPtcElems * 16; }
  __host__ __device__ size_t a_bytes() const { return kPtcDigits * a_plane(); }
  __host__ __device__ size_t x_bytes() const { return size_t(kPtcElems) * 2 * nb * sizeof(double); }
  __host__ __device__ size_t smem() const { return a_bytes() + kPtcPad + kPtcDigits * b_plane() + x_bytes() + 64; }
};

// Split a finite FP64 value into a signed integer T of at most 62 bits
// relative to the largest biased exponent E of its row or column
// (x = T 2^(E - 1084)), then into balanced base-256 digits (top first) as
// BF16 bit patterns h[0] .. h[7].  Adding 128 to each of the seven low bytes
// makes every low digit plus 128 a plain byte (no carries), so a digit is a
// byte extract; the top digit is the top byte, signed (|d_0| <= 65).  A digit
// d in [-256, 256] becomes BF16 through the exact FP32 difference
// (2^23 + 256 + d) - (2^23 + 256), whose low 16 bits are zero.
__device__ __forceinline__ void ptc_digit_bits(double v, int E, uint32_t* h) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(v));
  const int ex = int((bits >> 52) & 0x7FF);
  const unsigned long long frac = bits & ((1ull << 52) - 1);
  const long long mant = (long long)(ex ? (frac | (1ull << 52)) : frac);
  const int sh = (ex ? ex : 1) - E + 9;   // <= 9: mant < 2^53 -> |T| < 2^62
  long long T = sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> (-sh)) : 0);
  if (bits >> 63) T = -T;
  const unsigned long long Tp = static_cast<unsigned long long>(T) + 0x0080808080808080ull;
  const uint32_t lo = uint32_t(Tp), hi = uint32_t(Tp >> 32);
  const int top = int(static_cast<signed char>(hi >> 24));
  h[0] = __float_as_uint(__int_as_float(0x4B000000 + 256 + top) - 8388864.0f) >> 16;
#pragma unroll
  for (int b = 1; b < kPtcDigits; ++b) {
    const int byte = 7 - b;   // digit b sits in byte 7 - b
    const uint32_t u = byte >= 4 ? (hi >> (8 * (byte - 4))) & 0xFFu : (lo >> (8 * byte)) & 0xFFu;
    h[b] = __float_as_uint(__int_as_float(0x4B000000 + 128 + int(u)) - 8388864.0f) >> 16;
  }
}

// The biased exponent used for the scaling (1 for zeros and subnormals).
__device__ __forceinline__ int ptc_exp(double v) {
  const int ex = int((static_cast<unsigned long long>(__double_as_longlong(v)) >> 52) & 0x7FF);
  return ex ? ex : 1;
}

// Byte offset of (row, k) in a no-swizzle K-major plane whose K groups are
// lbo bytes apart.
__device__ __forceinline__ uint32_t ptc_off(int row, int k, int lbo) {
  return uint32_t((k >> 3) * lbo + (row >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// P's rows (one block per stored row p < R) and their digit planes.  M and J
// are the shared block's n_b x n_b matrices, column-major (entry (r, c) at
// c * n_b + r); c12 = (c1, c2) on the device.  planes: kPtcDigits planes of
// a_plane() bytes; pexp[p]: the row's largest biased exponent (0x7FF: the row
// holds Inf or NaN).
__global__ void __launch_bounds__(128) k_pc_tc_planes(const double* __restrict__ M, const double* __restrict__ J,
                                                       int nb, const double* __restrict__ c12,
                                                       __nv_bfloat16* __restrict__ planes, int* __restrict__ pexp) {
  const PtcDims D(nb);
  const int p = blockIdx.x;
  extern __shared__ double s_row[];   // [2 nb]: row p of P, then [nb]: row r of J M
  double* s_jm = s_row + 2 * nb;
  __shared__ int s_e;
  const int n2 = 2 * nb;
  const bool live = p < n2;
  const int r = p < nb ? p : p - nb;
  const double c1 = c12[0], c2 = c12[1];
  if (live)
    for (int c = threadIdx.x; c < nb; c += blockDim.x) {
      double t = 0.0;
      for (int k = 0; k < nb; ++k) t = fma(J[size_t(k) * nb + r], M[size_t(c) * nb + k], t);
      s_jm[c] = t;
    }
  __syncthreads();
  if (live)
    for (int c = threadIdx.x; c < nb; c += blockDim.x) {
      const double m = M[size_t(c) * nb + r], jm = s_jm[c];
      if (p < nb) { s_row[c] = m; s_row[nb + c] = -c2 * jm; }
      else { s_row[c] = jm; s_row[nb + c] = m - c1 * jm; }
    }
  if (threadIdx.x == 0) s_e = 1;
  __syncthreads();
  int e = 1;
  if (live)
    for (int k = threadIdx.x; k < n2; k += blockDim.x) e = max(e, ptc_exp(s_row[k]));
  atomicMax(&s_e, e);
  __syncthreads();
  const int E = s_e;
  if (threadIdx.x == 0) pexp[p] = E;
  unsigned char* base = reinterpret_cast<unsigned char*>(planes);
  const int lbo = D.R * 16;
  for (int k = threadIdx.x; k < D.K; k += blockDim.x) {
    uint32_t h[kPtcDigits];
    ptc_digit_bits(live && k < n2 && E != 0x7FF ? s_row[k] : 0.0, E == 0x7FF ? 1 : E, h);
    const uint32_t o = ptc_off(p, k, lbo);
#pragma unroll
    for (int a = 0; a < kPtcDigits; ++a)
      *reinterpret_cast<unsigned short*>(base + a * D.a_plane() + o) = static_cast<unsigned short>(h[a]);
  }
}

// The FP64 value (-1)^neg m 2^sh sc_m 2^sc_e rounded once to nearest (m != 0;
// sc_m: the scale's 53-bit significand at bits 63..11), formed with integer
// operations only (GB300's FP64 pipe is the narrow one).  Returns false when
// the result leaves the normal range (the caller then takes the FP64 route).
__device__ __forceinline__ bool ptc_finish(unsigned long long m, int sh, bool neg, unsigned long long sc_m, int sc_e,
                                           double* out) {
  const int lz = __clzll(m);
  m <<= lz;
  sh -= lz;                                        // m * 2^sh, bit 63 set
  unsigned long long hi = __umul64hi(m, sc_m), lo = m * sc_m;
  int e = sh + sc_e + 64;                          // hi * 2^e + lo * 2^(e - 64)
  if (!(hi >> 63)) {
    hi = (hi << 1) | (lo >> 63);
    lo <<= 1;
    e -= 1;
  }
  unsigned long long mant = hi >> 11;              // 53 bits; value = mant 2^(e + 11)
  const bool rb = (hi >> 10) & 1ull, rest = ((hi & 0x3FFull) | lo) != 0ull;
  if (rb && (rest || (mant & 1ull))) {
    mant += 1ull;
    if (mant >> 53) { mant >>= 1; e += 1; }
  }
  const int be = e + 63 + 1023;
  if (be < 1 || be > 2046) return false;
  *out = __longlong_as_double((long long)(((unsigned long long)neg << 63) | ((unsigned long long)be << 52) |
                                          (mant & ((1ull << 52) - 1))));
  return true;
}

// out (+)= P (scale * in) for every element: in = (xW, xS) (n_b values per
// element each, column jidx of stride ld when jidx is given), out = (oW, oS).
struct PcApplyTc {
  const __nv_bfloat16* planes; const int* pexp;
  const double* xW; const double* xS;
  const double* scale; const int* jidx; size_t ld;
  double* oW; double* oS;
  const int* skip;
  int accumulate;
  int nb, nE;
  int* err;
};

__global__ void __launch_bounds__(kPtcThreads, 1) k_pc_apply_tc(PcApplyTc a) {
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(1024) unsigned char ptc_smem[];
  const PtcDims D(a.nb);
  const int nb = a.nb, n2 = 2 * nb;
  unsigned char* sP = ptc_smem;
  unsigned char* sX = ptc_smem + D.a_bytes() + kPtcPad;
  double* sXd = reinterpret_cast<double*>(sX + kPtcDigits * D.b_plane());            // [32][2 n_b] inputs
  uint64_t* bars = reinterpret_cast<uint64_t*>(sXd + kPtcElems * n2);                // [0] P copied, [1] MMAs done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);
  __shared__ int s_ex[kPtcElems];
  __shared__ int s_ok, s_fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long e0 = (long long)blockIdx.x * kPtcElems;
  if (threadIdx.x == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bars[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&bars[1])), "r"(kPtcIssuers));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "r"(kPtcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t abytes = uint32_t(D.a_bytes());
  if (threadIdx.x == 0) {   // P's planes: one bulk copy (sizes and addresses multiples of 16)
    const uint32_t mb = smem_u32(&bars[0]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mb), "r"(abytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(sP)),
                 "l"(reinterpret_cast<uint64_t>(a.planes)), "r"(abytes), "r"(mb)
                 : "memory");
  }
  // the tile's inputs (32 elements x (w, sigma)), coalesced, into shared
  // memory: sXd[j][k], k < n_b from xW, n_b <= k < 2 n_b from xS
  {
    const size_t off = a.jidx ? size_t(*a.jidx) * a.ld : 0;
    const long long nlive = a.nE - e0 < kPtcElems ? a.nE - e0 : kPtcElems;
    const int nv = kPtcElems * nb;
    const double* gw = a.xW + off + size_t(e0) * nb;
    const double* gs = a.xS + off + size_t(e0) * nb;
#pragma unroll 4
    for (int t = threadIdx.x; t < nv; t += kPtcThreads) {
      const int j = t / nb, c = t - j * nb;
      const bool live = j < nlive;
      sXd[j * n2 + c] = live ? gw[t] : 0.0;
      sXd[j * n2 + nb + c] = live ? gs[t] : 0.0;
    }
  }
  __syncthreads();
  // X's digit planes: 16 threads per element, pairs of entries (2i, 2i + 1)
  // for i = q, q + 16, ... (zero past 2 n_b), one 4-byte store per plane and pair
  {
    const int j = threadIdx.x >> 4, q = threadIdx.x & 15;
    const double* xr = sXd + j * n2;
    int E = 1;
    for (int k = q; k < n2; k += 16) E = max(E, ptc_exp(xr[k]));
#pragma unroll
    for (int w = 1; w < 16; w <<= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, w));
    if (q == 0) s_ex[j] = E;
    const int lbo = kPtcElems * 16;
    for (int i = q; i < D.K / 2; i += 16) {
      uint32_t h0[kPtcDigits], h1[kPtcDigits];
      const int k = 2 * i;
      const bool fin = E != 0x7FF;   // a column with Inf or NaN: zero digits, NaN outputs
      const double v0 = fin && k < n2 ? xr[k] : 0.0, v1 = fin && k + 1 < n2 ? xr[k + 1] : 0.0;
      ptc_digit_bits(v0, fin ? E : 1, h0);
      ptc_digit_bits(v1, fin ? E : 1, h1);
      const uint32_t o = ptc_off(j, k, lbo);
#pragma unroll
      for (int b = 0; b < kPtcDigits; ++b)
        *reinterpret_cast<uint32_t*>(sX + b * D.b_plane() + o) = h0[b] | (h1[b] << 16);
    }
  }
  // the generic-proxy stores above are read by the tensor cores (async proxy)
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  __syncthreads();
  // the plane-pair products: lane 0 of warps 0..3 each issues the levels
  // L = i, i + 4, ... (13, 8, 10 and 12 of the 43 pairs; independent
  // accumulators, so the issue order between them does not matter) and
  // commits them to bars[1], which completes after the four commits
  if (lane == 0 && warp < kPtcIssuers) {
    bool ok = tc_mbar_wait(smem_u32(&bars[0]), 0);
    if (ok) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      constexpr uint32_t idesc = tc_idesc(128, kPtcElems);
      const uint32_t alb = uint32_t(D.R * 16), blb = uint32_t(kPtcElems * 16);
      // descriptors of plane 0, K step 0; a plane or K step moves the start
      // address field (address >> 4) by its byte offset >> 4
      const uint64_t ad0 = tc_desc(smem_u32(sP), alb, 128), bd0 = tc_desc(smem_u32(sX), blb, 128);
      const uint64_t astep = uint64_t(2 * alb) >> 4, bstep = uint64_t(2 * blb) >> 4;
      const int nks = D.K / 16;
      for (int L = warp; L < kPtcLevels; L += kPtcIssuers) {
        uint32_t acc = 0;
        const int a0 = L > kPtcDigits - 1 ? L - (kPtcDigits - 1) : 0;
        const int a1 = L < kPtcDigits - 1 ? L : kPtcDigits - 1;
        const uint32_t dcol = tmem + uint32_t(L * kPtcElems);
        for (int pa = a0; pa <= a1; ++pa) {
          uint64_t ad = ad0 + (uint64_t(pa * D.a_plane()) >> 4);
          uint64_t bd = bd0 + (uint64_t((L - pa) * D.b_plane()) >> 4);
          for (int ks = 0; ks < nks; ++ks) {
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            acc = 1;
            ad += astep;
            bd += bstep;
          }
        }
      }
    } else {
      s_fail = 1;
      tc_mbar_wait(smem_u32(&bars[0]), 0);   // the copy still in flight (bounded)
    }
    // committed also after a failed wait (nothing issued: it arrives at once)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_u32(&bars[1]))
                 : "memory");
    if (warp == 0) {
      const bool done = tc_mbar_wait(smem_u32(&bars[1]), 0);
      if (!done) tc_mbar_wait(smem_u32(&bars[1]), 0);   // the products still in flight (bounded)
      s_ok = done ? 1 : 0;
    }
  }
  __syncthreads();
  const bool ok_all = s_ok && !s_fail;
  if (threadIdx.x == 0 && !ok_all) atomicExch(a.err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  // warp w: rows p = 32 (w % 4) + lane of P (its tensor-memory lanes), the 8
  // elements 8 (w / 4) ..; the nine level loads in flight before one wait
  const int lq = warp & 3, cg = warp >> 2;
  const int p = lq * 32 + lane;
  const double sc = a.scale ? (a.jidx ? a.scale[*a.jidx] : *a.scale) : 1.0;
  // the scale as significand and exponent for ptc_finish (a zero, subnormal
  // or non-finite scale takes the FP64 route)
  const unsigned long long scb = static_cast<unsigned long long>(__double_as_longlong(sc));
  const int sce = int((scb >> 52) & 0x7FF);
  const bool sc_int = sce != 0 && sce != 0x7FF;
  const unsigned long long sc_m = ((scb & ((1ull << 52) - 1)) | (1ull << 52)) << 11;
  const int sc_e = sce - 1023 - 63;
  const bool sc_neg = (scb >> 63) != 0;
  if (lq * 32 < n2) {
    long long qh[8], ql[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) { qh[j] = 0; ql[j] = 0; }
    if (ok_all) {
      uint32_t v[kPtcLevels][8];
#pragma unroll
      for (int L = 0; L < kPtcLevels; ++L) {
        const uint32_t taddr = tmem + (uint32_t(lq * 32) << 16) + uint32_t(L * kPtcElems + cg * 8);
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                     : "=r"(v[L][0]), "=r"(v[L][1]), "=r"(v[L][2]), "=r"(v[L][3]), "=r"(v[L][4]), "=r"(v[L][5]),
                       "=r"(v[L][6]), "=r"(v[L][7])
                     : "r"(taddr));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        int D[kPtcLevels];
#pragma unroll
        for (int L = 0; L < kPtcLevels; ++L) D[L] = __float2int_rn(__uint_as_float(v[L][j]));
        qh[j] = (long long)D[0] * 16777216ll + (long long)D[1] * 65536ll + (long long)D[2] * 256ll + D[3];
        ql[j] = ((long long)D[4] << 32) + (long long)D[5] * 16777216ll + (long long)D[6] * 65536ll +
                (long long)D[7] * 256ll + D[8];
      }
    }
    if (p < n2) {
      const int EP = a.pexp[p];
      double* out = p < nb ? a.oW : a.oS;
      const int r = p < nb ? p : p - nb;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = cg * 8 + j;
        const long long e = e0 + c;
        if (e >= a.nE) break;
        const int EX = s_ex[c];
        double y;
        if (!ok_all || EX == 0x7FF || EP == 0x7FF) {
          y = __longlong_as_double(0x7FF8000000000000ll);
        } else {
          // Q = Qhi 2^40 + Qlo exactly as a 128-bit integer (|Q| < 2^84), its
          // leading 64 bits with a sticky bit for the rest converted once
          // (correct rounding), the powers of two added to the exponent field
          const unsigned long long alo = (unsigned long long)qh[j] << 40;
          unsigned long long lo = alo + (unsigned long long)ql[j];
          long long hi = (qh[j] >> 24) + (ql[j] >> 63) + (lo < alo ? 1 : 0);
          const bool neg = hi < 0;
          if (neg) {
            lo = ~lo + 1ull;
            hi = ~hi + (lo == 0ull ? 1 : 0);
          }
          unsigned long long m = lo;
          int sh = EP + EX - 2120;
          if (hi != 0) {
            const int lz = __clzll(hi);   // hi < 2^20: 44 <= lz <= 63
            m = ((unsigned long long)hi << lz) | (lo >> (64 - lz)) | ((lo << lz) != 0ull ? 1ull : 0ull);
            sh += 64 - lz;
          }
          if (m == 0ull) {
            y = 0.0 * sc;
          } else if (!(sc_int && ptc_finish(m, sh, neg != sc_neg, sc_m, sc_e, &y))) {
            y = ldexp(__ull2double_rn(m), sh);
            if (neg) y = -y;
            y *= sc;
          }
        }
        const size_t o = size_t(e) * nb + r;
        if (a.accumulate) y += out[o];
        out[o] = y;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kPtcCols));
}

}  // namespace hbpc
