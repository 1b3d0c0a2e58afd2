// BF16 tensor-core GEMM with FP32 accumulation and a fused epilogue:
//   C[m][n] = sum_k A[m][k] * B[n][k]        (both operands K-contiguous, "NT")
// A: M x K row-major BF16 (lda), B: N x K row-major BF16 (ldb); the epilogue
// functor receives (m, n, acc) for every valid output element.
//
// Block tile 128 x 64 x 32, four warps (2 x 2), each warp 64 x 32 built from
// mma.sync.m16n8k16 BF16 instructions; global -> shared copies with cp.async
// (16 bytes, zero fill past the matrix edge), two stages.  Requirements: K, lda,
// ldb multiples of 8 elements and 16-byte aligned base pointers (checked by the
// host launcher).  Used by the learned block preconditioner's network.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace hbpc {

constexpr int kGemmBM = 128, kGemmBN = 64, kGemmBK = 32;
constexpr int kGemmPad = 8;                       // bf16 padding per smem row
constexpr int kGemmLd = kGemmBK + kGemmPad;       // 40 bf16 = 80 bytes per row
constexpr int kGemmThreads = 128;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ __forceinline__ uint32_t lds32(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

__device__ __forceinline__ void mma_bf16_16816(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Copy one K-slab (rows [r0, r0+ROWS) of a K-contiguous matrix, columns
// [k0, k0+32)) into shared memory; out-of-range chunks are zero filled.
template <int ROWS>
__device__ __forceinline__ void gemm_load_tile(__nv_bfloat16* s, const __nv_bfloat16* g, int ld, int nrows,
                                               int K, int r0, int k0) {
  // ROWS x 32 bf16 = ROWS x 4 chunks of 16 bytes
  for (int c = threadIdx.x; c < ROWS * 4; c += kGemmThreads) {
    const int r = c >> 2, kc = (c & 3) * 8;
    const int gr = r0 + r, gk = k0 + kc;
    const bool valid = gr < nrows && gk < K;
    const __nv_bfloat16* src = valid ? g + size_t(gr) * ld + gk : g;
    cp_async16(s + r * kGemmLd + kc, src, valid);
  }
}

template <class Epi>
__global__ void __launch_bounds__(kGemmThreads) k_gemm_bf16_nt(const __nv_bfloat16* __restrict__ A, int lda,
                                                             const __nv_bfloat16* __restrict__ B, int ldb,
                                                             int M, int N, int K, Epi epi) {
  __shared__ __align__(16) __nv_bfloat16 sA[2][kGemmBM * kGemmLd];
  __shared__ __align__(16) __nv_bfloat16 sB[2][kGemmBN * kGemmLd];
  const int m0 = blockIdx.y * kGemmBM, n0 = blockIdx.x * kGemmBN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp >> 1) * 64, wn = (warp & 1) * 32;   // warp tile origin in the block tile
  const int g = lane >> 2, t = lane & 3;
  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
  const int nk = (K + kGemmBK - 1) / kGemmBK;
  gemm_load_tile<kGemmBM>(sA[0], A, lda, M, K, m0, 0);
  gemm_load_tile<kGemmBN>(sB[0], B, ldb, N, K, n0, 0);
  cp_async_commit();
  for (int kt = 0; kt < nk; ++kt) {
    const int cur = kt & 1;
    cp_async_wait_all();
    __syncthreads();
    if (kt + 1 < nk) {
      gemm_load_tile<kGemmBM>(sA[cur ^ 1], A, lda, M, K, m0, (kt + 1) * kGemmBK);
      gemm_load_tile<kGemmBN>(sB[cur ^ 1], B, ldb, N, K, n0, (kt + 1) * kGemmBK);
    }
    cp_async_commit();
    const __nv_bfloat16* a_s = sA[cur];
    const __nv_bfloat16* b_s = sB[cur];
#pragma unroll
    for (int kk = 0; kk < kGemmBK; kk += 16) {
      uint32_t af[4][4], bf[4][2];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = wm + i * 16 + g;
        af[i][0] = lds32(a_s + r * kGemmLd + kk + t * 2);
        af[i][1] = lds32(a_s + (r + 8) * kGemmLd + kk + t * 2);
        af[i][2] = lds32(a_s + r * kGemmLd + kk + 8 + t * 2);
        af[i][3] = lds32(a_s + (r + 8) * kGemmLd + kk + 8 + t * 2);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n = wn + j * 8 + g;
        bf[j][0] = lds32(b_s + n * kGemmLd + kk + t * 2);
        bf[j][1] = lds32(b_s + n * kGemmLd + kk + 8 + t * 2);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16_16816(acc[i][j], af[i], bf[j]);
    }
  }
  cp_async_wait_all();
  // epilogue: acc[i][j] = rows (g, g + 8) of m16 tile i, cols (2t, 2t + 1) of n8 tile j
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int m = m0 + wm + i * 16 + g + (r >= 2 ? 8 : 0);
        const int n = n0 + wn + j * 8 + t * 2 + (r & 1);
        if (m < M && n < N) epi(m, n, acc[i][j][r]);
      }
}

}  // namespace hbpc
