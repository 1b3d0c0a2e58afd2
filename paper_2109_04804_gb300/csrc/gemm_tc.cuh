// BF16 GEMM on the 5th-generation tensor cores (tcgen05.mma, accumulator in
// tensor memory) with FP32 accumulation and a fused epilogue:
//   C[m][n] = sum_k A[m][k] * B[n][k]        (both operands K-contiguous, "NT")
// A: M x K row-major BF16 (lda), B: N x K row-major BF16 (ldb); the epilogue
// functor receives (m, n, acc) for every valid output element.
//
// One CTA (four warps) per 128 x 128 output tile.  K is walked in chunks of 64
// through two shared-memory stages: all threads copy a chunk of A and B into
// the canonical no-swizzle K-major layout of the tensor-core operand
// descriptors (8-row x 16-byte core matrices; along K 128 bytes apart, along
// M/N 1024 bytes apart), then one thread issues the chunk's four
// tcgen05.mma (M = 128, N = 128, K = 16 each) and commits them to the stage's
// mbarrier, which the copy into that stage waits for two chunks later.  The
// 128 x 128 FP32 accumulator occupies 128 tensor-memory columns (row m in lane
// m); after the last chunk every warp reads its 32 lanes (tcgen05.ld) and
// applies the epilogue.  Requirements: K, lda, ldb multiples of 8 elements,
// 16-byte aligned base pointers (checked by the host launcher).  Every wait
// is bounded: a wait that runs out sets *err, skips the epilogue and the CTA
// still frees its tensor memory.  Used by the learned block preconditioner's
// network (Sec. 3.2.3 structure; the network has no counterpart in the paper).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace hbpc {

constexpr int kTcBM = 128, kTcBN = 128, kTcKC = 64, kTcThreads = 128;
constexpr int kTcStageBytes = (kTcBM + kTcBN) * kTcKC * 2;     // one stage of A and B (32 KB)
constexpr int kTcSmem = 2 * kTcStageBytes + 64;                 // two stages, mbarriers, TMEM slot
constexpr uint32_t kTcCols = 128;                               // tensor-memory columns (FP32 accumulator)
constexpr long long kTcWaitLimit = 1ll << 24;                   // polls of an mbarrier before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor of a no-swizzle K-major operand: start
// address, leading-dimension (K) and stride-dimension (M/N) byte offsets of
// the core matrices (all >> 4), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = uint64_t((saddr >> 4) & 0x3FFFu);
  d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ bool tc_mbar_wait(uint32_t addr, uint32_t parity) {
  for (long long i = 0; i < kTcWaitLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Copy chunk [k0, k0 + 64) of rows [r0, r0 + 128) of a K-contiguous matrix
// into the core-matrix layout at s (zero past the matrix edges).
__device__ __forceinline__ void tc_load_chunk(unsigned char* s, const __nv_bfloat16* g, int ld, int nrows, int K,
                                              int r0, int k0) {
  for (int c = threadIdx.x; c < 128 * (kTcKC / 8); c += kTcThreads) {
    const int r = c / (kTcKC / 8), kc = c - r * (kTcKC / 8);
    const int gr = r0 + r, gk = k0 + kc * 8;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (gr < nrows && gk < K) v = *reinterpret_cast<const uint4*>(g + size_t(gr) * ld + gk);
    *reinterpret_cast<uint4*>(s + (r >> 3) * (kTcKC / 8) * 128 + kc * 128 + (r & 7) * 16) = v;
  }
}

template <class Epi>
__global__ void __launch_bounds__(kTcThreads) k_gemm_bf16_tc(const __nv_bfloat16* __restrict__ A, int lda,
                                                           const __nv_bfloat16* __restrict__ B, int ldb, int M,
                                                           int N, int K, Epi epi, int* err) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(tc_smem + 2 * kTcStageBytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tc_smem + 2 * kTcStageBytes + 16);
  const int m0 = blockIdx.y * kTcBM, n0 = blockIdx.x * kTcBN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "r"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = tc_idesc(kTcBM, kTcBN);
  constexpr uint32_t lbo = 128, sbo = (kTcKC / 8) * 128;
  const int nc = (K + kTcKC - 1) / kTcKC;
  bool ok = true;
  for (int c = 0; c < nc && ok; ++c) {
    const int s = c & 1;
    // the stage's previous MMAs (chunk c - 2) have read it (the outcome is
    // made uniform over the CTA before anyone leaves the loop)
    if (c >= 2) ok = tc_mbar_wait(smem_u32(&mbar[s]), uint32_t(((c - 2) >> 1) & 1));
    ok = __syncthreads_and(ok) != 0;
    if (!ok) break;
    unsigned char* stg = tc_smem + s * kTcStageBytes;
    tc_load_chunk(stg, A, lda, M, K, m0, c * kTcKC);
    tc_load_chunk(stg + kTcBM * kTcKC * 2, B, ldb, N, K, n0, c * kTcKC);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t sa = smem_u32(stg), sb = smem_u32(stg + kTcBM * kTcKC * 2);
#pragma unroll
      for (int kk = 0; kk < kTcKC; kk += 16) {
        const uint64_t ad = tc_desc(sa + kk * 16, lbo, sbo);
        const uint64_t bd = tc_desc(sb + kk * 16, lbo, sbo);
        const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(&mbar[s]))
                   : "memory");
    }
  }
  // the last commit completes after every MMA of this CTA
  if (ok && nc > 0) ok = tc_mbar_wait(smem_u32(&mbar[(nc - 1) & 1]), uint32_t(((nc - 1) >> 1) & 1));
  ok = __syncthreads_and(ok) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (ok) {
    const int row = warp * 32 + lane;
    const int m = m0 + row;
#pragma unroll 1
    for (int col = 0; col < kTcBN; col += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + (uint32_t(warp * 32) << 16) + uint32_t(col);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
          "[%16];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (m < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + col + j;
          if (n < N) epi(m, n, __uint_as_float(r[j]));
        }
      }
    }
  } else if (threadIdx.x == 0) {
    atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTcCols));
}

}  // namespace hbpc
