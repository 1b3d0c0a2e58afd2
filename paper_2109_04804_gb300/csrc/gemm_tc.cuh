// BF16 GEMM on the 5th-generation tensor cores (tcgen05.mma, accumulator in
// tensor memory) with FP32 accumulation and a fused epilogue:
//   C[m][n] = sum_k A[m][k] * B[n][k]        (both operands K-contiguous, "NT")
// A: M x K row-major BF16 (lda), B: N x K row-major BF16 (ldb); the epilogue
// functor receives (m, n, acc) for every valid output element.
//
// One CTA (four warps) per 128 x 128 output tile.  K is walked in chunks of 64
// through two shared-memory stages.  One thread drives the pipeline: it loads
// a chunk of A and B with TMA (cp.async.bulk.tensor, 2-D tensor maps with
// 8 x 128 boxes: eight 16-byte K-slices of 128 rows per operand and chunk,
// which land as the no-swizzle K-major core-matrix layout of the tensor-core
// operand descriptors: 8-row x 16-byte core matrices, 128 bytes apart along
// M/N and 2048 bytes apart along K; rows and columns past the matrix edges are
// zero-filled by TMA), waits for the chunk's mbarrier transaction count,
// issues its four tcgen05.mma (M = 128, N = 128, K = 16 each) and commits them
// to the stage's second mbarrier, which the next load into that stage waits
// for; the next chunk's load is issued before the current chunk's MMAs.  The
// 128 x 128 FP32 accumulator occupies 128 tensor-memory columns (row m in lane
// m); after the last chunk every warp reads its 32 lanes (tcgen05.ld) and
// applies the epilogue.  Requirements: K, lda, ldb multiples of 8 elements
// (TMA: 16-byte aligned K coordinates and row strides), 16-byte aligned base
// pointers (checked by the host launcher).  Every wait is bounded: a wait
// that runs out sets *err, waits (bounded) for the copies and MMAs already
// issued, skips the epilogue, and the CTA still frees its tensor memory.  Used
// by the learned block preconditioner's network (Sec. 3.2.3 structure; the
// network has no counterpart in the paper).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <type_traits>

namespace hbpc {

constexpr int kTcBM = 128, kTcBN = 128, kTcKC = 64, kTcThreads = 128;
constexpr int kTcStageBytes = (kTcBM + kTcBN) * kTcKC * 2;     // one stage of A and B (32 KB)
constexpr int kTcSmem = 2 * kTcStageBytes + 64;                 // two stages, four mbarriers, TMEM slot
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

// One 8 x 128 box of a 2-D BF16 tensor map (coordinates: K element, row)
// into shared memory, completing on the mbarrier's transaction count.
__device__ __forceinline__ void tc_tma_box(uint32_t dst, const CUtensorMap* map, int k, int row, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(k), "r"(row), "r"(mbar)
      : "memory");
}

// An epilogue with kStore16 takes the 16 consecutive columns a thread reads
// from tensor memory at once (store16(m, n0, acc_bits, N)), so that it can
// write them with vector stores.
template <class Epi, class = void> struct TcStore16 { static constexpr bool value = false; };
template <class Epi> struct TcStore16<Epi, std::void_t<decltype(Epi::kStore16)>> {
  static constexpr bool value = Epi::kStore16;
};

template <class Epi>
__global__ void __launch_bounds__(kTcThreads) k_gemm_bf16_tc(const __grid_constant__ CUtensorMap ta,
                                                           const __grid_constant__ CUtensorMap tb, int M, int N, int K,
                                                           Epi epi, int* err) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(tc_smem + 2 * kTcStageBytes);   // chunk loaded, per stage
  uint64_t* done = full + 2;                                                     // chunk's MMAs done, per stage
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 2);
  __shared__ int s_ok;
  const int m0 = blockIdx.y * kTcBM, n0 = blockIdx.x * kTcBN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 4; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&full[i])));
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
  if (threadIdx.x == 0) {
    constexpr uint32_t idesc = tc_idesc(kTcBM, kTcBN);
    constexpr uint32_t lbo = 2048, sbo = 128;   // core matrices: along K, along M/N
    const int nc = (K + kTcKC - 1) / kTcKC;
    auto load = [&](int c, int s) {
      const uint32_t st = smem_u32(tc_smem + s * kTcStageBytes), mb = smem_u32(&full[s]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mb), "r"(kTcStageBytes)
                   : "memory");
      for (int g = 0; g < kTcKC / 8; ++g) {
        tc_tma_box(st + g * 2048, &ta, c * kTcKC + g * 8, m0, mb);
        tc_tma_box(st + kTcBM * kTcKC * 2 + g * 2048, &tb, c * kTcKC + g * 8, n0, mb);
      }
    };
    bool ok = true;
    int loaded = 0, waited = 0, committed = 0;   // chunks loaded, their loads waited for, MMAs committed
    load(0, 0);
    loaded = 1;
    for (int c = 0; c < nc && ok; ++c) {
      const int s = c & 1;
      if (c + 1 < nc) {   // the next chunk into the other stage, once chunk c - 1's MMAs have read it
        if (c >= 1) ok = tc_mbar_wait(smem_u32(&done[s ^ 1]), uint32_t(((c - 1) >> 1) & 1));
        if (!ok) break;
        load(c + 1, s ^ 1);
        loaded = c + 2;
      }
      ok = tc_mbar_wait(smem_u32(&full[s]), uint32_t((c >> 1) & 1));
      if (!ok) break;
      waited = c + 1;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t sa = smem_u32(tc_smem + s * kTcStageBytes), sb = sa + kTcBM * kTcKC * 2;
#pragma unroll
      for (int kk = 0; kk < kTcKC; kk += 16) {
        const uint64_t ad = tc_desc(sa + (kk / 8) * 2048, lbo, sbo);
        const uint64_t bd = tc_desc(sb + (kk / 8) * 2048, lbo, sbo);
        const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(&done[s]))
                   : "memory");
      committed = c + 1;
    }
    // the last commit completes after every MMA of this CTA
    if (ok && nc > 0) ok = tc_mbar_wait(smem_u32(&done[(nc - 1) & 1]), uint32_t(((nc - 1) >> 1) & 1));
    if (!ok) {
      // drain (bounded) what is still in flight before the CTA releases its memory
      for (int c = waited; c < loaded; ++c) tc_mbar_wait(smem_u32(&full[c & 1]), uint32_t((c >> 1) & 1));
      if (committed > 0)
        tc_mbar_wait(smem_u32(&done[(committed - 1) & 1]), uint32_t(((committed - 1) >> 1) & 1));
      atomicExch(err, 1);
    }
    s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (s_ok) {
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
        if constexpr (TcStore16<Epi>::value) {
          epi.store16(m, n0 + col, r, N);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int n = n0 + col + j;
            if (n < N) epi(m, n, __uint_as_float(r[j]));
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTcCols));
}

// Host: the 2-D tensor map of a K-contiguous BF16 matrix (rows x K, row
// stride ld elements) with the kernel's 8 x 128 box; false if the driver's
// encoder is unavailable or rejects the layout.
inline bool tc_tensor_map(CUtensorMap* map, const __nv_bfloat16* base, int K, int rows, int ld) {
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Encode encode = []() -> Encode {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<Encode>(f);
  }();
  if (!encode) return false;
  const cuuint64_t dims[2] = {cuuint64_t(K), cuuint64_t(rows)};
  const cuuint64_t strides[1] = {cuuint64_t(ld) * 2};
  const cuuint32_t box[2] = {8, cuuint32_t(kTcBM)};
  const cuuint32_t estr[2] = {1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace hbpc
