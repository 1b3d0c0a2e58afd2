// FP64 arithmetic throughput probe: the denominator of the ALU roofline of the
// FP64 kernels (the measured HBM copy bandwidth is the other denominator).
// Independent FMA chains per thread, many resident warps per SM.
#include <cuda_runtime.h>

#include "../../include/hbpc.h"

namespace {
constexpr int kChains = 8;

__global__ void k_fma_chains(double* out, int iters, double a, double b) {
  double acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = double(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  out[size_t(blockIdx.x) * blockDim.x + threadIdx.x] = s;
}
}  // namespace

extern "C" hbpc_status hbpc_fp64_fma_peak(double* gflops) {
  if (!gflops) return HBPC_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HBPC_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HBPC_ERR_CUDA;
  const int blocks = sms * 8, threads = 256, iters = 4000;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * size_t(blocks) * threads) != cudaSuccess) return HBPC_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    k_fma_chains<<<blocks, threads>>>(out, iters, 1.0000001, 1e-9);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return HBPC_ERR_CUDA;
  *gflops = 2.0 * kChains * double(iters) * blocks * threads / (best * 1e-3) / 1e9;
  return HBPC_OK;
}
