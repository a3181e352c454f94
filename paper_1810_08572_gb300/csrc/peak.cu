// Measured FP64 FMA rate of the GPU: the second roof of the FP64 sparse
// kernels (one fused multiply-add per 12 bytes of an ELL row).  Not part of
// the method; the benchmark reports its kernels against this figure and the
// copy bandwidth.
#include "common.cuh"

#define FVS_API extern "C" __attribute__((visibility("default")))

namespace fvs {

// eight independent FMA chains per thread keep the FP64 pipe fed; the result
// is written so the chains cannot be removed
__global__ void k_fma_chains(int64_t iters, double m, double c, double* out) {
  double a[8];
  for (int k = 0; k < 8; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == 12345.678) out[0] = s;   // never true for these inputs; keeps the work
}

}  // namespace fvs

using namespace fvs;

FVS_API fvs_status fvs_measure_fp64_fma(int64_t iters, double* gflops) {
  if (!gflops || iters <= 0) {
    set_error("fvs_measure_fp64_fma: bad argument");
    return FVS_ERR_ARG;
  }
  cudaStream_t st = nullptr;
  FVS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double* out = nullptr;
  fvs_status r = FVS_OK;
  const int blocks = sm_count() * 8, threads = 256;
  float ms = 0.f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      cudaMallocAsync((void**)&out, sizeof(double), st) != cudaSuccess) {
    set_error("fvs_measure_fp64_fma: CUDA set-up failed");
    r = FVS_ERR_CUDA;
  } else {
    k_fma_chains<<<blocks, threads, 0, st>>>(iters / 10 + 1, 0.9999999, 1e-7, out);   // warm-up
    FVS_COUNT_LAUNCH();
    cudaEventRecord(e0, st);
    k_fma_chains<<<blocks, threads, 0, st>>>(iters, 0.9999999, 1e-7, out);
    FVS_COUNT_LAUNCH();
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      set_error("fvs_measure_fp64_fma: %s", cudaGetErrorString(cudaGetLastError()));
      r = FVS_ERR_CUDA;
    }
  }
  if (out) cudaFreeAsync(out, st);
  cudaStreamSynchronize(st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  if (r != FVS_OK) return r;
  *gflops = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3) / 1e9;
  return FVS_OK;
}
