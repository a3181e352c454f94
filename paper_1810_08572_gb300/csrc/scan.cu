// Exclusive prefix sum of int32 counts (active-set compaction, CSR offsets).
// Three launches: per-block scan with block totals, scan of the totals in
// one block, add-back.  Deterministic (integer).
#include "scan.cuh"

namespace fvs {

static constexpr int SB = 1024;  // elements per block (one per thread)

__global__ void k_scan_block(int64_t n, const int32_t* __restrict__ in, int32_t* __restrict__ out,
                             int32_t* __restrict__ bsum) {
  __shared__ int32_t sh[32];
  const int64_t i = blockIdx.x * (int64_t)SB + threadIdx.x;
  const int32_t v = i < n ? in[i] : 0;
  // warp inclusive scan
  int32_t x = v;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    int32_t t = sh[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    sh[lane] = t;
  }
  __syncthreads();
  const int32_t incl = x + (w > 0 ? sh[w - 1] : 0);
  if (i < n) out[i] = incl - v;
  if (threadIdx.x == SB - 1) bsum[blockIdx.x] = incl;
}

__global__ void k_scan_sums(int nb, int32_t* __restrict__ bsum, int32_t* __restrict__ total) {
  // one block; sequential chunks per thread, then a block scan of chunk sums
  __shared__ int32_t sh[1024];
  const int per = (nb + blockDim.x - 1) / blockDim.x;
  const int lo = threadIdx.x * per, hi = min(nb, lo + per);
  int32_t s = 0;
  for (int i = lo; i < hi; ++i) s += bsum[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t acc = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      const int32_t x = sh[t];
      sh[t] = acc;
      acc += x;
    }
    *total = acc;
  }
  __syncthreads();
  int32_t acc = sh[threadIdx.x];
  for (int i = lo; i < hi; ++i) {
    const int32_t x = bsum[i];
    bsum[i] = acc;
    acc += x;
  }
}

__global__ void k_scan_add(int64_t n, int32_t* __restrict__ out, const int32_t* __restrict__ bsum) {
  const int64_t i = blockIdx.x * (int64_t)SB + threadIdx.x;
  if (i < n) out[i] += bsum[blockIdx.x];
}

fvs_status ScanWork::ensure(int64_t n) {
  const int64_t nb = (n + SB - 1) / SB + 1;
  FVS_TRY(bsum.alloc((size_t)nb));
  FVS_TRY(total.alloc(1));
  return FVS_OK;
}

fvs_status exclusive_scan(cudaStream_t s, ScanWork& w, int64_t n, const int32_t* in, int32_t* out) {
  FVS_TRY(w.ensure(n));
  if (n == 0) {
    FVS_CUDA(cudaMemsetAsync(w.total.p, 0, sizeof(int32_t), s));
    return FVS_OK;
  }
  const int nb = (int)((n + SB - 1) / SB);
  k_scan_block<<<nb, SB, 0, s>>>(n, in, out, w.bsum); FVS_COUNT_LAUNCH();
  k_scan_sums<<<1, 1024, 0, s>>>(nb, w.bsum, w.total); FVS_COUNT_LAUNCH();
  k_scan_add<<<nb, SB, 0, s>>>(n, out, w.bsum); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

}  // namespace fvs
