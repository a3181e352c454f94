// Shared helpers of the fvs CUDA library: error plumbing, device buffers,
// small device utilities.  Every host function that can fail returns an
// fvs_status and records a message; nothing aborts or traps.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "../../include/fvs.h"

namespace fvs {

void set_error(const char* fmt, ...);

#define FVS_TRY(expr)                  \
  do {                                 \
    fvs_status _s = (expr);            \
    if (_s != FVS_OK) return _s;       \
  } while (0)

#define FVS_CUDA(expr)                                                              \
  do {                                                                              \
    cudaError_t _e = (expr);                                                        \
    if (_e != cudaSuccess) {                                                        \
      ::fvs::set_error("%s:%d %s: %s", __FILE__, __LINE__, #expr, cudaGetErrorString(_e)); \
      return _e == cudaErrorMemoryAllocation ? FVS_ERR_NOMEM : FVS_ERR_CUDA;         \
    }                                                                               \
  } while (0)

#define FVS_LAUNCH_CHECK() FVS_CUDA(cudaGetLastError())

// every kernel launch of the library bumps this process-wide counter
extern unsigned long long g_launches;
#define FVS_COUNT_LAUNCH() __atomic_add_fetch(&::fvs::g_launches, 1ULL, __ATOMIC_RELAXED)

// Stream-ordered allocation: buffers are allocated and freed on the stream
// of the object being worked on (set by the entry points), so concurrent
// solvers on different streams never synchronise the whole device through
// cudaFree.
extern thread_local cudaStream_t g_alloc_stream;
struct AllocStream {
  cudaStream_t prev;
  explicit AllocStream(cudaStream_t s) : prev(g_alloc_stream) { g_alloc_stream = s; }
  ~AllocStream() { g_alloc_stream = prev; }
};

// Owning device buffer (freed on destruction).
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFreeAsync(p, g_alloc_stream);
    p = nullptr;
    n = 0;
  }
  fvs_status alloc(size_t count) {
    if (count <= n && p) return FVS_OK;
    release();
    if (count == 0) return FVS_OK;
    cudaError_t e = cudaMallocAsync((void**)&p, count * sizeof(T), g_alloc_stream);
    if (e != cudaSuccess) {
      p = nullptr;
      set_error("cudaMallocAsync of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? FVS_ERR_NOMEM : FVS_ERR_CUDA;
    }
    n = count;
    return FVS_OK;
  }
  fvs_status zero(cudaStream_t s) {
    if (!p) return FVS_OK;
    cudaError_t e = cudaMemsetAsync(p, 0, n * sizeof(T), s);
    if (e != cudaSuccess) {
      set_error("cudaMemsetAsync: %s", cudaGetErrorString(e));
      return FVS_ERR_CUDA;
    }
    return FVS_OK;
  }
  operator T*() const { return p; }
};

inline int grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 2147483647LL) g = 2147483647;
  return (int)g;
}

// Persistent-style grids: a multiple of the SM count for grid-stride loops.
int sm_count();
inline int stride_grid(int64_t n, int block, int per_sm = 8) {
  int64_t want = (n + block - 1) / block;
  int64_t cap = (int64_t)sm_count() * per_sm;
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  return (int)want;
}

// ---------------------------------------------------------------------------
// device utilities
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum of one double per thread; result valid in thread 0.
// blockDim.x must be a multiple of 32 and at most 1024.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0) v = warp_sum(v);
  __syncthreads();
  return v;
}
__device__ __forceinline__ double block_max(double v, double* sh) {
  v = warp_max(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : -1.0e300;
  if (w == 0) v = warp_max(v);
  __syncthreads();
  return v;
}

// One ELL row, acc + sum_k val[k*n + i] x[col[k*n + i]] in slot order: the
// matrix streams through once per product, so its loads are marked
// evict-first (ld.global.cs) to leave the cache to the x gathers; the slot
// stride is a pointer increment rather than a 64-bit multiply per entry.
template <typename T>
__device__ __forceinline__ T ell_row(int64_t n, int w, const int32_t* __restrict__ col, const T* __restrict__ val,
                                     const T* __restrict__ x, int64_t i, T acc) {
  const int32_t* cp = col + i;
  const T* vp = val + i;
#pragma unroll 9
  for (int k = 0; k < w; ++k) {
    acc = fma(__ldcs(vp), x[__ldcs(cp)], acc);
    cp += n;
    vp += n;
  }
  return acc;
}

// 3x3 inverse by cofactors; returns the determinant.
__device__ __forceinline__ double inv3(const double a[9], double r[9]) {
  const double c00 = a[4] * a[8] - a[5] * a[7];
  const double c01 = a[5] * a[6] - a[3] * a[8];
  const double c02 = a[3] * a[7] - a[4] * a[6];
  const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
  const double id = 1.0 / det;
  r[0] = c00 * id;
  r[1] = (a[2] * a[7] - a[1] * a[8]) * id;
  r[2] = (a[1] * a[5] - a[2] * a[4]) * id;
  r[3] = c01 * id;
  r[4] = (a[0] * a[8] - a[2] * a[6]) * id;
  r[5] = (a[2] * a[3] - a[0] * a[5]) * id;
  r[6] = c02 * id;
  r[7] = (a[1] * a[6] - a[0] * a[7]) * id;
  r[8] = (a[0] * a[4] - a[1] * a[3]) * id;
  return det;
}

// position of value v in the sorted list a[0..n) stored with stride s, or -1
__device__ __forceinline__ int find_sorted(const int32_t* a, int64_t s, int n, int32_t v) {
  int lo = 0, hi = n - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int32_t x = a[(int64_t)mid * s];
    if (x == v) return mid;
    if (x < v) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

// ---------------------------------------------------------------------------
// Optional per-kernel timing with CUDA events on the launching stream.
// A solver registers the matrices it wants tracked under a label; while a
// profiler is active on the calling thread, launches on those matrices are
// bracketed by events and credited with their algorithmic bytes.
// ---------------------------------------------------------------------------
struct Prof {
  struct Rec { int cls; double bytes; cudaEvent_t a, b; };
  struct Cls { std::string name; int64_t launches = 0; double ms = 0.0; double bytes = 0.0; };
  bool on = false;
  std::vector<std::pair<const void*, std::string>> labels;
  std::vector<Cls> classes;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  ~Prof();
  void label(const void* key, const char* name);
  const char* label_of(const void* key) const;
  int begin(const void* key, const char* kernel, double bytes, cudaStream_t s);
  void end(int token, cudaStream_t s);
  fvs_status collect();          // waits, folds event pairs into classes
  void reset();
};
extern thread_local Prof* g_prof;

struct ProfScope {
  int tok = -1;
  cudaStream_t s;
  ProfScope(const void* key, const char* kernel, double bytes, cudaStream_t st) : s(st) {
    if (g_prof && g_prof->on) tok = g_prof->begin(key, kernel, bytes, st);
  }
  ~ProfScope() {
    if (tok >= 0 && g_prof) g_prof->end(tok, s);
  }
};

}  // namespace fvs
