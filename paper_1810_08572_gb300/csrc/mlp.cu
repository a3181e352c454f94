// Learned surrogate of the UQ map (stochastic process inputs -> the
// microstructure outputs of Section 2.6, Eq. 22-23), replacing the plain
// solve inside Monte Carlo sampling (Section 2.7 uses a polynomial-chaos
// surrogate for the same role).
//
// A multilayer perceptron with GELU hidden layers and a linear output,
// BF16 weights and activations, FP32 accumulation in tensor memory on the
// tcgen05 tensor cores, FP32 master weights and Adam moments.  Every
// dimension is padded to a multiple of 16 with zeros that stay zero.
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "common.cuh"

namespace fvs {

#define GS(i, n) for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

enum { EPI_GELU = 0, EPI_LINEAR = 1, EPI_DGRAD = 2, EPI_WGRAD = 3 };

struct Epi {
  const float* bias;   // [N]           (GELU, LINEAR)
  float* z;            // [M x ldo] f32  pre-activations to keep (GELU, LINEAR) or read (DGRAD)
  bf16* hout;          // [M x ldo] bf16 activations (GELU) / previous delta (DGRAD)
  float* fout;         // [M x ldo] f32  output (LINEAR) / weight gradient (WGRAD)
  int ldo;
};

// ---------------------------------------------------------------------------
// C[M x N] = sum_k A(m, k) B(n, k) with A(m, k) = A[m*am + k*ak], B(n, k) =
// B[n*bn + k*bk] (BF16), N <= 128, K a multiple of 16, on the
// 5th-generation tensor cores (tcgen05) with a fused epilogue: one CTA of
// four warps per 128 rows of C, all N (<= 128) columns in one tile, K in
// chunks of 64.  Each chunk of A (128 x 64) and B (N x 64) is staged in
// shared memory in the canonical K-major layout without swizzle (core
// matrices of 8 rows x 16 bytes; 128 bytes between core matrices along K,
// 1024 bytes between groups of 8 rows), one thread issues the chunk's
// 128 x N x 16 BF16 MMAs into an FP32 accumulator in tensor memory and
// commits them to an mbarrier, and after the last chunk every warp reads
// its 32 accumulator lanes with tcgen05.ld for the fused epilogue.  Waits are
// bounded: a wait that runs out sets *err and the CTA still frees its
// tensor memory.
// ---------------------------------------------------------------------------
constexpr int TC_KC = 64;
constexpr int TC_COLS = 128;   // tensor-memory columns of a CTA (N <= 128)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ int tc_off(int r, int k) { return (r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }
// shared-memory matrix descriptor: start address, leading and stride byte
// offsets (16-byte units), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46);
}
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t phase) {
  uint32_t done = 0;
  for (int it = 0; it < (1 << 22) && !done; ++it)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(phase));
  return done != 0;
}

// fused epilogue of one 128-row tile: warp group `warp` (0-3) reads its 32
// accumulator lanes (rows m0 + 32 warp + lane) from tensor memory, 16
// columns at a time from c_begin in steps of c_step (two warps of the same
// group split the columns by starting 16 apart with a step of 32)
template <int EPI>
__device__ __forceinline__ void tc_epilogue(uint32_t taddr, int warp, int lane, int m0, int M, int N, const Epi& e,
                                            int c_begin = 0, int c_step = 16) {
  const int m = m0 + warp * 32 + lane;
  for (int c0 = c_begin; c0 < N; c0 += c_step) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    if (m >= M) continue;
    const int64_t o0 = (int64_t)m * e.ldo + c0;
    if ((e.ldo & 7) == 0) {
      // a lane's 16 columns as 16-byte vectors (row offsets are multiples of 8 elements)
      float v[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
      if (EPI == EPI_GELU || EPI == EPI_LINEAR) {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] += e.bias[c0 + j];
      }
      if (EPI == EPI_DGRAD) {
#pragma unroll
        for (int j = 0; j < 16; j += 4) {
          const float4 z = *reinterpret_cast<const float4*>(e.z + o0 + j);
          v[j] *= gelu_grad(z.x); v[j + 1] *= gelu_grad(z.y); v[j + 2] *= gelu_grad(z.z); v[j + 3] *= gelu_grad(z.w);
        }
      }
      float* f32out = EPI == EPI_GELU ? e.z : e.fout;
      if ((EPI == EPI_LINEAR || EPI == EPI_WGRAD || EPI == EPI_GELU) && f32out) {
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4*>(f32out + o0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
      }
      if (EPI == EPI_GELU || EPI == EPI_DGRAD) {
        uint32_t h[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float a = EPI == EPI_GELU ? gelu(v[2 * j]) : v[2 * j];
          const float b = EPI == EPI_GELU ? gelu(v[2 * j + 1]) : v[2 * j + 1];
          const __nv_bfloat162 hb = __floats2bfloat162_rn(a, b);
          h[j] = *reinterpret_cast<const uint32_t*>(&hb);
        }
        uint4* dst = reinterpret_cast<uint4*>(e.hout + o0);
        dst[0] = make_uint4(h[0], h[1], h[2], h[3]);
        dst[1] = make_uint4(h[4], h[5], h[6], h[7]);
      }
      continue;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int n = c0 + j;
      const int64_t o = o0 + j;
      float v = __uint_as_float(r[j]);
      if (EPI == EPI_GELU) {
        v += e.bias[n];
        if (e.z) e.z[o] = v;
        e.hout[o] = __float2bfloat16(gelu(v));
      } else if (EPI == EPI_LINEAR) {
        v += e.bias[n];
        e.fout[o] = v;
      } else if (EPI == EPI_DGRAD) {
        e.hout[o] = __float2bfloat16(v * gelu_grad(e.z[o]));
      } else {
        e.fout[o] = v;
      }
    }
  }
}

template <int EPI>
__global__ void __launch_bounds__(128, 1) k_mlp_gemm_tc(int M, int N, int K, const bf16* __restrict__ A, int am, int ak,
                                                        const bf16* __restrict__ B, int bn, int bk, Epi e, int* err) {
  __shared__ __align__(1024) unsigned char sa[128 * TC_KC * 2];
  __shared__ __align__(1024) unsigned char sb[TC_COLS * TC_KC * 2];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t taddr_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * 128;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&taddr_s)),
                 "r"(TC_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t taddr = taddr_s;
  // kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both
  // K-major, N >> 3, M >> 4
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  const bf16 zero = __float2bfloat16(0.f);
  uint32_t phase = 0;
  bool ok = true;
  for (int k0 = 0; k0 < K && ok; k0 += TC_KC) {
    const int kc = min(TC_KC, K - k0);
    // stage A(m, k) and B(n, k).  Rows contiguous in k go as 16-byte core
    // matrix rows (eight consecutive threads take the eight rows of one core
    // matrix: one 128-byte shared-memory wavefront, no bank conflicts);
    // otherwise element by element with the index that is contiguous in
    // memory running fastest.
    const int nch = kc >> 3;
    if (ak == 1 && (am & 7) == 0) {
      for (int t = tid; t < 128 * nch; t += 128) {
        const int q = t >> 3, ch = q % nch, r = (q / nch) * 8 + (t & 7);
        const int m = m0 + r;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (m < M) v = *reinterpret_cast<const uint4*>(A + (int64_t)m * am + k0 + ch * 8);
        *reinterpret_cast<uint4*>(sa + tc_off(r, ch * 8)) = v;
      }
    } else {
      for (int t = tid; t < 128 * kc; t += 128) {
        const int r = ak == 1 ? t / kc : t % 128, k = ak == 1 ? t % kc : t / 128;
        const int m = m0 + r;
        *(bf16*)(sa + tc_off(r, k)) = m < M ? A[(int64_t)m * am + (int64_t)(k0 + k) * ak] : zero;
      }
    }
    if (bk == 1 && (bn & 7) == 0) {
      for (int t = tid; t < N * nch; t += 128) {
        const int q = t >> 3, ch = q % nch, r = (q / nch) * 8 + (t & 7);
        *reinterpret_cast<uint4*>(sb + tc_off(r, ch * 8)) =
            *reinterpret_cast<const uint4*>(B + (int64_t)r * bn + k0 + ch * 8);
      }
    } else {
      for (int t = tid; t < N * kc; t += 128) {
        const int r = bk == 1 ? t / kc : t % N, k = bk == 1 ? t % kc : t / N;
        *(bf16*)(sb + tc_off(r, k)) = B[(int64_t)r * bn + (int64_t)(k0 + k) * bk];
      }
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      for (int kk = 0; kk < kc / 16; ++kk) {
        const uint64_t ad = tc_desc(smem_u32(sa) + kk * 256), bd = tc_desc(smem_u32(sb) + kk * 256);
        const uint32_t accum = (k0 > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
            "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&mbar)));
    }
    if (!tc_wait(smem_u32(&mbar), phase)) {
      ok = false;
      if (lane == 0) atomicOr(err, 1);
      tc_wait(smem_u32(&mbar), phase);   // give the MMAs in flight a second bounded chance
    }
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
  }
  if (ok) tc_epilogue<EPI>(taddr, warp, lane, m0, M, N, e);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TC_COLS));
}

// ---------------------------------------------------------------------------
// Forward GEMM (activations A [M x K] row-major times weights B [N x K],
// K <= 128, N <= 128) as a persistent kernel: each CTA stages the weights
// once, allocates its tensor-memory accumulator once, and walks the 128-row
// tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... with eight warps (two per
// accumulator lane group in the epilogue)  The A tile of the next
// tile is copied into the other of two shared-memory buffers (cp.async,
// 16-byte core-matrix rows, zero fill past M) while the current tile's MMAs
// and epilogue run.  Layouts, descriptors and the epilogue are those of
// k_mlp_gemm_tc; every wait on the MMAs is bounded and the decision to stop
// is taken by the whole CTA (__syncthreads_or), which then drains its copies
// and frees its tensor memory.
// ---------------------------------------------------------------------------
constexpr int TC_CHUNK_BYTES = 128 * TC_KC * 2;   // one K chunk of 128 rows
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
// rows of A's tile m0 into buffer sa (K in chunks of TC_KC, 16-byte pieces)
__device__ __forceinline__ void tc_stage_a_async(unsigned char* sa, const bf16* A, int M, int K, int m0, int tid,
                                                 int nthr) {
  const int nchunk = (K + TC_KC - 1) / TC_KC;
  for (int c = 0; c < nchunk; ++c) {
    const int k0 = c * TC_KC, kc = min(TC_KC, K - k0), nch = kc >> 3;
    unsigned char* base = sa + c * TC_CHUNK_BYTES;
    for (int t = tid; t < 128 * nch; t += nthr) {
      const int q = t >> 3, ch = q % nch, r = (q / nch) * 8 + (t & 7);
      const int m = m0 + r;
      const bf16* src = m < M ? A + (int64_t)m * K + k0 + ch * 8 : A;
      cp_async16(smem_u32(base + tc_off(r, ch * 8)), src, m < M ? 16 : 0);
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int EPI>
__global__ void __launch_bounds__(256, 1) k_mlp_fwd_tc(int M, int N, int K, const bf16* __restrict__ A,
                                                       const bf16* __restrict__ B, Epi e, int* err) {
  extern __shared__ __align__(1024) unsigned char tc_dyn[];
  const int nchunk = (K + TC_KC - 1) / TC_KC;
  unsigned char* sb = tc_dyn;                               // nchunk chunks
  unsigned char* sa0 = tc_dyn + nchunk * TC_CHUNK_BYTES;    // 2 x nchunk chunks
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t taddr_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = (M + 127) / 128;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&taddr_s)),
                 "r"(TC_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
  // the weights, once
  for (int c = 0; c < nchunk; ++c) {
    const int k0 = c * TC_KC, kc = min(TC_KC, K - k0), nch = kc >> 3;
    for (int t = tid; t < N * nch; t += blockDim.x) {
      const int q = t >> 3, ch = q % nch, r = (q / nch) * 8 + (t & 7);
      *reinterpret_cast<uint4*>(sb + c * TC_CHUNK_BYTES + tc_off(r, ch * 8)) =
          *reinterpret_cast<const uint4*>(B + (int64_t)r * K + k0 + ch * 8);
    }
  }
  if (blockIdx.x < ntiles) tc_stage_a_async(sa0, A, M, K, blockIdx.x * 128, tid, blockDim.x);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t taddr = taddr_s;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  uint32_t phase = 0;
  int buf = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int next = tile + gridDim.x;
    if (next < ntiles) {
      tc_stage_a_async(sa0 + (buf ^ 1) * nchunk * TC_CHUNK_BYTES, A, M, K, next * 128, tid, blockDim.x);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const unsigned char* sa = sa0 + buf * nchunk * TC_CHUNK_BYTES;
      for (int c = 0; c < nchunk; ++c) {
        const int kc = min(TC_KC, K - c * TC_KC);
        for (int kk = 0; kk < kc / 16; ++kk) {
          const uint64_t ad = tc_desc(smem_u32(sa + c * TC_CHUNK_BYTES) + kk * 256);
          const uint64_t bd = tc_desc(smem_u32(sb + c * TC_CHUNK_BYTES) + kk * 256);
          const uint32_t accum = (c > 0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
              "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&mbar)));
    }
    const bool late = __syncthreads_or(!tc_wait(smem_u32(&mbar), phase) ? 1 : 0);
    if (late) {
      if (tid == 0) atomicOr(err, 1);
      tc_wait(smem_u32(&mbar), phase);   // the MMAs in flight get a second bounded chance
      break;
    }
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;");
    // eight warps: warp w reads accumulator lanes 32 (w % 4) .. +31, the
    // 16-column blocks starting at 16 (w / 4), every other one
    tc_epilogue<EPI>(taddr, warp & 3, lane, tile * 128, M, N, e, 16 * (warp >> 2), 32);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();   // accumulator read before the next tile's MMAs; buffer free for reuse
    asm volatile("tcgen05.fence::after_thread_sync;");
    buf ^= 1;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TC_COLS));
}

// inputs (double, [n x nin]) -> normalised BF16 rows padded to kin
__global__ void k_mlp_in(int64_t n, int nin, int kin, const double* X, const float* mu, const float* sd, bf16* H) {
  GS(i, n * (int64_t)kin) {
    const int64_t r = i / kin;
    const int c = (int)(i - r * kin);
    const float v = c < nin ? (float)((X[r * nin + c] - (double)mu[c]) / (double)sd[c]) : 0.f;
    H[i] = __float2bfloat16(v);
  }
}
// output rows (f32, padded) -> de-normalised doubles [n x nout]
__global__ void k_mlp_out(int64_t n, int nout, int kout, const float* Y, const float* mu, const float* sd, double* out) {
  GS(i, n * (int64_t)nout) {
    const int64_t r = i / nout;
    const int c = (int)(i - r * nout);
    out[i] = (double)Y[r * kout + c] * (double)sd[c] + (double)mu[c];
  }
}
// MSE loss on normalised targets; delta = 2 (y - t) / (n nout) as BF16, loss partials
__global__ void k_mlp_loss(int64_t n, int nout, int kout, const float* Y, const double* T, const float* mu,
                           const float* sd, bf16* delta, double* part) {
  __shared__ double sh[32];
  double acc = 0.0;
  const double scale = 2.0 / ((double)n * nout);
  GS(i, n * (int64_t)kout) {
    const int64_t r = i / kout;
    const int c = (int)(i - r * kout);
    float d = 0.f;
    if (c < nout) {
      const double tn = (T[r * nout + c] - (double)mu[c]) / (double)sd[c];
      const double diff = (double)Y[i] - tn;
      acc += diff * diff;
      d = (float)(scale * diff);
    }
    delta[i] = __float2bfloat16(d);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}
__global__ void k_sum_final(int nb, const double* part, double scale, double* out) {
  __shared__ double sh[32];
  double a = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) a += part[b];
  a = block_sum(a, sh);
  if (threadIdx.x == 0) *out = a * scale;
}
// bias gradient: db[n] = sum_m delta[m][n] (one thread per column)
__global__ void k_bias_grad(int M, int N, const bf16* delta, float* db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += __bfloat162float(delta[(int64_t)m * N + n]);
  db[n] = s;
}
// Adam on FP32 master weights; refresh the BF16 copy.  mask keeps padding at
// zero.  omb1 = 1 - b1, omb2 = 1 - b2 and the bias corrections c1 = 1 - b1^t,
// c2 = 1 - b2^t come from the host in double precision: formed in FP32,
// 1 - b2^t loses about five digits to cancellation (b2^t is near 1).
__global__ void k_adam(int64_t n, float* w, float* m, float* v, const float* g, const uint8_t* mask, float lr,
                       float b1, float omb1, float b2, float omb2, float eps, float c1, float c2, bf16* wb) {
  GS(i, n) {
    if (!mask[i]) continue;
    const float gi = g[i];
    const float mi = b1 * m[i] + omb1 * gi;
    const float vi = b2 * v[i] + omb2 * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16(wi);
  }
}
__global__ void k_to_bf16(int64_t n, const float* a, bf16* b) {
  GS(i, n) b[i] = __float2bfloat16(a[i]);
}
// counter-based initialisation: uniform(-lim, lim) from a 64-bit mix of (seed, index)
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ULL;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
  return x ^ (x >> 31);
}
__global__ void k_init_w(int64_t n, int kpad, int nin_real, int nout_real, uint64_t seed, float lim, float* w,
                         uint8_t* mask) {
  GS(i, n) {
    const int r = (int)(i / kpad), c = (int)(i - (int64_t)r * kpad);
    const bool live = r < nout_real && c < nin_real;
    const double u = (double)(mix64(seed ^ (uint64_t)i * 0x2545f4914f6cdd1dULL) >> 11) * (1.0 / 9007199254740992.0);
    w[i] = live ? (float)((2.0 * u - 1.0) * lim) : 0.f;
    mask[i] = live;
  }
}

}  // namespace fvs

// ---------------------------------------------------------------------------
// the surrogate object
// ---------------------------------------------------------------------------
using namespace fvs;

struct fvs_surrogate_s {
  cudaStream_t stream = nullptr;
  int nin = 0, nout = 0, hidden = 0, nlayers = 0;   // nlayers = hidden layers
  std::vector<int> kd;       // padded widths: kd[0] input, kd[L] output
  std::vector<int> real;     // real widths
  // per layer l (0..L-1): W [kd[l+1] x kd[l]], b [kd[l+1]]
  DBuf<float> w32, m, v, g;  // all layer weights then all biases, flattened
  DBuf<bf16> wb;             // BF16 copy of the weights part
  DBuf<uint8_t> mask;
  std::vector<int64_t> woff, boff;
  int64_t nw = 0, nparam = 0;
  DBuf<float> mu_in, sd_in, mu_out, sd_out;
  int64_t step = 0;
  // work (sized for the largest batch seen)
  int64_t cap = 0;
  std::vector<DBuf<bf16>*> H;   // activations per layer input (L+1 buffers)
  std::vector<DBuf<float>*> Z;  // pre-activations per layer output
  DBuf<bf16> d0, d1;
  DBuf<float> Y;
  DBuf<double> part, lossv, Xd, Td;
  DBuf<int> tc_err;          // set by a tensor-core GEMM whose bounded wait ran out
  ~fvs_surrogate_s() {
    for (auto* p : H) delete p;
    for (auto* p : Z) delete p;
  }
};

namespace fvs {

static fvs_status sg_work(fvs_surrogate_s* s, int64_t n) {
  if (n <= s->cap) return FVS_OK;
  const int L = (int)s->kd.size() - 1;
  for (auto* p : s->H) delete p;
  for (auto* p : s->Z) delete p;
  s->H.clear();
  s->Z.clear();
  for (int l = 0; l <= L; ++l) {
    s->H.push_back(new DBuf<bf16>());
    FVS_TRY(s->H.back()->alloc((size_t)n * s->kd[l] + 16));
  }
  for (int l = 0; l < L; ++l) {
    s->Z.push_back(new DBuf<float>());
    FVS_TRY(s->Z.back()->alloc((size_t)n * s->kd[l + 1] + 16));
  }
  int kmax = 0;
  for (int k : s->kd) kmax = std::max(kmax, k);
  FVS_TRY(s->d0.alloc((size_t)n * kmax + 16));
  FVS_TRY(s->d1.alloc((size_t)n * kmax + 16));
  FVS_TRY(s->Y.alloc((size_t)n * s->kd[L] + 16));
  FVS_TRY(s->part.alloc(1024));
  FVS_TRY(s->lossv.alloc(1));
  s->cap = n;
  return FVS_OK;
}

static int tc_grid(int64_t M) { return (int)((M + 127) / 128); }

// forward layer C = A W^T with the fused epilogue: the persistent kernel
// (up to four CTAs per SM, weights staged once per CTA, next A tile copied
// while the current one is multiplied) where K and N fit one tile, else one
// CTA a tile
template <int EPI>
static fvs_status tc_forward(cudaStream_t st, int64_t n, int N, int K, const bf16* A, const bf16* W, const Epi& e,
                             int* err) {
  if (K <= 128 && N <= 128) {
    const int nchunk = (K + TC_KC - 1) / TC_KC;
    const size_t smem = (size_t)3 * nchunk * TC_CHUNK_BYTES;
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
      FVS_CUDA(cudaFuncSetAttribute(k_mlp_fwd_tc<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    3 * 2 * TC_CHUNK_BYTES));
      attr_set[dev] = true;
    }
    // CTAs per SM: tensor memory allows four (128 columns each), shared memory
    // 227 KB / (smem + 1 KB)
    const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(4, (227 * 1024) / (smem + 1024)));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tc_grid(n), (int64_t)per_sm * sm_count()));
    k_mlp_fwd_tc<EPI><<<grid, 256, smem, st>>>((int)n, N, K, A, W, e, err);
  } else {
    k_mlp_gemm_tc<EPI><<<tc_grid(n), 128, 0, st>>>((int)n, N, K, A, K, 1, W, K, 1, e, err);
  }
  FVS_COUNT_LAUNCH();
  return FVS_OK;
}

// forward pass of n normalised BF16 rows already in H[0]; keep Z when training
static fvs_status sg_forward(fvs_surrogate_s* s, int64_t n, bool keep) {
  const int L = (int)s->kd.size() - 1;
  cudaStream_t st = s->stream;
  for (int l = 0; l < L; ++l) {
    const int K = s->kd[l], N = s->kd[l + 1];
    Epi e{};
    e.bias = s->w32.p + s->boff[l];
    e.ldo = N;
    const bf16* W = s->wb.p + s->woff[l];
    if (l < L - 1) {
      e.z = keep ? s->Z[l]->p : nullptr;
      e.hout = s->H[l + 1]->p;
      FVS_TRY(tc_forward<EPI_GELU>(st, n, N, K, s->H[l]->p, W, e, s->tc_err.p));
    } else {
      e.fout = s->Y.p;
      FVS_TRY(tc_forward<EPI_LINEAR>(st, n, N, K, s->H[l]->p, W, e, s->tc_err.p));
    }
  }
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

// gradients of the loss at the current weights for n rows (X, T on device)
static fvs_status sg_gradients(fvs_surrogate_s* s, int64_t n, double* loss_host) {
  const int L = (int)s->kd.size() - 1;
  cudaStream_t st = s->stream;
  FVS_TRY(sg_work(s, n));
  k_mlp_in<<<stride_grid(n * s->kd[0], 256), 256, 0, st>>>(n, s->nin, s->kd[0], s->Xd.p, s->mu_in.p, s->sd_in.p,
                                                          s->H[0]->p); FVS_COUNT_LAUNCH();
  FVS_TRY(sg_forward(s, n, true));
  const int nb = 256;
  k_mlp_loss<<<nb, 256, 0, st>>>(n, s->nout, s->kd[L], s->Y.p, s->Td.p, s->mu_out.p, s->sd_out.p, s->d0.p,
                                 s->part.p); FVS_COUNT_LAUNCH();
  k_sum_final<<<1, 256, 0, st>>>(nb, s->part.p, 1.0 / ((double)n * s->nout), s->lossv.p); FVS_COUNT_LAUNCH();
  bf16* dcur = s->d0.p;
  bf16* dnext = s->d1.p;
  for (int l = L - 1; l >= 0; --l) {
    const int K = s->kd[l], N = s->kd[l + 1];
    // weight gradient dW[N x K] = delta^T H_l : A(m=n, k=b) = delta[b*N + n], B(n'=k, k=b) = H[b*K + k]
    Epi e{};
    e.fout = s->g.p + s->woff[l];
    e.ldo = K;
    k_mlp_gemm_tc<EPI_WGRAD><<<tc_grid(N), 128, 0, st>>>(N, K, (int)((n + 15) / 16 * 16), dcur, 1, N,
                                                         s->H[l]->p, 1, K, e, s->tc_err.p); FVS_COUNT_LAUNCH();
    k_bias_grad<<<(N + 127) / 128, 128, 0, st>>>((int)n, N, dcur, s->g.p + s->boff[l]); FVS_COUNT_LAUNCH();
    if (l > 0) {
      // delta_{l-1} = (delta_l W_l) * gelu'(Z_{l-1}): A(m=b, k=n) = delta[b*N + n], B(n'=k, k=n) = W[n*K + k]
      Epi d{};
      d.z = s->Z[l - 1]->p;
      d.hout = dnext;
      d.ldo = K;
      k_mlp_gemm_tc<EPI_DGRAD><<<tc_grid(n), 128, 0, st>>>((int)n, K, N, dcur, N, 1, s->wb.p + s->woff[l], 1, K, d,
                                                          s->tc_err.p);
      FVS_COUNT_LAUNCH();
      std::swap(dcur, dnext);
    }
  }
  FVS_LAUNCH_CHECK();
  if (loss_host) {
    FVS_CUDA(cudaMemcpyAsync(loss_host, s->lossv.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    FVS_CUDA(cudaStreamSynchronize(st));
  }
  return FVS_OK;
}

}  // namespace fvs

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
#define FVS_API extern "C" __attribute__((visibility("default")))

namespace fvs {
__global__ void k_zero_rows_bf16(int64_t from, int64_t to, int k, bf16* h) {
  GS(i, (to - from) * (int64_t)k) h[from * k + i] = __float2bfloat16(0.f);
}

// flattened real parameters (oracle order: per layer W row-major, then b) <-> padded device layout
static void layout(const fvs_surrogate_s* s, std::vector<int64_t>& dev_index) {
  dev_index.clear();
  const int L = (int)s->kd.size() - 1;
  for (int l = 0; l < L; ++l) {
    for (int r = 0; r < s->real[l + 1]; ++r)
      for (int c = 0; c < s->real[l]; ++c) dev_index.push_back(s->woff[l] + (int64_t)r * s->kd[l] + c);
    for (int r = 0; r < s->real[l + 1]; ++r) dev_index.push_back(s->boff[l] + r);
  }
}

static fvs_status upload_xt(fvs_surrogate_s* s, const double* X, const double* T, int64_t n) {
  FVS_TRY(s->Xd.alloc((size_t)n * s->nin + 1));
  FVS_CUDA(cudaMemcpyAsync(s->Xd.p, X, n * s->nin * sizeof(double), cudaMemcpyHostToDevice, s->stream));
  if (T) {
    FVS_TRY(s->Td.alloc((size_t)n * s->nout + 1));
    FVS_CUDA(cudaMemcpyAsync(s->Td.p, T, n * s->nout * sizeof(double), cudaMemcpyHostToDevice, s->stream));
  }
  return FVS_OK;
}

static fvs_status zero_padding_rows(fvs_surrogate_s* s, int64_t n) {
  const int64_t nr = (n + 15) / 16 * 16;
  if (nr == n) return FVS_OK;
  for (size_t l = 0; l < s->H.size(); ++l) {
    k_zero_rows_bf16<<<1, 256, 0, s->stream>>>(n, nr, s->kd[l], s->H[l]->p); FVS_COUNT_LAUNCH();
  }
  // delta buffers hold rows of different widths (>= 16): clear everything
  // past the first n rows of the narrowest width once; live rows are rewritten
  int kmax = 0;
  for (int k : s->kd) kmax = std::max(kmax, k);
  const size_t tail = s->d0.n - (size_t)n * 16;
  FVS_CUDA(cudaMemsetAsync(s->d0.p + (size_t)n * 16, 0, tail * sizeof(bf16), s->stream));
  FVS_CUDA(cudaMemsetAsync(s->d1.p + (size_t)n * 16, 0, tail * sizeof(bf16), s->stream));
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}
}  // namespace fvs

FVS_API fvs_status fvs_surrogate_create(int32_t n_in, int32_t n_hidden, int32_t n_hidden_layers, int32_t n_out,
                                        uint64_t seed, void* stream, fvs_surrogate* out) {
  if (!out || n_in < 1 || n_in > 128 || n_out < 1 || n_out > 128 || n_hidden < 1 || n_hidden > 128 ||
      n_hidden_layers < 1 || n_hidden_layers > 16) {
    set_error("fvs_surrogate_create: widths must be 1..128, hidden layers 1..16");
    return FVS_ERR_ARG;
  }
  *out = nullptr;
  fvs_surrogate_s* s = new fvs_surrogate_s();
  s->stream = (cudaStream_t)stream;
  AllocStream as(s->stream);
  auto pad = [](int x) { return (x + 15) / 16 * 16; };
  s->nin = n_in; s->nout = n_out; s->hidden = n_hidden; s->nlayers = n_hidden_layers;
  s->real.push_back(n_in);
  for (int l = 0; l < n_hidden_layers; ++l) s->real.push_back(n_hidden);
  s->real.push_back(n_out);
  for (int r : s->real) s->kd.push_back(pad(r));
  const int L = (int)s->kd.size() - 1;
  int64_t off = 0;
  for (int l = 0; l < L; ++l) { s->woff.push_back(off); off += (int64_t)s->kd[l + 1] * s->kd[l]; }
  s->nw = off;
  for (int l = 0; l < L; ++l) { s->boff.push_back(off); off += s->kd[l + 1]; }
  s->nparam = off;
  fvs_status r = FVS_OK;
  if (r == FVS_OK) r = s->w32.alloc(s->nparam);
  if (r == FVS_OK) r = s->m.alloc(s->nparam);
  if (r == FVS_OK) r = s->v.alloc(s->nparam);
  if (r == FVS_OK) r = s->g.alloc(s->nparam);
  if (r == FVS_OK) r = s->wb.alloc(s->nw);
  if (r == FVS_OK) r = s->mask.alloc(s->nparam);
  if (r == FVS_OK) r = s->mu_in.alloc(128);
  if (r == FVS_OK) r = s->sd_in.alloc(128);
  if (r == FVS_OK) r = s->mu_out.alloc(128);
  if (r == FVS_OK) r = s->sd_out.alloc(128);
  if (r == FVS_OK) r = s->tc_err.alloc(1);
  if (r != FVS_OK) { delete s; return r; }
  s->w32.zero(s->stream); s->m.zero(s->stream); s->v.zero(s->stream); s->g.zero(s->stream);
  s->mask.zero(s->stream);
  s->tc_err.zero(s->stream);
  for (int l = 0; l < L; ++l) {
    const int64_t n = (int64_t)s->kd[l + 1] * s->kd[l];
    const float lim = sqrtf(6.0f / (float)s->real[l]);
    k_init_w<<<stride_grid(n, 256), 256, 0, s->stream>>>(n, s->kd[l], s->real[l], s->real[l + 1],
                                                        seed * 1315423911ULL + l, lim, s->w32.p + s->woff[l],
                                                        s->mask.p + s->woff[l]);
    FVS_COUNT_LAUNCH();
  }
  // biases: live entries start at zero
  {
    std::vector<uint8_t> bm(s->nparam - s->nw, 0);
    for (int l = 0; l < L; ++l)
      for (int r2 = 0; r2 < s->real[l + 1]; ++r2) bm[s->boff[l] - s->nw + r2] = 1;
    cudaMemcpyAsync(s->mask.p + s->nw, bm.data(), bm.size(), cudaMemcpyHostToDevice, s->stream);
    cudaStreamSynchronize(s->stream);
  }
  k_to_bf16<<<stride_grid(s->nw, 256), 256, 0, s->stream>>>(s->nw, s->w32.p, s->wb.p);
  FVS_COUNT_LAUNCH();
  std::vector<float> one(128, 1.0f), zero(128, 0.0f);
  cudaMemcpyAsync(s->mu_in.p, zero.data(), 512, cudaMemcpyHostToDevice, s->stream);
  cudaMemcpyAsync(s->sd_in.p, one.data(), 512, cudaMemcpyHostToDevice, s->stream);
  cudaMemcpyAsync(s->mu_out.p, zero.data(), 512, cudaMemcpyHostToDevice, s->stream);
  cudaMemcpyAsync(s->sd_out.p, one.data(), 512, cudaMemcpyHostToDevice, s->stream);
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) {
    set_error("fvs_surrogate_create: %s", cudaGetErrorString(cudaGetLastError()));
    delete s;
    return FVS_ERR_CUDA;
  }
  *out = s;
  return FVS_OK;
}

namespace fvs {
// input and output widths of a model (the UQ surrogate mode checks them)
fvs_status surrogate_dims(fvs_surrogate s, int* nin, int* nout) {
  if (!s) {
    set_error("NULL surrogate");
    return FVS_ERR_ARG;
  }
  *nin = s->nin;
  *nout = s->nout;
  return FVS_OK;
}
}  // namespace fvs

FVS_API fvs_status fvs_surrogate_destroy(fvs_surrogate s) {
  if (!s) return FVS_ERR_ARG;
  cudaStream_t st = s->stream;
  {
    AllocStream as(st);
    cudaStreamSynchronize(st);
    delete s;
  }
  cudaStreamSynchronize(st);
  return FVS_OK;
}

FVS_API fvs_status fvs_surrogate_set_scaling(fvs_surrogate s, const double* mu_in, const double* sd_in,
                                             const double* mu_out, const double* sd_out) {
  if (!s || !mu_in || !sd_in || !mu_out || !sd_out) {
    set_error("fvs_surrogate_set_scaling: NULL argument");
    return FVS_ERR_ARG;
  }
  std::vector<float> a(128, 0.f), b(128, 1.f), c(128, 0.f), d(128, 1.f);
  for (int i = 0; i < s->nin; ++i) {
    if (!(sd_in[i] > 0)) { set_error("fvs_surrogate_set_scaling: non-positive scale"); return FVS_ERR_ARG; }
    a[i] = (float)mu_in[i]; b[i] = (float)sd_in[i];
  }
  for (int i = 0; i < s->nout; ++i) {
    if (!(sd_out[i] > 0)) { set_error("fvs_surrogate_set_scaling: non-positive scale"); return FVS_ERR_ARG; }
    c[i] = (float)mu_out[i]; d[i] = (float)sd_out[i];
  }
  FVS_CUDA(cudaMemcpyAsync(s->mu_in.p, a.data(), 512, cudaMemcpyHostToDevice, s->stream));
  FVS_CUDA(cudaMemcpyAsync(s->sd_in.p, b.data(), 512, cudaMemcpyHostToDevice, s->stream));
  FVS_CUDA(cudaMemcpyAsync(s->mu_out.p, c.data(), 512, cudaMemcpyHostToDevice, s->stream));
  FVS_CUDA(cudaMemcpyAsync(s->sd_out.p, d.data(), 512, cudaMemcpyHostToDevice, s->stream));
  FVS_CUDA(cudaStreamSynchronize(s->stream));
  return FVS_OK;
}

FVS_API int64_t fvs_surrogate_num_params(fvs_surrogate s) {
  if (!s) return -1;
  std::vector<int64_t> idx;
  layout(s, idx);
  return (int64_t)idx.size();
}

FVS_API fvs_status fvs_surrogate_params(fvs_surrogate s, double* inout, int64_t len, int set) {
  if (!s || !inout) {
    set_error("fvs_surrogate_params: NULL argument");
    return FVS_ERR_ARG;
  }
  AllocStream as(s->stream);
  std::vector<int64_t> idx;
  layout(s, idx);
  if (len < (int64_t)idx.size()) {
    set_error("fvs_surrogate_params: need %lld values", (long long)idx.size());
    return FVS_ERR_ARG;
  }
  std::vector<float> h(s->nparam);
  FVS_CUDA(cudaMemcpyAsync(h.data(), s->w32.p, s->nparam * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
  FVS_CUDA(cudaStreamSynchronize(s->stream));
  if (set) {
    for (size_t i = 0; i < idx.size(); ++i) h[idx[i]] = (float)inout[i];
    FVS_CUDA(cudaMemcpyAsync(s->w32.p, h.data(), s->nparam * sizeof(float), cudaMemcpyHostToDevice, s->stream));
    k_to_bf16<<<stride_grid(s->nw, 256), 256, 0, s->stream>>>(s->nw, s->w32.p, s->wb.p);
    FVS_COUNT_LAUNCH();
    FVS_CUDA(cudaStreamSynchronize(s->stream));
  } else {
    for (size_t i = 0; i < idx.size(); ++i) inout[i] = (double)h[idx[i]];
  }
  return FVS_OK;
}

// FVS_ERR_TIMEOUT if a tensor-core GEMM gave up waiting on its MMAs (the
// flag is cleared for the next call)
static fvs_status tc_check(fvs_surrogate s) {
  int h = 0;
  FVS_CUDA(cudaMemcpyAsync(&h, s->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  FVS_CUDA(cudaStreamSynchronize(s->stream));
  if (h) {
    s->tc_err.zero(s->stream);
    set_error("surrogate: a tensor-core GEMM timed out waiting for its MMAs");
    return FVS_ERR_TIMEOUT;
  }
  return FVS_OK;
}

FVS_API fvs_status fvs_surrogate_gradients(fvs_surrogate s, const double* X, const double* T, int64_t n,
                                           double* grad, int64_t grad_len, double* loss) {
  if (!s || !X || !T || !grad || n <= 0) {
    set_error("fvs_surrogate_gradients: bad argument");
    return FVS_ERR_ARG;
  }
  AllocStream as(s->stream);
  std::vector<int64_t> idx;
  layout(s, idx);
  if (grad_len < (int64_t)idx.size()) {
    set_error("fvs_surrogate_gradients: need %lld values", (long long)idx.size());
    return FVS_ERR_ARG;
  }
  FVS_TRY(upload_xt(s, X, T, n));
  FVS_TRY(sg_work(s, n + 16));
  FVS_TRY(zero_padding_rows(s, n));
  FVS_TRY(sg_gradients(s, n, loss));
  std::vector<float> h(s->nparam);
  FVS_CUDA(cudaMemcpyAsync(h.data(), s->g.p, s->nparam * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
  FVS_CUDA(cudaStreamSynchronize(s->stream));
  FVS_TRY(tc_check(s));
  for (size_t i = 0; i < idx.size(); ++i) grad[i] = (double)h[idx[i]];
  return FVS_OK;
}

FVS_API fvs_status fvs_surrogate_train(fvs_surrogate s, const double* X, const double* T, int64_t n, int32_t epochs,
                                       double lr, double* final_loss) {
  if (!s || !X || !T || n <= 0 || epochs < 0 || !(lr > 0)) {
    set_error("fvs_surrogate_train: bad argument");
    return FVS_ERR_ARG;
  }
  AllocStream as(s->stream);
  FVS_TRY(upload_xt(s, X, T, n));
  FVS_TRY(sg_work(s, n + 16));
  FVS_TRY(zero_padding_rows(s, n));
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  for (int e = 0; e < epochs; ++e) {
    FVS_TRY(sg_gradients(s, n, nullptr));
    ++s->step;
    const double c1 = 1.0 - pow(b1, (double)s->step), c2 = 1.0 - pow(b2, (double)s->step);
    k_adam<<<stride_grid(s->nparam, 256), 256, 0, s->stream>>>(s->nparam, s->w32.p, s->m.p, s->v.p, s->g.p,
                                                              s->mask.p, (float)lr, (float)b1, (float)(1.0 - b1),
                                                              (float)b2, (float)(1.0 - b2), (float)eps, (float)c1,
                                                              (float)c2, nullptr);
    FVS_COUNT_LAUNCH();
    k_to_bf16<<<stride_grid(s->nw, 256), 256, 0, s->stream>>>(s->nw, s->w32.p, s->wb.p);
    FVS_COUNT_LAUNCH();
  }
  FVS_LAUNCH_CHECK();
  double l = 0.0;
  FVS_TRY(sg_gradients(s, n, &l));
  FVS_TRY(tc_check(s));
  if (final_loss) *final_loss = l;
  return FVS_OK;
}

FVS_API fvs_status fvs_surrogate_predict(fvs_surrogate s, const double* X, double* Y, int64_t n, int on_device) {
  if (!s || !X || !Y || n <= 0) {
    set_error("fvs_surrogate_predict: bad argument");
    return FVS_ERR_ARG;
  }
  AllocStream as(s->stream);
  const int L = (int)s->kd.size() - 1;
  const double* Xd = X;
  if (!on_device) {
    FVS_TRY(upload_xt(s, X, nullptr, n));
    Xd = s->Xd.p;
  }
  FVS_TRY(sg_work(s, n + 16));
  k_mlp_in<<<stride_grid(n * s->kd[0], 256), 256, 0, s->stream>>>(n, s->nin, s->kd[0], Xd, s->mu_in.p, s->sd_in.p,
                                                                  s->H[0]->p);
  FVS_COUNT_LAUNCH();
  FVS_TRY(sg_forward(s, n, false));
  DBuf<double> out;
  double* Yd = Y;
  if (!on_device) {
    FVS_TRY(out.alloc((size_t)n * s->nout));
    Yd = out.p;
  }
  k_mlp_out<<<stride_grid(n * s->nout, 256), 256, 0, s->stream>>>(n, s->nout, s->kd[L], s->Y.p, s->mu_out.p,
                                                                  s->sd_out.p, Yd);
  FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  if (!on_device) FVS_CUDA(cudaMemcpyAsync(Y, Yd, n * s->nout * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  FVS_CUDA(cudaStreamSynchronize(s->stream));
  return tc_check(s);
}
