// Sparse linear algebra kernels and Krylov drivers (Section 2.5: the paper
// uses AMG-preconditioned Krylov solvers; these are the GPU-native ones).
#include <cstdlib>

#include "la.cuh"

namespace fvs {

static constexpr int RB = 256;  // threads per reduction block

// ---------------------------------------------------------------------------
// SpMV and residual (ELL, one thread per row, slot-major coalesced loads)
// ---------------------------------------------------------------------------
__global__ void k_spmv(int64_t n, int w, const int32_t* __restrict__ col, const double* __restrict__ val,
                       const double* __restrict__ x, double* __restrict__ y,
                       const double* __restrict__ dextra) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double acc = ell_row(n, w, col, val, x, i, dextra ? dextra[i] * x[i] : 0.0);
    y[i] = acc;
  }
}

__global__ void k_residual(int64_t n, int w, const int32_t* __restrict__ col, const double* __restrict__ val,
                           const double* __restrict__ x, const double* __restrict__ b, double* __restrict__ r,
                           const double* __restrict__ dextra) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double acc = ell_row(n, w, col, val, x, i, dextra ? dextra[i] * x[i] : 0.0);
    r[i] = b[i] - acc;
  }
}

fvs_status spmv(cudaStream_t s, const Ell& A, const double* x, double* y, const double* dextra) {
  if (A.n == 0) return FVS_OK;
  ProfScope ps(&A, "spmv", (double)A.n * (12.0 * A.w + 16.0 + (dextra ? 8.0 : 0.0)), s);
  k_spmv<<<stride_grid(A.n, 256), 256, 0, s>>>(A.n, A.w, A.col, A.val, x, y, dextra); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

fvs_status residual(cudaStream_t s, const Ell& A, const double* x, const double* b, double* r,
                    const double* dextra) {
  if (A.n == 0) return FVS_OK;
  ProfScope ps(&A, "residual", (double)A.n * (12.0 * A.w + 24.0 + (dextra ? 8.0 : 0.0)), s);
  k_residual<<<stride_grid(A.n, 256), 256, 0, s>>>(A.n, A.w, A.col, A.val, x, b, r, dextra); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

// ---------------------------------------------------------------------------
// Deterministic reductions: fixed grid, block partials, single-block final sum
// ---------------------------------------------------------------------------
__global__ void k_dot2_part(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                            const double* __restrict__ c, const double* __restrict__ d, double* __restrict__ part) {
  __shared__ double sh[32];
  double s0 = 0.0, s1 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    s0 = fma(a[i], b[i], s0);
    if (c) s1 = fma(c[i], d[i], s1);
  }
  s0 = block_sum(s0, sh);
  s1 = block_sum(s1, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s0;
    part[gridDim.x + blockIdx.x] = s1;
  }
}

__global__ void k_maxdiff2_part(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                                const double* __restrict__ c, const double* __restrict__ d, double* __restrict__ part) {
  __shared__ double sh[32];
  double s0 = 0.0, s1 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    s0 = fmax(s0, fabs(a[i] - b[i]));
    if (c) s1 = fmax(s1, fabs(c[i] - d[i]));
  }
  s0 = block_max(s0, sh);
  s1 = block_max(s1, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s0;
    part[gridDim.x + blockIdx.x] = s1;
  }
}

// Final sum of partials into slots; mode 1 = max.  Before overwriting s0,
// the previous value is moved to s0_old (if >= 0): the Krylov drivers keep
// rho_{k-1} that way without a separate launch.
__global__ void k_final2(int nb, const double* __restrict__ part, double* __restrict__ sc, int s0, int s1,
                         int s0_old, int mode) {
  __shared__ double sh[32];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    if (mode) {
      a = fmax(a, part[i]);
      b = fmax(b, part[nb + i]);
    } else {
      a += part[i];
      b += part[nb + i];
    }
  }
  if (mode) {
    a = block_max(a, sh);
    b = block_max(b, sh);
  } else {
    a = block_sum(a, sh);
    b = block_sum(b, sh);
  }
  if (threadIdx.x == 0) {
    if (s0_old >= 0) sc[s0_old] = sc[s0];
    sc[s0] = a;
    if (s1 >= 0) sc[s1] = b;
  }
}

fvs_status Reducer::init() {
  cudaStream_t st = g_alloc_stream;
  blocks = 8 * sm_count();   // full occupancy for the fused SpMV + reduction kernels
  FVS_TRY(part.alloc(2 * (size_t)blocks));
  FVS_TRY(sc.alloc(S_NSLOT));
  FVS_TRY(sc.zero(st));
  FVS_TRY(ticket.alloc(1));
  FVS_TRY(ticket.zero(st));
  FVS_TRY(iter.alloc(1));
  FVS_TRY(iter.zero(st));
  if (!host) FVS_CUDA(cudaMallocHost(&host, S_NSLOT * sizeof(double)));
  return FVS_OK;
}

fvs_status Reducer::dot(cudaStream_t s, int64_t n, const double* x, const double* y, int slot) {
  k_dot2_part<<<blocks, RB, 0, s>>>(n, x, y, nullptr, nullptr, part); FVS_COUNT_LAUNCH();
  k_final2<<<1, 1024, 0, s>>>(blocks, part, sc, slot, -1, -1, 0); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

fvs_status Reducer::dot2(cudaStream_t s, int64_t n, const double* a, const double* b, const double* c,
                         const double* d, int s0, int s1) {
  k_dot2_part<<<blocks, RB, 0, s>>>(n, a, b, c, d, part); FVS_COUNT_LAUNCH();
  k_final2<<<1, 1024, 0, s>>>(blocks, part, sc, s0, s1, -1, 0); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

fvs_status Reducer::max_abs_diff2(cudaStream_t s, int64_t n, const double* a, const double* b,
                                  const double* c, const double* d, int s0, int s1) {
  k_maxdiff2_part<<<blocks, RB, 0, s>>>(n, a, b, c, d, part); FVS_COUNT_LAUNCH();
  k_final2<<<1, 1024, 0, s>>>(blocks, part, sc, s0, s1, -1, 1); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

fvs_status Reducer::fetch(cudaStream_t s) {
  FVS_CUDA(cudaMemcpyAsync(host, sc.p, S_NSLOT * sizeof(double), cudaMemcpyDeviceToHost, s));
  FVS_CUDA(cudaStreamSynchronize(s));
  return FVS_OK;
}

// ---------------------------------------------------------------------------
// vector kernels
// ---------------------------------------------------------------------------
#define GRID_STRIDE(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

__global__ void k_copy(int64_t n, const double* __restrict__ a, double* __restrict__ b) {
  GRID_STRIDE(i, n) b[i] = a[i];
}
__global__ void k_fill(int64_t n, double v, double* __restrict__ a) {
  GRID_STRIDE(i, n) a[i] = v;
}
fvs_status vcopy(cudaStream_t s, int64_t n, const double* a, double* b) {
  if (n <= 0) return FVS_OK;
  k_copy<<<stride_grid(n, 256), 256, 0, s>>>(n, a, b); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}
fvs_status vfill(cudaStream_t s, int64_t n, double v, double* a) {
  if (n <= 0) return FVS_OK;
  k_fill<<<stride_grid(n, 256), 256, 0, s>>>(n, v, a); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

__global__ void k_jacobi_apply(int64_t n, const double* __restrict__ diag, const double* __restrict__ dextra,
                               const double* __restrict__ r, double* __restrict__ z) {
  GRID_STRIDE(i, n) {
    const double d = diag[i] + (dextra ? dextra[i] : 0.0);
    z[i] = r[i] / d;
  }
}

// z = dinv r: the inverse diagonal is formed once per linear system by its
// owner (an FP64 division per row per application costs more than the
// memory traffic of this kernel on this part)
__global__ void k_jacobi_mul(int64_t n, const double* __restrict__ dinv, const double* __restrict__ r,
                             double* __restrict__ z) {
  GRID_STRIDE(i, n) z[i] = dinv[i] * r[i];
}

fvs_status JacobiPrecond::apply(cudaStream_t s, const double* r, double* z) {
  if (A->n == 0) return FVS_OK;
  if (dinv) k_jacobi_mul<<<stride_grid(A->n, 256), 256, 0, s>>>(A->n, dinv, r, z);
  else k_jacobi_apply<<<stride_grid(A->n, 256), 256, 0, s>>>(A->n, A->diag, dextra, r, z);
  FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

fvs_status KrylovWork::ensure(int64_t n) {
  const size_t m = (size_t)n + 1;
  FVS_TRY(r.alloc(m)); FVS_TRY(rh.alloc(m)); FVS_TRY(p.alloc(m)); FVS_TRY(ph.alloc(m));
  FVS_TRY(v.alloc(m)); FVS_TRY(sv.alloc(m)); FVS_TRY(sh.alloc(m)); FVS_TRY(t.alloc(m));
  FVS_TRY(z.alloc(m)); FVS_TRY(q.alloc(m));
  return FVS_OK;
}

// safe quotient for Krylov scalars (a breakdown shows up as a stalled residual)
__device__ __forceinline__ double sdiv(double a, double b) { return b != 0.0 ? a / b : 0.0; }

// ---------------------------------------------------------------------------
// Fused reductions: every block writes its partial sums; the last block to
// finish (ticket) adds the partials in block order, so the result does not
// depend on scheduling, and then applies the scalar bookkeeping.
// ---------------------------------------------------------------------------
enum { FIN_RV = 0, FIN_TSTT = 1, FIN_RR_RHO = 2, FIN_PQ = 3, FIN_RR = 4, FIN_RZ = 5 };

__device__ void finish2(double a, double b, double* part, unsigned int* ticket, double* sc, int mode) {
  __shared__ double sh[32];
  __shared__ bool last;
  a = block_sum(a, sh);
  b = block_sum(b, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = a;
    part[gridDim.x + blockIdx.x] = b;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double x = 0.0, y = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    x += ((volatile double*)part)[i];
    y += ((volatile double*)part)[gridDim.x + i];
  }
  x = block_sum(x, sh);
  y = block_sum(y, sh);
  if (threadIdx.x == 0) {
    switch (mode) {
      case FIN_RV: sc[S_RV] = x; break;
      case FIN_TSTT: sc[S_TS] = x; sc[S_TT] = y; break;
      case FIN_RR_RHO:
        // alpha and omega of this iteration are kept for the next beta
        sc[S_ALPHA] = sdiv(sc[S_RHO], sc[S_RV]);
        sc[S_OMEGA] = sdiv(sc[S_TS], sc[S_TT]);
        sc[S_RR] = x;
        sc[S_RHO_OLD] = sc[S_RHO];
        sc[S_RHO] = y;
        sc[S_FIRST] = 0.0;
        break;
      case FIN_PQ: sc[S_PQ] = x; break;
      case FIN_RR: sc[S_RR] = x; sc[S_FIRST] = 0.0; break;
      case FIN_RZ: sc[S_RZ_OLD] = sc[S_RZ]; sc[S_RZ] = x; break;
    }
    *ticket = 0u;
  }
}

// y = A x (+ dextra x); sums d.y (and y.y when YY)
template <int MODE, bool YY, bool DX>
__global__ void __launch_bounds__(256, 8) k_spmv_dot(int64_t n, int w, const int32_t* __restrict__ col,
                                                     const double* __restrict__ val, const double* __restrict__ x,
                                                     double* __restrict__ y, const double* __restrict__ dextra,
                                                     const double* __restrict__ d, double* part,
                                                     unsigned int* ticket, double* sc) {
  double a = 0.0, b = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double acc = ell_row(n, w, col, val, x, i, DX ? dextra[i] * x[i] : 0.0);
    y[i] = acc;
    a = fma(d[i], acc, a);
    if (YY) b = fma(acc, acc, b);
  }
  finish2(a, b, part, ticket, sc, MODE);
}

// BiCGStab: x += alpha ph + omega sh ; r = s - omega t ; sums r.r and rh.r
__global__ void k_bicg_xr_dot(int64_t n, double* __restrict__ sc, const double* __restrict__ ph,
                              const double* __restrict__ sh, const double* __restrict__ sv,
                              const double* __restrict__ t, const double* __restrict__ rh, double* __restrict__ x,
                              double* __restrict__ r, double* part, unsigned int* ticket) {
  const double alpha = sdiv(sc[S_RHO], sc[S_RV]);
  const double omega = sdiv(sc[S_TS], sc[S_TT]);
  double a = 0.0, b = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * ph[i] + omega * sh[i];
    const double ri = sv[i] - omega * t[i];
    r[i] = ri;
    a = fma(ri, ri, a);
    b = fma(rh[i], ri, b);
  }
  finish2(a, b, part, ticket, sc, FIN_RR_RHO);
}

// CG: x += alpha p ; r -= alpha q ; sums r.r
__global__ void k_cg_xr_dot(int64_t n, double* __restrict__ sc, const double* __restrict__ p,
                            const double* __restrict__ q, double* __restrict__ x, double* __restrict__ r,
                            double* part, unsigned int* ticket) {
  const double alpha = sdiv(sc[S_RZ], sc[S_PQ]);
  double a = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    a = fma(ri, ri, a);
  }
  finish2(a, 0.0, part, ticket, sc, FIN_RR);
}
// sums r.z (rz moved to rz_old)
__global__ void k_dot_rz(int64_t n, const double* __restrict__ r, const double* __restrict__ z, double* part,
                         unsigned int* ticket, double* sc) {
  double a = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a = fma(r[i], z[i], a);
  finish2(a, 0.0, part, ticket, sc, FIN_RZ);
}

// BiCGStab: p = r + beta (p - omega v), beta = (rho/rho_old)(alpha/omega)
__global__ void k_bicg_p(int64_t n, const double* __restrict__ sc, const double* __restrict__ r,
                         const double* __restrict__ v, double* __restrict__ p, int first) {
  first = first || sc[S_FIRST] != 0.0;
  const double beta = first ? 0.0 : sdiv(sc[S_RHO], sc[S_RHO_OLD]) * sdiv(sc[S_ALPHA], sc[S_OMEGA]);
  const double om = sc[S_OMEGA];
  GRID_STRIDE(i, n) p[i] = first ? r[i] : r[i] + beta * (p[i] - om * v[i]);
}
// s = r - alpha v, alpha = rho / (rh . v)
__global__ void k_bicg_s(int64_t n, const double* __restrict__ sc, const double* __restrict__ r,
                         const double* __restrict__ v, double* __restrict__ sv) {
  const double alpha = sdiv(sc[S_RHO], sc[S_RV]);
  GRID_STRIDE(i, n) sv[i] = r[i] - alpha * v[i];
}
__global__ void k_cg_p(int64_t n, const double* __restrict__ sc, const double* __restrict__ z,
                       double* __restrict__ p, int first) {
  first = first || sc[S_FIRST] != 0.0;
  const double beta = first ? 0.0 : sdiv(sc[S_RZ], sc[S_RZ_OLD]);
  GRID_STRIDE(i, n) p[i] = first ? z[i] : z[i] + beta * p[i];
}

static inline bool bad(double v) { return !(v == v) || v > 1e300 || v < -1e300; }

static fvs_status spmv_dot(cudaStream_t s, Reducer& red, const Ell& A, const double* x, double* y,
                           const double* dextra, const double* d, bool yy, int mode) {
  ProfScope ps(&A, "spmv", (double)A.n * (12.0 * A.w + 24.0 + (dextra ? 8.0 : 0.0)), s);
#define FVS_SPMV_DOT(M_, Y_, D_) \
  k_spmv_dot<M_, Y_, D_><<<red.blocks, 256, 0, s>>>(A.n, A.w, A.col, A.val, x, y, dextra, d, red.part, red.ticket, red.sc)
  if (mode == FIN_RV) { if (dextra) FVS_SPMV_DOT(FIN_RV, false, true); else FVS_SPMV_DOT(FIN_RV, false, false); }
  else if (mode == FIN_TSTT) { if (dextra) FVS_SPMV_DOT(FIN_TSTT, true, true); else FVS_SPMV_DOT(FIN_TSTT, true, false); }
  else { if (dextra) FVS_SPMV_DOT(FIN_PQ, false, true); else FVS_SPMV_DOT(FIN_PQ, false, false); }
#undef FVS_SPMV_DOT
  (void)yy;
  FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

// ---------------------------------------------------------------------------
// CUDA-graph replay of one Krylov iteration (launch overhead dominates the
// small levels of the V-cycle and small meshes).  The first iteration runs
// eagerly; the next ones replay a captured graph while its key (operator,
// vectors, preconditioner state) is unchanged.  Disabled while kernels are
// being timed and by FVS_NO_GRAPHS.
// ---------------------------------------------------------------------------
bool graphs_enabled() {
  static int cached = -1;
  if (cached < 0) cached = getenv("FVS_NO_GRAPHS") ? 0 : 1;
  return cached == 1 && !(g_prof && g_prof->on);
}

static uint64_t mixk(uint64_t h, uint64_t v) {
  h ^= v + 0x9e3779b97f4a7c15ULL + (h << 6) + (h >> 2);
  return h;
}

static uint64_t graph_key(const Ell& A, const double* dextra, const Precond& M, const double* b, const double* x,
                          const KrylovWork& w, const Reducer& red) {
  uint64_t h = 1469598103934665603ULL;
  h = mixk(h, (uint64_t)(uintptr_t)A.val.p);
  h = mixk(h, (uint64_t)(uintptr_t)A.col.p);
  h = mixk(h, (uint64_t)A.n * 131 + (uint64_t)A.w);
  h = mixk(h, (uint64_t)(uintptr_t)dextra);
  h = mixk(h, M.signature());
  h = mixk(h, (uint64_t)(uintptr_t)b);
  h = mixk(h, (uint64_t)(uintptr_t)x);
  h = mixk(h, (uint64_t)(uintptr_t)w.r.p);
  h = mixk(h, (uint64_t)(uintptr_t)w.p.p);
  h = mixk(h, (uint64_t)(uintptr_t)red.sc.p);
  h = mixk(h, (uint64_t)(uintptr_t)red.part.p);
  return h ? h : 1;
}

template <typename F>
static fvs_status run_body(cudaStream_t s, IterGraph* g, uint64_t key, bool first, F& body) {
  if (first || !g || g->disabled || !graphs_enabled() || s == nullptr) return body(first);
  if (!g->exec || g->key != key) {
    g->reset();
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      g->disabled = true;
      return body(first);
    }
    const unsigned long long before = __atomic_load_n(&g_launches, __ATOMIC_RELAXED);
    fvs_status r = body(false);
    g->kernels = __atomic_load_n(&g_launches, __ATOMIC_RELAXED) - before;
    __atomic_sub_fetch(&g_launches, g->kernels, __ATOMIC_RELAXED);   // counted when replayed
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (r != FVS_OK || e != cudaSuccess || !graph) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      g->disabled = true;
      return body(first);
    }
    e = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      cudaGetLastError();
      g->exec = nullptr;
      g->disabled = true;
      return body(first);
    }
    g->key = key;
  }
  FVS_CUDA(cudaGraphLaunch(g->exec, s));
  __atomic_add_fetch(&g_launches, g->kernels, __ATOMIC_RELAXED);
  return FVS_OK;
}

// Loop controllers: the last node of each iteration decides on the device
// whether the conditional while-node runs the body again (no host round
// trip per iteration).  Bounded by maxit; a NaN residual or a breakdown of
// the BiCGStab recurrence also stops the loop (the host then restarts or
// reports).
__global__ void k_ctl_bicg(cudaGraphConditionalHandle h, double* sc, int* it, int maxit) {
  const int n = ++(*it);
  sc[S_ITER] = (double)n;
  const double rr = sc[S_RR];
  const bool go = n < maxit && rr > sc[S_TOL2] && rr == rr && rr < 1e300 && sc[S_TT] != 0.0 &&
                  sc[S_RV] != 0.0 && sc[S_RHO] != 0.0;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}
__global__ void k_ctl_cg(cudaGraphConditionalHandle h, double* sc, int* it, int maxit) {
  const int n = ++(*it);
  sc[S_ITER] = (double)n;
  const double rr = sc[S_RR];
  const bool go = n < maxit && rr > sc[S_TOL2] && rr == rr && rr < 1e300;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}
__global__ void k_loop_init(double* sc, int* it, double tol2, int fresh) {
  sc[S_FIRST] = fresh ? 1.0 : 0.0;
  *it = 0;
  sc[S_ITER] = 0.0;
  sc[S_TOL2] = tol2;
}

// Runs up to maxit iterations of body() as one graph launch with a
// conditional while-node; returns false (nothing launched) when the loop
// graph cannot be used, so the caller iterates from the host instead.
template <typename F>
static bool run_loop(cudaStream_t s, IterGraph* g, uint64_t key, Reducer& red, double tol2, int maxit, bool bicg, bool fresh,
                     F& body, fvs_status& st) {
  st = FVS_OK;
  if (!g || g->loop_disabled || !graphs_enabled() || s == nullptr || maxit <= 0) return false;
  if (!g->loop || g->loop_key != key) {
    if (g->loop) cudaGraphExecDestroy(g->loop);
    g->loop = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphConditionalHandle h;
    bool ok = cudaGraphCreate(&graph, 0) == cudaSuccess;
    ok = ok && cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    cudaGraphNodeParams p = {};
    cudaGraphNode_t node;
    if (ok) {
      p.type = cudaGraphNodeTypeConditional;
      p.conditional.handle = h;
      p.conditional.type = cudaGraphCondTypeWhile;
      p.conditional.size = 1;
      ok = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &p) == cudaSuccess;
    }
    if (ok) {
      cudaGraph_t bodyg = p.conditional.phGraph_out[0];
      ok = cudaStreamBeginCaptureToGraph(s, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
           cudaSuccess;
      if (ok) {
        const unsigned long long before = __atomic_load_n(&g_launches, __ATOMIC_RELAXED);
        fvs_status r = body(false);
        if (bicg)
          k_ctl_bicg<<<1, 1, 0, s>>>(h, red.sc.p, red.iter.p, maxit);
        else
          k_ctl_cg<<<1, 1, 0, s>>>(h, red.sc.p, red.iter.p, maxit);
        g->loop_kernels = __atomic_load_n(&g_launches, __ATOMIC_RELAXED) - before + 1;
        __atomic_sub_fetch(&g_launches, g->loop_kernels - 1, __ATOMIC_RELAXED);
        cudaGraph_t out = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s, &out);
        ok = r == FVS_OK && e == cudaSuccess;
      }
    }
    if (ok) ok = cudaGraphInstantiate(&g->loop, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
      cudaGetLastError();
      if (g->loop) cudaGraphExecDestroy(g->loop);
      g->loop = nullptr;
      g->loop_disabled = true;
      return false;
    }
    g->loop_key = key;
  }
  k_loop_init<<<1, 1, 0, s>>>(red.sc.p, red.iter.p, tol2, fresh ? 1 : 0);
  FVS_COUNT_LAUNCH();
  const cudaError_t e = cudaGraphLaunch(g->loop, s);
  if (e != cudaSuccess) {
    set_error("cudaGraphLaunch: %s", cudaGetErrorString(e));
    st = FVS_ERR_CUDA;
  }
  return true;
}

fvs_status bicgstab(cudaStream_t s, Reducer& red, KrylovWork& w, const Ell& A, const double* dextra,
                    Precond& M, const double* b, double* x, double rtol, int maxit, Projector* proj,
                    SolveResult& res, double bnorm_floor, IterGraph* graph) {
  const int64_t n = A.n;
  res = SolveResult();
  if (n == 0) {
    res.converged = true;
    return FVS_OK;
  }
  FVS_TRY(w.ensure(n));
  const int grid = stride_grid(n, 256);
  FVS_TRY(residual(s, A, x, b, w.r, dextra));
  if (proj) FVS_TRY(proj->apply(s, w.r));
  FVS_TRY(vcopy(s, n, w.r, w.rh));
  // ||b|| of the (projected) right side; rho_0 = rh . r
  const double* bb = b;
  if (proj) {
    FVS_TRY(vcopy(s, n, b, w.q));
    FVS_TRY(proj->apply(s, w.q));
    bb = w.q;
  }
  FVS_TRY(red.dot2(s, n, bb, bb, w.r, w.r, S_BB, S_RR));
  FVS_TRY(red.dot(s, n, w.rh, w.r, S_RHO));
  FVS_TRY(red.fetch(s));
  double bnorm = fmax(sqrt(red.host[S_BB]), bnorm_floor);
  if (bnorm == 0.0) bnorm = 1.0;
  double rn = sqrt(red.host[S_RR]);
  res.relres = rn / bnorm;
  if (bad(rn) || bad(bnorm)) return FVS_OK;   // non-finite data: not converged, no iterations
  if (res.relres <= rtol) {
    res.converged = true;
    return FVS_OK;
  }
  // K x has zero sum on every singular part (zero column sums), so the
  // Krylov vectors stay in the range once r is projected
  auto body = [&](bool first) -> fvs_status {
    k_bicg_p<<<grid, 256, 0, s>>>(n, red.sc, w.r, w.v, w.p, first ? 1 : 0); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    FVS_TRY(M.apply(s, w.p, w.ph));
    FVS_TRY(spmv_dot(s, red, A, w.ph, w.v, dextra, w.rh, false, FIN_RV));
    k_bicg_s<<<grid, 256, 0, s>>>(n, red.sc, w.r, w.v, w.sv); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    FVS_TRY(M.apply(s, w.sv, w.sh));
    FVS_TRY(spmv_dot(s, red, A, w.sh, w.t, dextra, w.sv, true, FIN_TSTT));
    k_bicg_xr_dot<<<red.blocks, 256, 0, s>>>(n, red.sc, w.ph, w.sh, w.sv, w.t, w.rh, x, w.r, red.part,
                                              red.ticket); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    return FVS_OK;
  };
  const uint64_t key = graph_key(A, dextra, M, b, x, w, red) ^ 0x6b696367ULL;
  // the first iteration of a recurrence runs from the host; the following
  // ones run as one device-driven loop (or one graph replay per iteration)
  bool fresh = true;
  int it = 0;
  const double tol2 = (rtol * bnorm) * (rtol * bnorm);
  while (it < maxit) {
    bool looped = false;
    {
      fvs_status st = FVS_OK;
      looped = run_loop(s, graph, key, red, tol2, maxit - it, true, fresh, body, st);
      FVS_TRY(st);
    }
    if (!looped) FVS_TRY(run_body(s, graph, key, fresh, body));
    fresh = false;
    FVS_TRY(red.fetch(s));
    const int done = looped ? (int)red.host[S_ITER] : 1;
    if (looped) __atomic_add_fetch(&g_launches, graph->loop_kernels * (unsigned long long)done, __ATOMIC_RELAXED);
    it += done;
    rn = sqrt(red.host[S_RR]);
    res.iters = it;
    res.relres = rn / bnorm;
    if (bad(rn)) return FVS_OK;
    if (res.relres <= rtol) {
      res.converged = true;
      break;
    }
    // restart on breakdown of the shadow residual
    if (red.host[S_TT] == 0.0 || red.host[S_RV] == 0.0 || red.host[S_RHO] == 0.0) {
      FVS_TRY(residual(s, A, x, b, w.r, dextra));
      if (proj) FVS_TRY(proj->apply(s, w.r));
      FVS_TRY(vcopy(s, n, w.r, w.rh));
      FVS_TRY(red.dot(s, n, w.rh, w.r, S_RHO));
      fresh = true;
    }
  }
  // recompute the true residual (the recursive one drifts)
  FVS_TRY(residual(s, A, x, b, w.r, dextra));
  if (proj) FVS_TRY(proj->apply(s, w.r));
  FVS_TRY(red.dot(s, n, w.r, w.r, S_RR));
  FVS_TRY(red.fetch(s));
  res.relres = sqrt(red.host[S_RR]) / bnorm;
  res.converged = res.relres <= rtol * 10.0 && !bad(res.relres);
  return FVS_OK;
}

// ---------------------------------------------------------------------------
// preconditioned CG (symmetric systems)
// ---------------------------------------------------------------------------
fvs_status pcg(cudaStream_t s, Reducer& red, KrylovWork& w, const Ell& A, Precond& M, const double* b,
               double* x, double rtol, int maxit, Projector* proj, SolveResult& res, IterGraph* graph) {
  const int64_t n = A.n;
  res = SolveResult();
  if (n == 0) {
    res.converged = true;
    return FVS_OK;
  }
  FVS_TRY(w.ensure(n));
  const int grid = stride_grid(n, 256);
  FVS_TRY(residual(s, A, x, b, w.r, nullptr));
  if (proj) FVS_TRY(proj->apply(s, w.r));
  const double* bb = b;
  if (proj) {
    FVS_TRY(vcopy(s, n, b, w.q));
    FVS_TRY(proj->apply(s, w.q));
    bb = w.q;
  }
  FVS_TRY(red.dot2(s, n, bb, bb, w.r, w.r, S_BB, S_RR));
  FVS_TRY(red.fetch(s));
  double bnorm = sqrt(red.host[S_BB]);
  if (bnorm == 0.0) bnorm = 1.0;
  res.relres = sqrt(red.host[S_RR]) / bnorm;
  if (bad(res.relres) || bad(bnorm)) return FVS_OK;   // non-finite data: not converged
  if (res.relres <= rtol) {
    res.converged = true;
    return FVS_OK;
  }
  auto body = [&](bool first) -> fvs_status {
    FVS_TRY(M.apply(s, w.r, w.z));
    if (proj) FVS_TRY(proj->apply(s, w.z));
    k_dot_rz<<<red.blocks, 256, 0, s>>>(n, w.r, w.z, red.part, red.ticket, red.sc); FVS_COUNT_LAUNCH();
    k_cg_p<<<grid, 256, 0, s>>>(n, red.sc, w.z, w.p, first ? 1 : 0); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    FVS_TRY(spmv_dot(s, red, A, w.p, w.q, nullptr, w.p, false, FIN_PQ));
    k_cg_xr_dot<<<red.blocks, 256, 0, s>>>(n, red.sc, w.p, w.q, x, w.r, red.part, red.ticket); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    return FVS_OK;
  };
  const uint64_t key = graph_key(A, nullptr, M, b, x, w, red) ^ (proj ? 0x70636770ULL : 0x70636700ULL);
  const double tol2 = (rtol * bnorm) * (rtol * bnorm);
  for (int it = 0; it < maxit;) {
    bool looped = false;
    {
      fvs_status st = FVS_OK;
      looped = run_loop(s, graph, key, red, tol2, maxit - it, false, it == 0, body, st);
      FVS_TRY(st);
    }
    if (!looped) FVS_TRY(run_body(s, graph, key, it == 0, body));
    FVS_TRY(red.fetch(s));
    const int done = looped ? (int)red.host[S_ITER] : 1;
    if (looped) __atomic_add_fetch(&g_launches, graph->loop_kernels * (unsigned long long)done, __ATOMIC_RELAXED);
    it += done;
    const double rn = sqrt(red.host[S_RR]);
    res.iters = it;
    res.relres = rn / bnorm;
    if (bad(rn)) return FVS_OK;
    if (res.relres <= rtol) {
      res.converged = true;
      break;
    }
  }
  FVS_TRY(residual(s, A, x, b, w.r, nullptr));
  if (proj) FVS_TRY(proj->apply(s, w.r));
  FVS_TRY(red.dot(s, n, w.r, w.r, S_RR));
  FVS_TRY(red.fetch(s));
  res.relres = sqrt(red.host[S_RR]) / bnorm;
  res.converged = res.relres <= rtol * 10.0 && !bad(res.relres);
  return FVS_OK;
}

}  // namespace fvs
