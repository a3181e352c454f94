// Lockstep batch of plain solves (Section 2.7 sampling; every sample follows
// Section 2.2 steps 1-5 and the Eq. 22-23 outputs).  See batch.cuh for the
// layout.  All kernels here run over (rows x samples) with blocks of 32
// samples x 8 rows: a warp covers 32 consecutive samples of one row.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "batch.cuh"
#include "fslaw.cuh"
#include "solver.cuh"

namespace fvs {

// rows of this thread (blockDim = (32, 8)); the sample is blockIdx.y*32 + threadIdx.x
#define BROW(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; i < (n); i += (int64_t)gridDim.x * blockDim.y)
#define BSAMPLE const int s = blockIdx.y * 32 + threadIdx.x

static inline dim3 bblock() { return dim3(32, 8, 1); }
// launch shape of the operator kernels (chosen by the tuner at set-up)
static inline dim3 sblock(const BShape* sh) { return dim3(32, sh ? sh->rows : 8, 1); }
static inline dim3 sgrid(int64_t n, int tiles, const BShape* sh) {
  const int rows = sh ? sh->rows : 8, per_sm = sh ? sh->per_sm : 16;
  const int64_t rb = (n + rows - 1) / rows;
  const int64_t cap = std::max<int64_t>(1, (int64_t)sm_count() * per_sm / tiles);
  return dim3((unsigned)std::max<int64_t>(1, std::min(rb, cap)), (unsigned)tiles, 1);
}
// elementwise grids: about 16 blocks per SM in total
static inline dim3 bgrid(int64_t n, int tiles) {
  int64_t rb = (n + 7) / 8;
  int64_t cap = std::max<int64_t>(1, (int64_t)sm_count() * 16 / tiles);
  return dim3((unsigned)std::max<int64_t>(1, std::min(rb, cap)), (unsigned)tiles, 1);
}

__device__ __forceinline__ double bsdiv(double a, double b) { return b != 0.0 ? a / b : 0.0; }

template <typename T>
static inline void dswap_b(DBuf<T>& a, DBuf<T>& b) {
  T* p = a.p;
  const size_t n = a.n;
  a.p = b.p;
  a.n = b.n;
  b.p = p;
  b.n = n;
}

// ---------------------------------------------------------------------------
// deterministic per-sample reductions: block partials (fixed order over the
// 8 row lanes), then one pass per sample over the blocks in fixed order
// ---------------------------------------------------------------------------
// The block of a tile (group of 32 samples) that finishes last adds the
// tile's partials in fixed block order -- lane y takes blocks y, y+8, ...,
// then the lanes combine in fixed order, whatever block is last -- writes
// sc[slot*Sp + s] and resets the tile's counter (so graph replays start from
// zero).  Partials are read past L1 (other SMs wrote them).
__device__ __forceinline__ void kb_last_block_final(int Sp, const double* part, double* sc, int slot0, int slot1,
                                                    int take_max, int* cnt, double (*sh)[8][33]) {
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) last = atomicAdd(&cnt[blockIdx.y], 1) == (int)gridDim.x - 1 ? 1 : 0;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int nb = (int)gridDim.x;
  const int s = blockIdx.y * 32 + threadIdx.x;
  double u = 0.0, v = 0.0;
  for (int b = threadIdx.y; b < nb; b += 8) {
    const double pu = __ldcg(part + (int64_t)b * Sp + s), pv = __ldcg(part + ((int64_t)nb + b) * Sp + s);
    if (take_max) { u = fmax(u, pu); v = fmax(v, pv); } else { u += pu; v += pv; }
  }
  sh[0][threadIdx.y][threadIdx.x] = u;
  sh[1][threadIdx.y][threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.y == 0) {
    u = sh[0][0][threadIdx.x];
    v = sh[1][0][threadIdx.x];
    for (int k = 1; k < 8; ++k) {
      if (take_max) { u = fmax(u, sh[0][k][threadIdx.x]); v = fmax(v, sh[1][k][threadIdx.x]); }
      else { u += sh[0][k][threadIdx.x]; v += sh[1][k][threadIdx.x]; }
    }
    if (slot0 >= 0) sc[slot0 * Sp + s] = u;
    if (slot1 >= 0) sc[slot1 * Sp + s] = v;
  }
  if (threadIdx.x == 0 && threadIdx.y == 0) cnt[blockIdx.y] = 0;
}
__global__ void kb_dot2(int64_t n, int Sp, const double* a, const double* b, const double* c, const double* d,
                        double* part, double* sc, int slot0, int slot1, int* cnt) {
  __shared__ double sh[2][8][33];
  BSAMPLE;
  double x = 0.0, y = 0.0;
  BROW(i, n) {
    const int64_t e = i * Sp + s;
    x = fma(a[e], b[e], x);
    if (c) y = fma(c[e], d[e], y);
  }
  sh[0][threadIdx.y][threadIdx.x] = x;
  sh[1][threadIdx.y][threadIdx.x] = y;
  __syncthreads();
  if (threadIdx.y == 0) {
    double u = 0.0, v = 0.0;
    for (int k = 0; k < 8; ++k) { u += sh[0][k][threadIdx.x]; v += sh[1][k][threadIdx.x]; }
    part[(int64_t)blockIdx.x * Sp + s] = u;
    part[((int64_t)gridDim.x + blockIdx.x) * Sp + s] = v;
  }
  __syncthreads();
  kb_last_block_final(Sp, part, sc, slot0, slot1, 0, cnt, sh);
}
// max |a - b| and max |c - d| per sample
__global__ void kb_maxdiff2(int64_t n, int Sp, const double* a, const double* b, const double* c, const double* d,
                            double* part, double* sc, int slot0, int slot1, int* cnt) {
  __shared__ double sh[2][8][33];
  BSAMPLE;
  double x = 0.0, y = 0.0;
  BROW(i, n) {
    const int64_t e = i * Sp + s;
    x = fmax(x, fabs(a[e] - b[e]));
    y = fmax(y, fabs(c[e] - d[e]));
  }
  sh[0][threadIdx.y][threadIdx.x] = x;
  sh[1][threadIdx.y][threadIdx.x] = y;
  __syncthreads();
  if (threadIdx.y == 0) {
    double u = 0.0, v = 0.0;
    for (int k = 0; k < 8; ++k) { u = fmax(u, sh[0][k][threadIdx.x]); v = fmax(v, sh[1][k][threadIdx.x]); }
    part[(int64_t)blockIdx.x * Sp + s] = u;
    part[((int64_t)gridDim.x + blockIdx.x) * Sp + s] = v;
  }
  __syncthreads();
  kb_last_block_final(Sp, part, sc, slot0, slot1, 1, cnt, sh);
}

// ---------------------------------------------------------------------------
// operators: y = A x for (row, sample).  The neighbour values come from a
// gather functor: straight from x in global memory, or from the block's
// staged copy in shared memory (XStage).
// ---------------------------------------------------------------------------
template <typename V>
struct GatherGlobal {
  const V* x;
  const int32_t* col;
  int Sp, s;
  __device__ __forceinline__ V operator()(int64_t q) const { return x[(int64_t)col[q] * Sp + s]; }
};
template <typename V>
struct GatherStaged {
  const V* xs;          // [u][32] in shared memory
  const uint8_t* li;
  int lane;
  __device__ __forceinline__ V operator()(int64_t q) const { return xs[(int)li[q] * 32 + lane]; }
};
// acc + sum_{k < len} vf(k) g(k n + i), in slot order: the gathers of CH
// consecutive entries are issued before their multiply-adds, so a thread
// waits on one round of loads per CH entries instead of one per entry (the
// batched operators are bound by that latency: a warp serves one row of 32
// samples, and its loads are few and small)
constexpr int BCH = 9;
template <typename V, class G, class VF>
__device__ __forceinline__ V chunked_sum(int64_t n, int len, int64_t i, const G& g, const VF& vf, V acc) {
  int k = 0;
  for (; k + BCH <= len; k += BCH) {
    V xv[BCH];
#pragma unroll
    for (int c = 0; c < BCH; ++c) xv[c] = g((int64_t)(k + c) * n + i);
#pragma unroll
    for (int c = 0; c < BCH; ++c) acc = fma(vf(k + c), xv[c], acc);
  }
  if (k < len) {
    // the last, partial chunk (every row of a face-only stencil, 7 < BCH):
    // its gathers are issued together too, the missing slots re-read slot 0
    V xv[BCH - 1];
#pragma unroll
    for (int c = 0; c < BCH - 1; ++c) xv[c] = g((int64_t)(k + c < len ? k + c : 0) * n + i);
#pragma unroll
    for (int c = 0; c < BCH - 1; ++c)
      if (k + c < len) acc = fma(vf(k + c), xv[c], acc);
  }
  return acc;
}

// shared values: y = dg x + [mask] sum_k val[k][i] x[col]   (mask: solid rows keep dg x only)
struct OpShared {
  int64_t n;
  int w;
  const int32_t* col;
  const double* val;
  const double* dg;       // per (i, s), may be null
  const uint8_t* mask;    // per (i, s), may be null
  template <class G>
  __device__ __forceinline__ double row(int64_t i, int s, int Sp, const double* x, const G& g) const {
    const int64_t e = i * Sp + s;
    double acc = dg ? dg[e] * x[e] : 0.0;
    if (!mask || mask[e]) {
      const double* v = val;
      const int64_t nn = n;
      acc = chunked_sum(n, w, i, g, [v, nn, i](int k) { return v[(int64_t)k * nn + i]; }, acc);
    }
    return acc;
  }
};
// fine pressure operator: identity rows (o = -2), shared base rows (o = -1),
// per-sample re-assembled rows (o >= 0); V = double, or float for the FP32
// V-cycle (accumulation in V)
template <typename V>
struct OpPpe0T {
  int64_t n;
  int w;
  const int32_t* col;
  const V* base;
  const int32_t* ovr;
  const V* mval;
  template <class G>
  __device__ __forceinline__ V row(int64_t i, int s, int Sp, const V* x, const G& g) const {
    const int64_t e = i * Sp + s;
    const int32_t o = ovr[e];
    if (o == -2) return x[e];
    V acc = 0;
    if (o < 0) {
      const V* bv = base;
      const int64_t nn = n;
      acc = chunked_sum(n, w, i, g, [bv, nn, i](int k) { return bv[(int64_t)k * nn + i]; }, acc);
    } else {
      const V* mv = mval + (int64_t)o * w;
      acc = chunked_sum(n, w, i, g, [mv](int k) { return mv[k]; }, acc);
    }
    return acc;
  }
};
using OpPpe0 = OpPpe0T<double>;
// coarse levels: shared pattern, per-sample values
template <typename V>
struct OpCoarseT {
  int64_t n;
  int w;
  const int32_t* col;
  const V* val;
  const int32_t* rlen;   // stored entries per row (padding after), shared by all samples
  template <class G>
  __device__ __forceinline__ V row(int64_t i, int s, int Sp, const V* x, const G& g) const {
    const int len = rlen ? rlen[i] : w;
    const V* v = val;
    const int64_t nn = n;
    return chunked_sum(n, len, i, g, [v, nn, i, Sp, s](int k) { return v[((int64_t)k * nn + i) * Sp + s]; },
                       (V)0);
  }
};
using OpCoarse = OpCoarseT<double>;

// mode 0: y = A x;  1: y = b - A x;  2: y = x + omega dinv (b - A x)
template <class Op, typename V>
__global__ void kb_apply(Op op, int Sp, const V* x, const V* b, V* y, int mode, const V* dinv, V omega) {
  BSAMPLE;
  const GatherGlobal<V> g{x, op.col, Sp, s};
  BROW(i, op.n) {
    const int64_t e = i * Sp + s;
    const V ax = op.row(i, s, Sp, x, g);
    V out;
    if (mode == 0) out = ax;
    else if (mode == 1) out = b[e] - ax;
    else out = x[e] + omega * dinv[e] * (b[e] - ax);
    y[e] = out;
  }
}
// the same with x staged: block (32 samples, R rows) handles rows
// [R blockIdx.x, R blockIdx.x + R) and first loads x of the block's column
// list into shared memory (dynamic, umax x 32 values)
template <class Op, typename V>
__global__ void kb_apply_st(Op op, int Sp, const V* x, const V* b, V* y, int mode, const V* dinv, V omega,
                            const int32_t* uptr, const int32_t* ucol, const uint8_t* li) {
  extern __shared__ __align__(16) unsigned char kb_smem[];
  V* xs = reinterpret_cast<V*>(kb_smem);
  BSAMPLE;
  const int64_t blk = blockIdx.x;
  const int32_t u0 = uptr[blk], nu = uptr[blk + 1] - u0;
  for (int u = threadIdx.y; u < nu; u += blockDim.y) xs[u * 32 + threadIdx.x] = x[(int64_t)ucol[u0 + u] * Sp + s];
  __syncthreads();
  const int64_t i = blk * blockDim.y + threadIdx.y;
  if (i >= op.n) return;
  const GatherStaged<V> g{xs, li, (int)threadIdx.x};
  const int64_t e = i * Sp + s;
  const V ax = op.row(i, s, Sp, x, g);
  V out;
  if (mode == 0) out = ax;
  else if (mode == 1) out = b[e] - ax;
  else out = x[e] + omega * dinv[e] * (b[e] - ax);
  y[e] = out;
}


// ---------------------------------------------------------------------------
// Krylov vector updates with per-sample scalars; samples with act = 0 keep
// their vectors
// ---------------------------------------------------------------------------
__global__ void kb_copy(int64_t len, const double* a, double* b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}
__global__ void kb_scale(int64_t n, int Sp, const double* d, const double* r, double* z) {
  BSAMPLE;
  BROW(i, n) { const int64_t e = i * Sp + s; z[e] = d[e] * r[e]; }
}
__global__ void kb_bicg_p(int64_t n, int Sp, const double* sc, const uint8_t* act, const double* r, const double* v,
                          double* p) {
  BSAMPLE;
  if (!act[s]) return;
  const bool first = sc[B_FIRST * Sp + s] != 0.0;
  const double beta = first ? 0.0
                            : bsdiv(sc[B_RHO * Sp + s], sc[B_RHO_OLD * Sp + s]) *
                                  bsdiv(sc[B_ALPHA * Sp + s], sc[B_OMEGA * Sp + s]);
  const double om = sc[B_OMEGA * Sp + s];
  BROW(i, n) {
    const int64_t e = i * Sp + s;
    p[e] = first ? r[e] : r[e] + beta * (p[e] - om * v[e]);
  }
}
// alpha = rho / (rh . v); s = r - alpha v
__global__ void kb_bicg_s(int64_t n, int Sp, double* sc, const uint8_t* act, const double* r, const double* v,
                          double* sv) {
  BSAMPLE;
  if (!act[s]) return;
  const double alpha = bsdiv(sc[B_RHO * Sp + s], sc[B_RV * Sp + s]);
  if (blockIdx.x == 0 && threadIdx.y == 0) sc[B_ALPHA * Sp + s] = alpha;
  BROW(i, n) {
    const int64_t e = i * Sp + s;
    sv[e] = r[e] - alpha * v[e];
  }
}
// omega = (t . s) / (t . t); x += alpha ph + omega sh; r = s - omega t
__global__ void kb_bicg_xr(int64_t n, int Sp, double* sc, const uint8_t* act, const double* ph, const double* sh,
                           const double* sv, const double* t, double* x, double* r) {
  BSAMPLE;
  if (!act[s]) return;
  const double alpha = bsdiv(sc[B_RHO * Sp + s], sc[B_RV * Sp + s]);
  const double omega = bsdiv(sc[B_TS * Sp + s], sc[B_TT * Sp + s]);
  BROW(i, n) {
    const int64_t e = i * Sp + s;
    x[e] += alpha * ph[e] + omega * sh[e];
    r[e] = sv[e] - omega * t[e];
  }
}
// end of a BiCGStab iteration: omega kept, rho rotated, activity and
// breakdown (restart) per sample; counts[0] samples still active, counts[1] restarts
__global__ void kb_bicg_next(int Sp, double* sc, uint8_t* act, uint8_t* restart, int* counts) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Sp) return;
  restart[s] = 0;
  if (!act[s]) return;
  // sc[B_TMP] slots: the dot of this pass is in B_RR (r.r) and B_RZ (rh.r)
  const double omega = bsdiv(sc[B_TS * Sp + s], sc[B_TT * Sp + s]);
  sc[B_OMEGA * Sp + s] = omega;
  sc[B_RHO_OLD * Sp + s] = sc[B_RHO * Sp + s];
  sc[B_RHO * Sp + s] = sc[B_RZ * Sp + s];
  sc[B_FIRST * Sp + s] = 0.0;
  const double rr = sc[B_RR * Sp + s];
  if (!(rr > sc[B_TOL2 * Sp + s])) { act[s] = 0; return; }
  if (!(rr == rr) || fabs(rr) > 1e300) { act[s] = 0; return; }   // non-finite: stop this sample
  atomicAdd(&counts[0], 1);
  if (sc[B_TT * Sp + s] == 0.0 || sc[B_RV * Sp + s] == 0.0 || sc[B_RHO * Sp + s] == 0.0) {
    restart[s] = 1;
    atomicAdd(&counts[1], 1);
  }
}
// restart of the flagged samples: r and rh from the true residual in t
__global__ void kb_restart(int64_t n, int Sp, const uint8_t* restart, const double* rt, double* r, double* rh) {
  BSAMPLE;
  if (!restart[s]) return;
  BROW(i, n) {
    const int64_t e = i * Sp + s;
    r[e] = rt[e];
    rh[e] = rt[e];
  }
}
__global__ void kb_restart_scalars(int Sp, double* sc, const uint8_t* restart) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Sp || !restart[s]) return;
  sc[B_FIRST * Sp + s] = 1.0;
  sc[B_RHO * Sp + s] = sc[B_RZ * Sp + s];
}
// CG: p = z + (rz/rz_old) p ; after q = A p: x += alpha p, r -= alpha q
__global__ void kb_cg_p(int64_t n, int Sp, const double* sc, const uint8_t* act, const double* z, double* p) {
  BSAMPLE;
  if (!act[s]) return;
  const bool first = sc[B_FIRST * Sp + s] != 0.0;
  const double beta = first ? 0.0 : bsdiv(sc[B_RZ * Sp + s], sc[B_RZ_OLD * Sp + s]);
  BROW(i, n) {
    const int64_t e = i * Sp + s;
    p[e] = first ? z[e] : z[e] + beta * p[e];
  }
}
__global__ void kb_cg_xr(int64_t n, int Sp, const double* sc, const uint8_t* act, const double* p, const double* q,
                         double* x, double* r) {
  BSAMPLE;
  if (!act[s]) return;
  const double alpha = bsdiv(sc[B_RZ * Sp + s], sc[B_PQ * Sp + s]);
  BROW(i, n) {
    const int64_t e = i * Sp + s;
    x[e] += alpha * p[e];
    r[e] -= alpha * q[e];
  }
}
__global__ void kb_cg_next(int Sp, double* sc, uint8_t* act, int* counts) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Sp || !act[s]) return;
  sc[B_RZ_OLD * Sp + s] = sc[B_RZ * Sp + s];
  sc[B_FIRST * Sp + s] = 0.0;
  const double rr = sc[B_RR * Sp + s];
  if (!(rr > sc[B_TOL2 * Sp + s]) || !(rr == rr) || fabs(rr) > 1e300) { act[s] = 0; return; }
  atomicAdd(&counts[0], 1);
}
// start of a solve: tol2 = (rtol max(|b|, floor))^2, active where the
// residual is above it (and the sample takes part)
__global__ void kb_krylov_init(int Sp, double* sc, uint8_t* act, const uint8_t* take, const double* rtol_s,
                               double rtol, const double* floor, int* counts) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Sp) return;
  double bn = sqrt(sc[B_BB * Sp + s]);
  if (floor) bn = fmax(bn, floor[s]);
  if (bn == 0.0) bn = 1.0;
  const double rt = rtol_s ? rtol_s[s] : rtol;
  sc[B_TOL2 * Sp + s] = (rt * bn) * (rt * bn);
  sc[B_BB * Sp + s] = bn * bn;    // the norm the residual is judged against
  sc[B_FIRST * Sp + s] = 1.0;
  sc[B_OMEGA * Sp + s] = 1.0;
  sc[B_ALPHA * Sp + s] = 1.0;
  const bool a = (!take || take[s]) && sc[B_RR * Sp + s] > sc[B_TOL2 * Sp + s];
  act[s] = a ? 1 : 0;
  if (a) atomicAdd(&counts[0], 1);
}

// ---------------------------------------------------------------------------
// V-cycle pieces
// ---------------------------------------------------------------------------
template <typename V>
__global__ void kb_jac0(int64_t n, int Sp, V omega, const V* dinv, const V* b, V* x) {
  BSAMPLE;
  BROW(i, n) { const int64_t e = i * Sp + s; x[e] = omega * dinv[e] * b[e]; }
}
template <typename V>
__global__ void kb_restrict(int64_t nc, int Sp, const int32_t* mptr, const int32_t* midx, const V* r, V* bc) {
  BSAMPLE;
  BROW(I, nc) {
    V a = 0;
    for (int32_t m = mptr[I]; m < mptr[I + 1]; ++m) a += r[(int64_t)midx[m] * Sp + s];
    bc[I * Sp + s] = a;
  }
}
// restriction and the next level's first Jacobi iterate (xc = omega Dc^-1 bc)
template <typename V>
__global__ void kb_restrict_jac0(int64_t nc, int Sp, const int32_t* mptr, const int32_t* midx, const V* r, V* bc,
                                 V omega, const V* dinvc, V* xc) {
  BSAMPLE;
  BROW(I, nc) {
    V a = 0;
    for (int32_t m = mptr[I]; m < mptr[I + 1]; ++m) a += r[(int64_t)midx[m] * Sp + s];
    const int64_t e = I * Sp + s;
    bc[e] = a;
    xc[e] = omega * dinvc[e] * a;
  }
}
// x += scale P yc (rows with ovr == -2 at the fine level take no correction)
template <typename V>
__global__ void kb_prolong(int64_t n, int Sp, const int32_t* agg, const int32_t* ovr, const V* yc, V scale, V* x) {
  BSAMPLE;
  BROW(i, n) {
    const int64_t e = i * Sp + s;
    const int32_t a = agg[i];
    if (a < 0 || (ovr && ovr[e] == -2)) continue;
    x[e] += scale * yc[(int64_t)a * Sp + s];
  }
}
// coarsest: y = Ainv_s b (Ainv with the null-space projections folded in),
// [(i*nc + j)*Sp + s]; FP64 accumulation
template <typename V>
__global__ void kb_coarse_solve(int nc, int Sp, const double* Ainv, const V* b, V* y) {
  BSAMPLE;
  BROW(i, nc) {
    double a = 0.0;
    for (int j = 0; j < nc; ++j) a = fma(Ainv[((int64_t)i * nc + j) * Sp + s], (double)b[(int64_t)j * Sp + s], a);
    y[i * Sp + s] = (V)a;
  }
}
__global__ void kb_to_float(int64_t n, const double* a, float* b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void kb_to_double(int64_t n, const float* a, double* b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

// ---------------------------------------------------------------------------
// per-sample Galerkin values on the shared aggregation: coarse entry q gets
// the sum of the listed fine entries (rows of cells without pressure left out)
// ---------------------------------------------------------------------------
__global__ void kb_galerkin0(int64_t nq, int64_t n, int w, int Sp, const int32_t* gptr, const int32_t* gidx,
                             const double* base, const int32_t* ovr, const double* mval, double* cval) {
  BSAMPLE;
  BROW(q, nq) {
    double a = 0.0;
    for (int32_t t = gptr[q]; t < gptr[q + 1]; ++t) {
      const int32_t e = gidx[t];
      const int32_t k = (int32_t)(e / n), i = (int32_t)(e - (int64_t)k * n);
      const int32_t o = ovr[(int64_t)i * Sp + s];
      if (o == -2) continue;
      a += o < 0 ? base[e] : mval[(int64_t)o * w + k];
    }
    cval[q * Sp + s] = a;
  }
}
__global__ void kb_galerkin(int64_t nq, int Sp, const int32_t* gptr, const int32_t* gidx, const double* val,
                            double* cval) {
  BSAMPLE;
  BROW(q, nq) {
    double a = 0.0;
    for (int32_t t = gptr[q]; t < gptr[q + 1]; ++t) a += val[(int64_t)gidx[t] * Sp + s];
    cval[q * Sp + s] = a;
  }
}
__global__ void kb_coarse_dinv(int64_t n, int Sp, const int32_t* dslot, const double* val, double* dinv) {
  BSAMPLE;
  BROW(i, n) {
    const int32_t k = dslot[i];
    const double d = k >= 0 ? val[((int64_t)k * n + i) * Sp + s] : 0.0;
    dinv[i * Sp + s] = d != 0.0 ? 1.0 / d : 0.0;
  }
}

// ---------------------------------------------------------------------------
// null-space labels and the per-part projection (fine level)
// ---------------------------------------------------------------------------
__global__ void kb_pull_labels(int64_t n, int Sp, const int32_t* agg, const int32_t* ovr, const int32_t* lab_c,
                               int32_t* lab) {
  BSAMPLE;
  BROW(i, n) {
    const int64_t e = i * Sp + s;
    const int32_t a = agg ? agg[i] : (int32_t)i;   // no aggregation: the level is the coarsest
    lab[e] = (a < 0 || (ovr && ovr[e] == -2)) ? -1 : lab_c[(int64_t)a * Sp + s];
  }
}
__global__ void kb_part_count(int64_t n, int Sp, int nc, const int32_t* lab, int* count) {
  BSAMPLE;
  BROW(i, n) {
    const int32_t c = lab[i * Sp + s];
    if (c >= 0) atomicAdd(&count[(int64_t)s * nc + c], 1);
  }
}
// compact ids of the singular parts that hold fine rows (at most BATCH_NCM per sample)
__global__ void kb_part_ids(int Sp, int nc, const int* count, const uint8_t* sing, const int* ncomp, int32_t* cid,
                            double* ccnt, int* err) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Sp) return;
  int k = 0;
  for (int c = 0; c < BATCH_NCM; ++c) ccnt[s * BATCH_NCM + c] = 0.0;
  for (int c = 0; c < nc; ++c) {
    int32_t id = -1;
    if (c < ncomp[s] && sing[(int64_t)c * Sp + s] && count[(int64_t)s * nc + c] > 0) {
      if (k < BATCH_NCM) {
        id = k;
        ccnt[s * BATCH_NCM + k] = (double)count[(int64_t)s * nc + c];
        ++k;
      } else {
        atomicOr(err, 16);
      }
    }
    cid[(int64_t)s * nc + c] = id;
  }
}
__global__ void kb_proj_part(int64_t n, int Sp, int nc, const int32_t* lab, const int32_t* cid, const double* v,
                             double* part, const double* ccnt, double* mean, int* cnt) {
  __shared__ double sh[BATCH_NCM][8][33];
  BSAMPLE;
  double a[BATCH_NCM];
  for (int k = 0; k < BATCH_NCM; ++k) a[k] = 0.0;
  BROW(i, n) {
    const int64_t e = i * Sp + s;
    const int32_t c = lab[e];
    if (c < 0) continue;
    const int32_t k = cid[(int64_t)s * nc + c];
    if (k >= 0) {
#pragma unroll
      for (int q = 0; q < BATCH_NCM; ++q) if (q == k) a[q] += v[e];
    }
  }
#pragma unroll
  for (int k = 0; k < BATCH_NCM; ++k) sh[k][threadIdx.y][threadIdx.x] = a[k];
  __syncthreads();
  if (threadIdx.y == 0) {
    for (int k = 0; k < BATCH_NCM; ++k) {
      double u = 0.0;
      for (int y = 0; y < 8; ++y) u += sh[k][y][threadIdx.x];
      part[((int64_t)k * gridDim.x + blockIdx.x) * Sp + s] = u;
    }
  }
  // the tile's last block forms the per-part means (fixed block order)
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) last = atomicAdd(&cnt[blockIdx.y], 1) == (int)gridDim.x - 1 ? 1 : 0;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int nb = (int)gridDim.x;
  for (int k = 0; k < BATCH_NCM; ++k) {
    const double c = ccnt[s * BATCH_NCM + k];
    double u = 0.0;
    if (c > 0.0)
      for (int b = threadIdx.y; b < nb; b += 8) u += __ldcg(part + ((int64_t)k * nb + b) * Sp + s);
    sh[0][threadIdx.y][threadIdx.x] = u;
    __syncthreads();
    if (threadIdx.y == 0) {
      double t = 0.0;
      for (int y = 0; y < 8; ++y) t += sh[0][y][threadIdx.x];
      mean[s * BATCH_NCM + k] = c > 0.0 ? t / c : 0.0;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && threadIdx.y == 0) cnt[blockIdx.y] = 0;
}
__global__ void kb_proj_sub(int64_t n, int Sp, int nc, const int32_t* lab, const int32_t* cid, const double* mean,
                            double* v) {
  BSAMPLE;
  BROW(i, n) {
    const int64_t e = i * Sp + s;
    const int32_t c = lab[e];
    if (c < 0) continue;
    const int32_t k = cid[(int64_t)s * nc + c];
    if (k >= 0) v[e] -= mean[s * BATCH_NCM + k];
  }
}

// ---------------------------------------------------------------------------
// host side: buffers, reductions
// ---------------------------------------------------------------------------
fvs_status BatchWork::ensure(size_t len) {
  for (DBuf<double>* b : {&r, &rh, &p, &ph, &v, &sv, &sh, &t, &z, &q}) FVS_TRY(b->alloc(len + 1));
  return FVS_OK;
}

Batch::~Batch() {
  if (host) cudaFreeHost(host);
}

static int red_blocks(int64_t n, int tiles) {
  const int64_t rb = (n + 7) / 8;
  const int64_t cap = std::max<int64_t>(1, (int64_t)sm_count() * 2 / tiles);
  return (int)std::max<int64_t>(1, std::min(rb, cap));
}

// sc[slot0] = a.b, sc[slot1] = c.d per sample (c null: slot1 unused)
static fvs_status bdot2(Batch& B, int64_t n, const double* a, const double* b, const double* c, const double* d,
                        int slot0, int slot1) {
  const int nb = red_blocks(n, B.tiles);
  kb_dot2<<<dim3(nb, B.tiles), bblock(), 0, B.stream>>>(n, B.Sp, a, b, c, d, B.part, B.sc, slot0, c ? slot1 : -1,
                                                        B.redcnt);
  FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}
static fvs_status bmaxdiff2(Batch& B, int64_t n, const double* a, const double* b, const double* c, const double* d,
                            int slot0, int slot1) {
  const int nb = red_blocks(n, B.tiles);
  kb_maxdiff2<<<dim3(nb, B.tiles), bblock(), 0, B.stream>>>(n, B.Sp, a, b, c, d, B.part, B.sc, slot0, slot1,
                                                            B.redcnt);
  FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}
static fvs_status bcopy(Batch& B, size_t len, const double* a, double* b) {
  kb_copy<<<stride_grid((int64_t)len, 256), 256, 0, B.stream>>>((int64_t)len, a, b); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}
static fvs_status read_counts(Batch& B, int* h, int n) {
  FVS_CUDA(cudaMemcpyAsync(h, B.kcount.p, n * sizeof(int), cudaMemcpyDeviceToHost, B.stream));
  FVS_CUDA(cudaStreamSynchronize(B.stream));
  return FVS_OK;
}
// the staged kernel fits when a block's column list (x of 32 samples)
// stays within the default 48 KB of dynamic shared memory
template <typename V>
static bool stage_fits(const XStage* st) {
  return st && st->R > 0 && (size_t)st->umax * 32 * sizeof(V) <= 48 * 1024;
}
template <class Op, typename V>
static void launch_apply(Batch& B, const Op& op, const V* x, const V* b, V* y, int mode, const V* dinv, V omega,
                         const BShape* sh) {
  const XStage* st = sh ? sh->stage : nullptr;
  if (stage_fits<V>(st)) {
    kb_apply_st<Op, V><<<dim3((unsigned)st->nblk, (unsigned)B.tiles, 1), dim3(32, st->R, 1),
                         (size_t)st->umax * 32 * sizeof(V), B.stream>>>(op, B.Sp, x, b, y, mode, dinv, omega,
                                                                        st->uptr, st->ucol, st->li);
  } else {
    kb_apply<Op, V><<<sgrid(op.n, B.tiles, sh), sblock(sh), 0, B.stream>>>(op, B.Sp, x, b, y, mode, dinv, omega);
  }
}
template <class Op>
static fvs_status bapply(Batch& B, const Op& op, const double* x, const double* b, double* y, int mode,
                         const double* dinv = nullptr, double omega = 0.0, const BShape* sh = nullptr) {
  launch_apply<Op, double>(B, op, x, b, y, mode, dinv, omega, sh);
  FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}
template <class Op>
static fvs_status bapplyf(Batch& B, const Op& op, const float* x, const float* b, float* y, int mode,
                          const float* dinv = nullptr, float omega = 0.0f, const BShape* sh = nullptr) {
  launch_apply<Op, float>(B, op, x, b, y, mode, dinv, omega, sh);
  FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

// ---------------------------------------------------------------------------
// launch-shape autotuner: rows per block (the block is 32 samples x rows) and
// blocks per SM, timed with CUDA events on the live operator and buffers
// (the operator kernels only write their output, so repeated launches are
// harmless); the fastest shape is kept for that operator
// ---------------------------------------------------------------------------
template <class Op, typename V>
static fvs_status tune_apply(Batch& B, const Op& op, const V* x, const V* b, V* y, const V* dinv, BShape& out,
                             const XStage* stage = nullptr) {
  out = BShape();
  if (getenv("FVS_NO_TUNE") || op.n <= 0) return FVS_OK;
  cudaEvent_t e0, e1;
  FVS_CUDA(cudaEventCreate(&e0));
  FVS_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  std::vector<BShape> cand;
  for (int rows : {4, 8, 16, 32})
    for (int per_sm : {8, 16, 32})
      if (32 * rows * per_sm <= 2048 * 4) cand.push_back(BShape{rows, per_sm, nullptr});   // past full occupancy: no
  if (stage_fits<V>(stage)) cand.push_back(BShape{stage->R, 0, stage});
  for (const BShape& sh : cand) {
    launch_apply<Op, V>(B, op, x, b, y, 2, dinv, (V)0.5, &sh);
    if (cudaGetLastError() != cudaSuccess) continue;   // shape not launchable (registers): skip it
    cudaEventRecord(e0, B.stream);
    for (int r = 0; r < 3; ++r) launch_apply<Op, V>(B, op, x, b, y, 2, dinv, (V)0.5, &sh);
    cudaEventRecord(e1, B.stream);
    const cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms < best) { best = ms; out = sh; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

// ---------------------------------------------------------------------------
// AMG: the aggregation of the base operator, per-sample Galerkin values
// ---------------------------------------------------------------------------
__global__ void kb_scale_copy(int64_t n, double a, const double* x, double* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}
__global__ void kb_copy_i32(int64_t n, const int32_t* a, int32_t* b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}
// the fine operator of every sample written out as per-sample ELL values
// (used when the fine level itself is the coarsest)
__global__ void kb_materialize0(int64_t n, int w, int Sp, const double* base, const int32_t* ovr, const int32_t* col,
                                const double* mval, double* out) {
  BSAMPLE;
  BROW(i, n) {
    const int32_t o = ovr[i * Sp + s];
    bool unit = false;    // identity row: 1 in the first slot holding the diagonal
    for (int k = 0; k < w; ++k) {
      const int64_t q = (int64_t)k * n + i;
      double v;
      if (o == -2) {
        v = (!unit && col[q] == (int32_t)i) ? 1.0 : 0.0;
        unit = unit || v != 0.0;
      }
      else if (o < 0) v = base[q];
      else v = mval[(int64_t)o * w + k];
      out[q * Sp + s] = v;
    }
  }
}

template <typename T>
static fvs_status download(cudaStream_t s, const T* d, size_t n, std::vector<T>& h) {
  h.resize(n);
  if (n) FVS_CUDA(cudaMemcpyAsync(h.data(), d, n * sizeof(T), cudaMemcpyDeviceToHost, s));
  return FVS_OK;
}
template <typename T>
static fvs_status upload(cudaStream_t s, const std::vector<T>& h, DBuf<T>& d) {
  FVS_TRY(d.alloc(h.size() + 1));
  if (!h.empty()) FVS_CUDA(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return FVS_OK;
}

// column lists of blocks of R consecutive rows (host, at set-up): every
// stored column of the ELL pattern [k*n + i], k < w
static fvs_status build_stage(cudaStream_t st, int64_t n, int w, const int32_t* dcol, int R, XStage& S) {
  S.R = 0;
  if (n <= 0) return FVS_OK;
  std::vector<int32_t> col((size_t)n * w);
  FVS_CUDA(cudaMemcpyAsync(col.data(), dcol, col.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  FVS_CUDA(cudaStreamSynchronize(st));
  const int64_t nblk = (n + R - 1) / R;
  std::vector<int32_t> uptr(nblk + 1, 0), ucol;
  std::vector<uint8_t> li((size_t)n * w);
  std::vector<int32_t> tmp;
  int umax = 0;
  for (int64_t b = 0; b < nblk; ++b) {
    const int64_t r0 = b * R, r1 = std::min<int64_t>(n, r0 + R);
    tmp.clear();
    for (int64_t i = r0; i < r1; ++i)
      for (int k = 0; k < w; ++k) tmp.push_back(col[(size_t)k * n + i]);
    std::sort(tmp.begin(), tmp.end());
    tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
    if (tmp.size() > 255) return FVS_OK;   // too many columns for a byte index: leave unstaged
    umax = std::max(umax, (int)tmp.size());
    for (int64_t i = r0; i < r1; ++i)
      for (int k = 0; k < w; ++k)
        li[(size_t)k * n + i] =
            (uint8_t)(std::lower_bound(tmp.begin(), tmp.end(), col[(size_t)k * n + i]) - tmp.begin());
    ucol.insert(ucol.end(), tmp.begin(), tmp.end());
    uptr[b + 1] = (int32_t)ucol.size();
  }
  FVS_TRY(upload(st, uptr, S.uptr));
  FVS_TRY(upload(st, ucol, S.ucol));
  FVS_TRY(upload(st, li, S.li));
  FVS_CUDA(cudaStreamSynchronize(st));
  S.R = R;
  S.nblk = nblk;
  S.umax = umax;
  return FVS_OK;
}

// The hierarchy of the base operator (every cell flowing) fixes the
// aggregates and the coarse patterns; the Galerkin map lists, for every coarse
// entry, the fine entries that sum into it.
fvs_status batch_amg_setup(Batch& B) {
  fvs_mesh m = B.mesh;
  cudaStream_t st = B.stream;
  const int64_t Nc = m->Nc;
  const int W = m->W;
  B.amg_ok = false;
  FVS_TRY(B.K0.alloc(Nc, W));
  FVS_CUDA(cudaMemcpyAsync(B.K0.col.p, m->Pb.col.p, (size_t)Nc * W * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  const double a = -1.0 / B.props.mat.rho;
  kb_scale_copy<<<stride_grid(Nc * W, 256), 256, 0, st>>>(Nc * W, a, m->Pb.val, B.K0.val); FVS_COUNT_LAUNCH();
  kb_scale_copy<<<stride_grid(Nc, 256), 256, 0, st>>>(Nc, a, m->Pb.diag, B.K0.diag); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  B.base.opt = B.aopt;
  B.base.opt.fp32 = false;
  if (B.fp32) {
    FVS_TRY(B.K0f.alloc((size_t)Nc * W + 1));
    kb_to_float<<<stride_grid(Nc * W, 256), 256, 0, st>>>(Nc * W, B.K0.val, B.K0f); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
  }
  {
    const fvs_status r = B.base.setup(st, B.K0);
    if (r != FVS_OK) return r;
  }
  const int L = B.base.levels();
  const int nc = (int)B.base.lv.back()->n;
  if (nc > amg_smem_coarsest()) {
    set_error("batched AMG: coarsest level of %d rows (at most %d)", nc, amg_smem_coarsest());
    return FVS_ERR_NOT_CONVERGED;
  }
  B.nc = nc;
  B.lv.clear();
  for (int l = 0; l < L; ++l) B.lv.emplace_back(new BLevel());
  const size_t Sp = (size_t)B.Sp;
  for (int l = 0; l < L; ++l) {
    AmgLevel* A = B.base.lv[l].get();
    BLevel& BL = *B.lv[l];
    BL.n = A->n;
    BL.w = A->A->w;
    BL.col = A->A->col.p;
    BL.rlen = A->rlen.n ? A->rlen.p : nullptr;
    if (l + 1 < L) {
      BL.agg = A->agg.p;
      BL.mptr = A->mptr.p;
      BL.midx = A->midx.p;
    }
    const size_t nS = (size_t)BL.n * Sp + 1;
    FVS_TRY(BL.dinv.alloc(nS)); FVS_TRY(BL.b.alloc(nS)); FVS_TRY(BL.x.alloc(nS)); FVS_TRY(BL.r.alloc(nS));
    FVS_TRY(BL.y.alloc(nS)); FVS_TRY(BL.lab.alloc(nS));
    if (l >= 1 || L == 1) FVS_TRY(BL.val.alloc((size_t)BL.n * BL.w * Sp + 1));
    if (B.fp32) {
      FVS_TRY(BL.dinvf.alloc(nS)); FVS_TRY(BL.bf.alloc(nS)); FVS_TRY(BL.xf.alloc(nS)); FVS_TRY(BL.rf.alloc(nS));
      FVS_TRY(BL.yf.alloc(nS));
      if (l >= 1) FVS_TRY(BL.valf.alloc((size_t)BL.n * BL.w * Sp + 1));
    }
    if (l >= 1) {
      std::vector<int32_t> hc;
      FVS_TRY(download(st, BL.col, (size_t)BL.n * BL.w, hc));
      FVS_CUDA(cudaStreamSynchronize(st));
      std::vector<int32_t> ds(BL.n, -1);
      for (int64_t i = 0; i < BL.n; ++i)
        for (int k = 0; k < BL.w; ++k)
          if (hc[(size_t)k * BL.n + i] == (int32_t)i) { ds[i] = k; break; }
      FVS_TRY(upload(st, ds, BL.dslot));
    }
  }
  // Galerkin maps
  std::vector<int32_t> nnb;
  FVS_TRY(download(st, m->nnb.p, (size_t)Nc, nnb));
  for (int l = 0; l + 1 < L; ++l) {
    BLevel& F = *B.lv[l];
    BLevel& C = *B.lv[l + 1];
    std::vector<int32_t> fcol, agg, mptr, midx, ccol;
    std::vector<double> fval;
    FVS_TRY(download(st, F.col, (size_t)F.n * F.w, fcol));
    FVS_TRY(download(st, F.agg, (size_t)F.n, agg));
    FVS_TRY(download(st, F.mptr, (size_t)C.n + 1, mptr));
    FVS_TRY(download(st, F.midx, (size_t)F.n, midx));
    FVS_TRY(download(st, C.col, (size_t)C.n * C.w, ccol));
    if (l >= 1) FVS_TRY(download(st, B.base.lv[l]->A->val.p, (size_t)F.n * F.w, fval));
    FVS_CUDA(cudaStreamSynchronize(st));
    const int64_t n = F.n, ncl = C.n;
    const int w = F.w, wc = C.w;
    const int64_t nq = (int64_t)wc * ncl;
    std::vector<int64_t> qs;
    std::vector<int32_t> es;
    qs.reserve((size_t)n * w);
    es.reserve((size_t)n * w);
    for (int64_t I = 0; I < ncl; ++I) {
      for (int32_t t = mptr[I]; t < mptr[I + 1]; ++t) {
        const int32_t i = midx[t];
        for (int k = 0; k < w; ++k) {
          const int64_t e = (int64_t)k * n + i;
          const bool real = l == 0 ? k < nnb[i] : (fcol[e] != i || fval[e] != 0.0);
          if (!real) continue;
          const int32_t J = agg[fcol[e]];
          int r = -1;
          for (int c = 0; c < wc; ++c)
            if (ccol[(size_t)c * ncl + I] == J) { r = c; break; }
          if (r < 0) continue;   // an entry the base operator has as an exact zero
          qs.push_back((int64_t)r * ncl + I);
          es.push_back((int32_t)e);
        }
      }
    }
    std::vector<int32_t> gptr(nq + 1, 0), gidx(es.size());
    for (int64_t q : qs) ++gptr[q + 1];
    for (int64_t q = 0; q < nq; ++q) gptr[q + 1] += gptr[q];
    std::vector<int32_t> cur(gptr.begin(), gptr.end() - 1);
    for (size_t t = 0; t < es.size(); ++t) gidx[cur[qs[t]]++] = es[t];
    FVS_TRY(upload(st, gptr, F.gptr));
    FVS_TRY(upload(st, gidx, F.gidx));
  }
  FVS_TRY(B.Ainv.alloc((size_t)nc * nc * Sp + 1));
  FVS_TRY(B.clab.alloc((size_t)nc * Sp + 1));
  FVS_TRY(B.csing.alloc((size_t)nc * Sp + 1));
  FVS_TRY(B.cncomp.alloc(Sp + 1));
  FVS_TRY(B.cid.alloc((size_t)nc * Sp + 1));
  FVS_TRY(B.ccount.alloc((size_t)nc * Sp + 1));
  FVS_TRY(B.ccnt.alloc((size_t)BATCH_NCM * Sp + 1));
  FVS_TRY(B.csum.alloc((size_t)BATCH_NCM * Sp + 1));
  // launch shapes of every level's operator, on the buffers of that level
  // (the fine rows all read their shared base row for the timing)
  FVS_CUDA(cudaMemsetAsync(B.ovr.p, 0xFF, (size_t)Nc * Sp * sizeof(int32_t), st));
  constexpr int STAGE_ROWS = 8;
  FVS_TRY(build_stage(st, Nc, W, B.K0.col.p, STAGE_ROWS, B.stage_p));
  for (int l = 0; l + 1 < L || (L == 1 && l == 0); ++l) {
    BLevel& F = *B.lv[l];
    const size_t nS = (size_t)F.n * Sp;
    if (l >= 1) FVS_TRY(build_stage(st, F.n, F.w, F.col, STAGE_ROWS, F.stage));
    const XStage* stg = l == 0 ? &B.stage_p : &F.stage;
    if (l >= 1) FVS_CUDA(cudaMemsetAsync(F.val.p, 0, (size_t)F.n * F.w * Sp * sizeof(double), st));
    if (B.fp32) {
      if (l >= 1) FVS_CUDA(cudaMemsetAsync(F.valf.p, 0, (size_t)F.n * F.w * Sp * sizeof(float), st));
      for (DBuf<float>* b : {&F.bf, &F.xf, &F.yf, &F.dinvf}) FVS_CUDA(cudaMemsetAsync(b->p, 0, nS * sizeof(float), st));
      if (l == 0)
        FVS_TRY(tune_apply(B, OpPpe0T<float>{Nc, W, B.K0.col.p, B.K0f.p, B.ovr.p, B.mvalf.p}, F.xf.p, F.bf.p, F.yf.p,
                           F.dinvf.p, F.shape, stg));
      else
        FVS_TRY(tune_apply(B, OpCoarseT<float>{F.n, F.w, F.col, F.valf.p, F.rlen}, F.xf.p, F.bf.p, F.yf.p, F.dinvf.p,
                           F.shape, stg));
    } else {
      for (DBuf<double>* b : {&F.b, &F.x, &F.y, &F.dinv}) FVS_CUDA(cudaMemsetAsync(b->p, 0, nS * sizeof(double), st));
      if (l == 0)
        FVS_TRY(tune_apply(B, OpPpe0{Nc, W, B.K0.col.p, B.K0.val.p, B.ovr.p, B.mval.p}, F.x.p, F.b.p, F.y.p, F.dinv.p,
                           F.shape, stg));
      else
        FVS_TRY(tune_apply(B, OpCoarse{F.n, F.w, F.col, F.val.p, F.rlen}, F.x.p, F.b.p, F.y.p, F.dinv.p, F.shape,
                           stg));
    }
    if (getenv("FVS_DEBUG"))
      fprintf(stderr, "[fvs batch] level %d (%lld rows): operator shape %d rows x %d per SM%s (stage umax %d)\n", l,
              (long long)F.n, F.shape.rows, F.shape.per_sm, F.shape.stage ? ", staged" : "", stg->umax);
  }
  FVS_CUDA(cudaStreamSynchronize(st));
  B.amg_ok = true;
  return FVS_OK;
}

// per step: Galerkin values of every level, coarse diagonals, the coarsest
// inverses, null-space labels and the projected parts of every sample
fvs_status batch_amg_values(Batch& B) {
  cudaStream_t st = B.stream;
  const int L = (int)B.lv.size();
  const int Sp = B.Sp;
  fvs_mesh m = B.mesh;
  for (int l = 0; l + 1 < L; ++l) {
    BLevel& F = *B.lv[l];
    BLevel& C = *B.lv[l + 1];
    const int64_t nq = (int64_t)C.w * C.n;
    if (l == 0)
      kb_galerkin0<<<bgrid(nq, B.tiles), bblock(), 0, st>>>(nq, F.n, F.w, Sp, F.gptr, F.gidx, B.K0.val, B.ovr,
                                                            B.mval, C.val);
    else
      kb_galerkin<<<bgrid(nq, B.tiles), bblock(), 0, st>>>(nq, Sp, F.gptr, F.gidx, F.val, C.val);
    FVS_COUNT_LAUNCH();
    kb_coarse_dinv<<<bgrid(C.n, B.tiles), bblock(), 0, st>>>(C.n, Sp, C.dslot, C.val, C.dinv); FVS_COUNT_LAUNCH();
    if (B.fp32) {
      const int64_t nv = C.n * (int64_t)C.w * Sp, nd = C.n * (int64_t)Sp;
      kb_to_float<<<stride_grid(nv, 256), 256, 0, st>>>(nv, C.val, C.valf); FVS_COUNT_LAUNCH();
      kb_to_float<<<stride_grid(nd, 256), 256, 0, st>>>(nd, C.dinv, C.dinvf); FVS_COUNT_LAUNCH();
    }
    FVS_LAUNCH_CHECK();
  }
  BLevel& Lc = *B.lv[L - 1];
  if (L == 1) {
    kb_materialize0<<<bgrid(Lc.n, B.tiles), bblock(), 0, st>>>(Lc.n, Lc.w, Sp, B.K0.val, B.ovr, Lc.col, B.mval,
                                                              Lc.val); FVS_COUNT_LAUNCH();
  }
  FVS_TRY(B.err.zero(st));
  FVS_TRY(amg_coarsest_batched(st, B.nc, Lc.w, Lc.col, Lc.val, Sp, B.Ainv, B.clab, B.csing, B.cncomp, B.err));
  // labels from the coarsest level down to the fine rows
  const int32_t* up = B.clab.p;
  for (int l = L - 2; l >= 0; --l) {
    kb_pull_labels<<<bgrid(B.lv[l]->n, B.tiles), bblock(), 0, st>>>(B.lv[l]->n, Sp, B.lv[l]->agg,
                                                                   l == 0 ? B.ovr.p : nullptr, up, B.lv[l]->lab);
    FVS_COUNT_LAUNCH();
    up = B.lv[l]->lab.p;
  }
  if (L == 1)
    kb_pull_labels<<<bgrid(Lc.n, B.tiles), bblock(), 0, st>>>(Lc.n, Sp, nullptr, B.ovr, B.clab, Lc.lab);
  if (L == 1) FVS_COUNT_LAUNCH();
  FVS_CUDA(cudaMemsetAsync(B.ccount.p, 0, (size_t)B.nc * Sp * sizeof(int), st));
  kb_part_count<<<bgrid(m->Nc, B.tiles), bblock(), 0, st>>>(m->Nc, Sp, B.nc, B.lv[0]->lab, B.ccount);
  FVS_COUNT_LAUNCH();
  kb_part_ids<<<B.tiles, 32, 0, st>>>(Sp, B.nc, B.ccount, B.csing, B.cncomp, B.cid, B.ccnt, B.err); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  int e = 0;
  FVS_CUDA(cudaMemcpyAsync(&e, B.err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  FVS_CUDA(cudaStreamSynchronize(st));
  if (e) {
    set_error("batched AMG: per-sample coarsest inverse failed (flags 0x%x)", e);
    return FVS_ERR_NOT_CONVERGED;
  }
  return FVS_OK;
}

// subtract the mean of every singular liquid part (fine level)
static fvs_status bproject(Batch& B, double* v) {
  const int64_t n = B.mesh->Nc;
  const int nb = red_blocks(n, B.tiles);
  kb_proj_part<<<dim3(nb, B.tiles), bblock(), 0, B.stream>>>(n, B.Sp, B.nc, B.lv[0]->lab, B.cid, v, B.part, B.ccnt,
                                                             B.csum, B.redcnt);
  FVS_COUNT_LAUNCH();
  kb_proj_sub<<<bgrid(n, B.tiles), bblock(), 0, B.stream>>>(n, B.Sp, B.nc, B.lv[0]->lab, B.cid, B.csum, v);
  FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

static OpPpe0 ppe_op(Batch& B) {
  fvs_mesh m = B.mesh;
  return OpPpe0{m->Nc, m->W, B.K0.col.p, B.K0.val.p, B.ovr.p, B.mval.p};
}

static fvs_status level_apply(Batch& B, int l, const double* x, const double* b, double* y, int mode,
                              const double* dinv, double omega) {
  BLevel& L = *B.lv[l];
  if (l == 0) return bapply(B, ppe_op(B), x, b, y, mode, dinv, omega, &L.shape);
  return bapply(B, OpCoarse{L.n, L.w, L.col, L.val.p, L.rlen}, x, b, y, mode, dinv, omega, &L.shape);
}
static fvs_status level_applyf(Batch& B, int l, const float* x, const float* b, float* y, int mode,
                               const float* dinv, float omega) {
  BLevel& L = *B.lv[l];
  if (l == 0) {
    fvs_mesh m = B.mesh;
    return bapplyf(B, OpPpe0T<float>{m->Nc, m->W, B.K0.col.p, B.K0f.p, B.ovr.p, B.mvalf.p}, x, b, y, mode, dinv,
                   omega, &L.shape);
  }
  return bapplyf(B, OpCoarseT<float>{L.n, L.w, L.col, L.valf.p, L.rlen}, x, b, y, mode, dinv, omega, &L.shape);
}

// one V-cycle on level l: y = M^-1 b (damped Jacobi, piecewise-constant
// transfers with over-correction, pinned dense coarsest inverse); V = double,
// or float for the mixed-precision path (FP32 copies of every level)
template <typename V>
static fvs_status bvcycle_t(Batch& B, int l, const V* b, V* y, bool x0_ready = false) {
  const int L = (int)B.lv.size();
  BLevel& F = *B.lv[l];
  const int Sp = B.Sp;
  cudaStream_t st = B.stream;
  const bool f32 = sizeof(V) == 4;
  if (l == L - 1) {
    kb_coarse_solve<V><<<bgrid(F.n, B.tiles), bblock(), 0, st>>>(B.nc, Sp, B.Ainv, b, y); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    return FVS_OK;
  }
  BLevel& C = *B.lv[l + 1];
  const V om = (V)B.aopt.omega;
  V* x = f32 ? (V*)F.xf.p : (V*)F.x.p;
  V* r = f32 ? (V*)F.rf.p : (V*)F.r.p;
  V* cb = f32 ? (V*)C.bf.p : (V*)C.b.p;
  V* cy = f32 ? (V*)C.yf.p : (V*)C.y.p;
  const V* dinv = f32 ? (const V*)F.dinvf.p : (const V*)F.dinv.p;
  if (!x0_ready) {
    kb_jac0<V><<<bgrid(F.n, B.tiles), bblock(), 0, st>>>(F.n, Sp, om, dinv, b, x); FVS_COUNT_LAUNCH();
  }
  if (f32) FVS_TRY(level_applyf(B, l, (const float*)x, (const float*)b, (float*)r, 1, nullptr, 0.0f));
  else FVS_TRY(level_apply(B, l, (const double*)x, (const double*)b, (double*)r, 1, nullptr, 0.0));
  // above a level that is not the coarsest the restriction also forms that
  // level's first Jacobi iterate
  const bool next_sweeps = l + 2 < L;
  if (next_sweeps) {
    V* cx = f32 ? (V*)C.xf.p : (V*)C.x.p;
    const V* cdinv = f32 ? (const V*)C.dinvf.p : (const V*)C.dinv.p;
    kb_restrict_jac0<V><<<bgrid(C.n, B.tiles), bblock(), 0, st>>>(C.n, Sp, F.mptr, F.midx, r, cb, om, cdinv, cx);
  } else {
    kb_restrict<V><<<bgrid(C.n, B.tiles), bblock(), 0, st>>>(C.n, Sp, F.mptr, F.midx, r, cb);
  }
  FVS_COUNT_LAUNCH();
  FVS_TRY(bvcycle_t<V>(B, l + 1, cb, cy, next_sweeps));
  kb_prolong<V><<<bgrid(F.n, B.tiles), bblock(), 0, st>>>(F.n, Sp, F.agg, l == 0 ? B.ovr.p : nullptr, cy,
                                                          (V)B.aopt.coarse_scale, x); FVS_COUNT_LAUNCH();
  if (f32) FVS_TRY(level_applyf(B, l, (const float*)x, (const float*)b, (float*)y, 2, (const float*)dinv, (float)om));
  else FVS_TRY(level_apply(B, l, (const double*)x, (const double*)b, (double*)y, 2, (const double*)dinv, (double)om));
  return FVS_OK;
}
static fvs_status bvcycle(Batch& B, int l, const double* b, double* y) { return bvcycle_t<double>(B, l, b, y); }

// FP32 V-cycle inside the FP64 Krylov method: z = M^-1 r with r, z FP64
static fvs_status bvcycle_mixed(Batch& B, const double* r, double* z) {
  BLevel& F = *B.lv[0];
  const int64_t len = F.n * (int64_t)B.Sp;
  kb_to_float<<<stride_grid(len, 256), 256, 0, B.stream>>>(len, r, F.bf); FVS_COUNT_LAUNCH();
  FVS_TRY(bvcycle_t<float>(B, 0, F.bf.p, F.yf.p));
  kb_to_double<<<stride_grid(len, 256), 256, 0, B.stream>>>(len, F.yf, z); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

// ---------------------------------------------------------------------------
// batched Krylov drivers: every sample runs its own recurrence (own scalars,
// own convergence); samples that converged, or take no part (take = 0),
// keep their vectors.  Returns the number of iterations of the slowest
// sample and, in 'failed', the samples whose true residual stayed above
// 10x the target.
// ---------------------------------------------------------------------------
__global__ void kb_krylov_fail(int Sp, const double* sc, const uint8_t* take, int* counts) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Sp || (take && !take[s])) return;
  const double rr = sc[B_RR * Sp + s];
  if (!(rr <= 100.0 * sc[B_TOL2 * Sp + s])) atomicAdd(&counts[2], 1);
}

struct NoProj {
  bool active() const { return false; }
  fvs_status operator()(double*) const { return FVS_OK; }
};

struct KrylovArgs {
  double rtol = 1e-8;
  const double* rtol_s = nullptr;   // per-sample tolerance (overrides rtol)
  const double* floor = nullptr;    // per-sample floor of the right-side norm
  const uint8_t* take = nullptr;    // samples taking part (null: all)
  int maxit = 1000;
  const BShape* shape = nullptr;    // tuned launch shape of the operator
};

template <class Op>
static fvs_status krylov_start(Batch& B, const Op& op, const double* b, double* x, const KrylovArgs& a,
                               bool projected, int& active) {
  BatchWork& w = B.kw;
  const int64_t n = op.n;
  const double* bb = projected ? w.q : b;
  FVS_TRY(bdot2(B, n, bb, bb, w.r, w.r, B_BB, B_RR));
  FVS_CUDA(cudaMemsetAsync(B.kcount.p, 0, 4 * sizeof(int), B.stream));
  kb_krylov_init<<<B.tiles, 32, 0, B.stream>>>(B.Sp, B.sc, B.kact, a.take, a.rtol_s, a.rtol, a.floor, B.kcount);
  FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  int h[4];
  FVS_TRY(read_counts(B, h, 1));
  active = h[0];
  return FVS_OK;
}

template <class Op, class Proj>
static fvs_status krylov_finish(Batch& B, const Op& op, const double* b, const double* x, Proj& proj,
                                const KrylovArgs& a, int& failed) {
  BatchWork& w = B.kw;
  FVS_TRY(bapply(B, op, x, b, w.t, 1, nullptr, 0.0, a.shape));
  FVS_TRY(proj(w.t));
  FVS_TRY(bdot2(B, op.n, w.t, w.t, nullptr, nullptr, B_RR, -1));
  FVS_CUDA(cudaMemsetAsync(B.kcount.p, 0, 4 * sizeof(int), B.stream));
  kb_krylov_fail<<<B.tiles, 32, 0, B.stream>>>(B.Sp, B.sc, a.take, B.kcount); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  int h[4];
  FVS_TRY(read_counts(B, h, 3));
  failed = h[2];
  return FVS_OK;
}

// Device-driven loop: one graph launch runs iterations of body() under a
// conditional while-node until no sample is active, a sample needs a
// restart, or maxit is reached.  counts[3] returns the iterations done.
__global__ void kb_ctl(cudaGraphConditionalHandle h, int* counts, int maxit) {
  const int n = ++counts[3];
  const bool go = n < maxit && counts[0] > 0 && counts[1] == 0;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}
__global__ void kb_ctl_init(int* counts) { counts[3] = 0; }

template <class Body>
static fvs_status bloop(Batch& B, BatchGraph& g, uint64_t key, Body& body, int maxit, bool& used) {
  used = false;
  cudaStream_t s = B.stream;
  if (g.disabled || !graphs_enabled() || maxit <= 0) return FVS_OK;
  if (!g.exec || g.key != key) {
    g.reset();
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
      ok = cudaStreamBeginCaptureToGraph(s, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        const unsigned long long before = __atomic_load_n(&g_launches, __ATOMIC_RELAXED);
        const fvs_status r = body();
        kb_ctl<<<1, 1, 0, s>>>(h, B.kcount, maxit);
        g.kernels = __atomic_load_n(&g_launches, __ATOMIC_RELAXED) - before + 1;
        __atomic_sub_fetch(&g_launches, g.kernels - 1, __ATOMIC_RELAXED);
        cudaGraph_t out = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s, &out);
        ok = r == FVS_OK && e == cudaSuccess;
      }
    }
    if (ok) ok = cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
      cudaGetLastError();
      g.reset();
      g.disabled = true;
      return FVS_OK;
    }
    g.key = key;
    g.maxit = maxit;
  }
  if (g.maxit != maxit) return FVS_OK;   // the iteration cap is part of the graph
  kb_ctl_init<<<1, 1, 0, s>>>(B.kcount); FVS_COUNT_LAUNCH();
  FVS_CUDA(cudaGraphLaunch(g.exec, s));
  used = true;
  return FVS_OK;
}

static uint64_t hkey(std::initializer_list<const void*> ptrs, uint64_t extra) {
  uint64_t h = 0x84222325cbf29ce4ULL ^ extra;
  for (const void* q : ptrs) h = (h ^ (uint64_t)(uintptr_t)q) * 0x100000001b3ULL;
  return h;
}

// runs iterations until no sample is active (graph loop when available);
// restart() handles samples whose recurrence broke down
template <class Body, class Restart>
static fvs_status bdrive(Batch& B, BatchGraph* g, uint64_t key, Body& body, Restart& restart, int maxit,
                         int& active, int& it) {
  it = 0;
  while (active > 0 && it < maxit) {
    bool used = false;
    if (g) FVS_TRY(bloop(B, *g, key, body, maxit, used));
    int h[4];
    if (used) {
      FVS_TRY(read_counts(B, h, 4));
      __atomic_add_fetch(&g_launches, g->kernels * (unsigned long long)h[3], __ATOMIC_RELAXED);
      it += h[3];
    } else {
      FVS_TRY(body());
      FVS_TRY(read_counts(B, h, 2));
      ++it;
    }
    active = h[0];
    if (active > 0 && h[1] > 0) FVS_TRY(restart());
  }
  return FVS_OK;
}

template <class Op, class Prec, class Proj>
static fvs_status bbicgstab(Batch& B, const Op& op, Prec& prec, Proj& proj, const double* b, double* x,
                            const KrylovArgs& a, int& iters, int& failed, BatchGraph* graph = nullptr) {
  const int64_t n = op.n;
  const int Sp = B.Sp;
  const size_t len = (size_t)n * Sp;
  BatchWork& w = B.kw;
  FVS_TRY(w.ensure(len));
  cudaStream_t st = B.stream;
  iters = 0;
  failed = 0;
  FVS_TRY(bapply(B, op, x, b, w.r, 1, nullptr, 0.0, a.shape));
  FVS_TRY(proj(w.r));
  FVS_TRY(bcopy(B, len, w.r, w.rh));
  if (proj.active()) {
    FVS_TRY(bcopy(B, len, b, w.q));
    FVS_TRY(proj(w.q));
  }
  int active = 0;
  FVS_TRY(krylov_start(B, op, b, x, a, proj.active(), active));
  FVS_TRY(bdot2(B, n, w.rh, w.r, nullptr, nullptr, B_RHO, -1));
  const dim3 g = bgrid(n, B.tiles);
  auto body = [&]() -> fvs_status {
    FVS_CUDA(cudaMemsetAsync(B.kcount.p, 0, 3 * sizeof(int), st));
    kb_bicg_p<<<g, bblock(), 0, st>>>(n, Sp, B.sc, B.kact, w.r, w.v, w.p); FVS_COUNT_LAUNCH();
    FVS_TRY(prec(w.p, w.ph));
    FVS_TRY(bapply(B, op, w.ph, nullptr, w.v, 0, nullptr, 0.0, a.shape));
    FVS_TRY(bdot2(B, n, w.rh, w.v, nullptr, nullptr, B_RV, -1));
    kb_bicg_s<<<g, bblock(), 0, st>>>(n, Sp, B.sc, B.kact, w.r, w.v, w.sv); FVS_COUNT_LAUNCH();
    FVS_TRY(prec(w.sv, w.sh));
    FVS_TRY(bapply(B, op, w.sh, nullptr, w.t, 0, nullptr, 0.0, a.shape));
    FVS_TRY(bdot2(B, n, w.t, w.sv, w.t, w.t, B_TS, B_TT));
    kb_bicg_xr<<<g, bblock(), 0, st>>>(n, Sp, B.sc, B.kact, w.ph, w.sh, w.sv, w.t, x, w.r); FVS_COUNT_LAUNCH();
    FVS_TRY(bdot2(B, n, w.r, w.r, w.rh, w.r, B_RR, B_RZ));
    kb_bicg_next<<<B.tiles, 32, 0, st>>>(Sp, B.sc, B.kact, B.krestart, B.kcount); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    return FVS_OK;
  };
  // restart the samples whose shadow residual broke down
  auto restart = [&]() -> fvs_status {
    FVS_TRY(bapply(B, op, x, b, w.t, 1, nullptr, 0.0, a.shape));
    FVS_TRY(proj(w.t));
    kb_restart<<<g, bblock(), 0, st>>>(n, Sp, B.krestart, w.t, w.r, w.rh); FVS_COUNT_LAUNCH();
    FVS_TRY(bdot2(B, n, w.rh, w.r, nullptr, nullptr, B_RZ, -1));
    kb_restart_scalars<<<B.tiles, 32, 0, st>>>(Sp, B.sc, B.krestart); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    return FVS_OK;
  };
  const uint64_t key = hkey({b, x, w.r.p, w.rh.p, w.p.p, w.ph.p, w.v.p, w.sv.p, w.sh.p, w.t.p, B.sc.p, B.kact.p},
                            B.batch_version * 0x9e3779b97f4a7c15ULL + 1);
  int it = 0;
  FVS_TRY(bdrive(B, graph, key, body, restart, a.maxit, active, it));
  iters = it;
  return krylov_finish(B, op, b, x, proj, a, failed);
}

template <class Op, class Prec, class Proj>
static fvs_status bpcg(Batch& B, const Op& op, Prec& prec, Proj& proj, const double* b, double* x,
                       const KrylovArgs& a, int& iters, int& failed, BatchGraph* graph = nullptr) {
  const int64_t n = op.n;
  const int Sp = B.Sp;
  const size_t len = (size_t)n * Sp;
  BatchWork& w = B.kw;
  FVS_TRY(w.ensure(len));
  cudaStream_t st = B.stream;
  iters = 0;
  failed = 0;
  FVS_TRY(bapply(B, op, x, b, w.r, 1, nullptr, 0.0, a.shape));
  FVS_TRY(proj(w.r));
  if (proj.active()) {
    FVS_TRY(bcopy(B, len, b, w.q));
    FVS_TRY(proj(w.q));
  }
  int active = 0;
  FVS_TRY(krylov_start(B, op, b, x, a, proj.active(), active));
  const dim3 g = bgrid(n, B.tiles);
  auto body = [&]() -> fvs_status {
    FVS_CUDA(cudaMemsetAsync(B.kcount.p, 0, 3 * sizeof(int), st));
    FVS_TRY(prec(w.r, w.z));
    FVS_TRY(proj(w.z));
    FVS_TRY(bdot2(B, n, w.r, w.z, nullptr, nullptr, B_RZ, -1));
    kb_cg_p<<<g, bblock(), 0, st>>>(n, Sp, B.sc, B.kact, w.z, w.p); FVS_COUNT_LAUNCH();
    FVS_TRY(bapply(B, op, w.p, nullptr, w.q, 0, nullptr, 0.0, a.shape));
    FVS_TRY(bdot2(B, n, w.p, w.q, nullptr, nullptr, B_PQ, -1));
    kb_cg_xr<<<g, bblock(), 0, st>>>(n, Sp, B.sc, B.kact, w.p, w.q, x, w.r); FVS_COUNT_LAUNCH();
    FVS_TRY(bdot2(B, n, w.r, w.r, nullptr, nullptr, B_RR, -1));
    kb_cg_next<<<B.tiles, 32, 0, st>>>(Sp, B.sc, B.kact, B.kcount); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    return FVS_OK;
  };
  auto restart = [&]() -> fvs_status { return FVS_OK; };
  const uint64_t key = hkey({b, x, w.r.p, w.z.p, w.p.p, w.q.p, B.sc.p, B.kact.p},
                            B.batch_version * 0x9e3779b97f4a7c15ULL + 2);
  int it = 0;
  FVS_TRY(bdrive(B, graph, key, body, restart, a.maxit, active, it));
  iters = it;
  return krylov_finish(B, op, b, x, proj, a, failed);
}

// ---------------------------------------------------------------------------
// the method's steps per (cell or face, sample)
// ---------------------------------------------------------------------------
struct BMat {
  double rho, k, cp, L, Ts, mu, beta, Tref, g0, g1, g2, C, eps;
  FsLaw law;    // solid fraction; its liquidus is replaced by each sample's
};

__device__ __forceinline__ FsLaw b_law(FsLaw w, double Tl) {
  w.Tl = Tl;
  return w;
}

// 1. tags (Section 2.4): LM iff T > T_sol; solid cells lose their velocity
__global__ void kb_tag(int64_t Nc, int Sp, const double* T, double Ts, const uint8_t* run, uint8_t* lm, double* u,
                       double* uold, int* nlm) {
  BSAMPLE;
  int cnt = 0;
  const bool r = run[s] != 0;
  BROW(c, Nc) {
    const int64_t e = c * Sp + s;
    const bool l = r && T[e] > Ts;
    lm[e] = l;
    cnt += l ? 1 : 0;
    if (!l && r) {
      for (int d = 0; d < 3; ++d) {
        u[(d * Nc + c) * Sp + s] = 0.0;
        uold[(d * Nc + c) * Sp + s] = 0.0;
      }
    }
  }
  if (cnt) atomicAdd(&nlm[s], cnt);
}
__global__ void kb_faces_open(int64_t Nf, int Sp, const int32_t* own, const int32_t* nei, const uint8_t* lm,
                              double* F, double* Fold, uint8_t* flow) {
  BSAMPLE;
  BROW(f, Nf) {
    const int32_t o = own[f], q = nei[f];
    const int64_t e = f * Sp + s;
    const bool open = q >= 0 && lm[(int64_t)o * Sp + s] && lm[(int64_t)q * Sp + s];
    if (!open) {
      F[e] = 0.0;
      Fold[e] = 0.0;
    } else {
      flow[(int64_t)o * Sp + s] = 1;
      flow[(int64_t)q * Sp + s] = 1;
    }
  }
}
__global__ void kb_ppe_cells(int64_t Nc, int Sp, const uint8_t* lm, const uint8_t* flow, uint8_t* ppe) {
  BSAMPLE;
  BROW(c, Nc) { const int64_t e = c * Sp + s; ppe[e] = lm[e] && flow[e]; }
}
__global__ void kb_vertex_nonppe(int64_t Nv, int Sp, const int32_t* vptr, const int32_t* vidx, const uint8_t* ppe,
                                 int32_t* nS) {
  BSAMPLE;
  BROW(v, Nv) {
    int n = 0;
    for (int32_t e = vptr[v]; e < vptr[v + 1]; ++e) n += ppe[(int64_t)vidx[e] * Sp + s] ? 0 : 1;
    nS[v * Sp + s] = n;
  }
}
// face cases of Section 2.4.2: 0 wall, 1 no solid neighbour, 2 solid neighbour only, 3 solid owner
__global__ void kb_face_case(int64_t Nf, int Sp, const int32_t* own, const int32_t* nei, const int32_t* fv,
                             const uint8_t* lm, const int32_t* nS, uint8_t* fcase) {
  BSAMPLE;
  BROW(f, Nf) {
    const int32_t o = own[f], q = nei[f];
    uint8_t c;
    if (q < 0) c = 0;
    else if (!(lm[(int64_t)o * Sp + s] && lm[(int64_t)q * Sp + s])) c = 3;
    else {
      int t = 0;
      for (int k = 0; k < 4; ++k) t += nS[(int64_t)fv[k * Nf + f] * Sp + s];
      c = t > 0 ? 2 : 1;
    }
    fcase[f * Sp + s] = c;
  }
}

// 2. momentum predictor (Eq. 6): per-sample diagonal, right sides and
// initial guesses; solid rows are identity rows with zero right side
__global__ void kb_mom_sys(int64_t Nc, int Sp, int W, const int32_t* Lcol, const double* Lval, const double* V,
                           const double* fs, BMat m, double dt, const uint8_t* lm, const int32_t* cf,
                           const int8_t* cfs, const int32_t* own, const int32_t* nei, const double* F,
                           const double* Fold, const double* u, const double* uold, const double* T, double* mdiag,
                           double* jd, double* rhs, double* x) {
  BSAMPLE;
  BROW(c, Nc) {
    const int64_t e = c * Sp + s;
    if (!lm[e]) {
      mdiag[e] = 1.0;
      jd[e] = 1.0;
      for (int d = 0; d < 3; ++d) {
        rhs[(d * Nc + c) * Sp + s] = 0.0;
        x[(d * Nc + c) * Sp + s] = 0.0;
      }
      continue;
    }
    const double f = fs[e];
    const double D = m.C * f * f / ((1.0 - f) * (1.0 - f) * (1.0 - f) + m.eps);
    const double Vc = V[c];
    double ad = 0.0;
    double lu[3] = {0, 0, 0};
    bool seen = false;
    for (int k = 0; k < W; ++k) {
      const int32_t j = Lcol[(int64_t)k * Nc + c];
      const double a = Lval[(int64_t)k * Nc + c];
      if (j == c && !seen) { ad = a; seen = true; }
      for (int d = 0; d < 3; ++d) lu[d] += a * u[(d * Nc + j) * Sp + s];
    }
    const double dg = (m.rho / dt + D) * Vc - 0.5 * m.mu * ad;
    mdiag[e] = dg;
    jd[e] = 1.0 / dg;
    double cn[3] = {0, 0, 0}, co[3] = {0, 0, 0};
    for (int t = 0; t < 6; ++t) {
      const int32_t fc = cf[t * Nc + c];
      const int32_t o = own[fc], q = nei[fc];
      if (q < 0) continue;
      const double sg = (double)cfs[t * Nc + c];
      const double fn = sg * F[(int64_t)fc * Sp + s], fo = sg * Fold[(int64_t)fc * Sp + s];
      for (int d = 0; d < 3; ++d) {
        cn[d] += fn * 0.5 * (u[(d * Nc + o) * Sp + s] + u[(d * Nc + q) * Sp + s]);
        co[d] += fo * 0.5 * (uold[(d * Nc + o) * Sp + s] + uold[(d * Nc + q) * Sp + s]);
      }
    }
    const double bf = -m.rho * m.beta * (T[e] - m.Tref) * Vc;
    const double g[3] = {m.g0, m.g1, m.g2};
    for (int d = 0; d < 3; ++d) {
      const double ud = u[(d * Nc + c) * Sp + s];
      rhs[(d * Nc + c) * Sp + s] = m.rho * Vc / dt * ud - m.rho * (1.5 * cn[d] - 0.5 * co[d]) + 0.5 * m.mu * lu[d] +
                                   bf * g[d];
      x[(d * Nc + c) * Sp + s] = ud;
    }
  }
}
__global__ void kb_max3_floor(int Sp, const double* sc, double* floor) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Sp) return;
  floor[s] = sqrt(fmax(fmax(sc[B_T0 * Sp + s], sc[B_T1 * Sp + s]), sc[B_T2 * Sp + s]));
}

// 3. pressure rows (Eq. 9, Section 2.4.2): identity rows for cells without
// pressure, the shared base row where no face of the cell is of case 2/3,
// else the row re-assembled from the faces with smeared coefficients (Eq. 16)
struct BPpe {
  int64_t Nc, Nf;
  int W;
  int Sp;
  const int32_t *cf, *own, *nei, *fv, *vc_ptr, *vc_idx, *nb, *nnb, *fnb, *nfnb;
  const int8_t* cfs;
  const double *cd, *ce, *cz, *bdiag;
  const uint8_t *ppe, *fcase;
  const int32_t* nS;
  double rho;
};
__device__ __forceinline__ bool b_modified(const BPpe& x, int64_t c, int s) {
  for (int t = 0; t < 6; ++t) {
    const uint8_t fc = x.fcase[(int64_t)x.cf[t * x.Nc + c] * x.Sp + s];
    if (fc == 2 || fc == 3) return true;
  }
  return false;
}
__global__ void kb_ppe_count(BPpe x, int* count) {
  BSAMPLE;
  int cnt = 0;
  BROW(c, x.Nc) {
    if (x.ppe[c * x.Sp + s] && b_modified(x, c, s)) ++cnt;
  }
  if (cnt) atomicAdd(count, cnt);
}
// nbl: the row's sorted neighbour list, copied to thread-local memory once
__device__ __forceinline__ void b_vertex(const BPpe& x, const int32_t* nbl, int s, int nn, int32_t v, double coef,
                                         double* acc) {
  const int32_t lo = x.vc_ptr[v], hi = x.vc_ptr[v + 1];
  const double share = coef / (double)(hi - lo);
  for (int32_t e = lo; e < hi; ++e) {
    const int32_t j = x.vc_idx[e];
    if (!x.ppe[(int64_t)j * x.Sp + s]) continue;
    const int p = find_sorted(nbl, 1, nn, j);
    if (p >= 0) acc[p] += share;
  }
}
__global__ void kb_ppe_rows(BPpe x, int32_t* ovr, double* mval, double* dinv, int* counter, int64_t cap, int* err) {
  BSAMPLE;
  double acc[FVS_MAX_NB];
  BROW(c, x.Nc) {
    const int64_t e = c * x.Sp + s;
    if (!x.ppe[e]) { ovr[e] = -2; dinv[e] = 1.0; continue; }
    if (!b_modified(x, c, s)) {
      ovr[e] = -1;
      const double d = x.bdiag[c];
      dinv[e] = d != 0.0 ? 1.0 / d : 0.0;
      continue;
    }
    const int o = atomicAdd(counter, 1);
    if (o >= cap) { atomicOr(err, 32); ovr[e] = -2; dinv[e] = 1.0; continue; }
    ovr[e] = o;
    const int nn = x.nnb[c];
    int32_t nbl[FVS_MAX_NB];
    for (int k = 0; k < nn; ++k) {
      acc[k] = 0.0;
      nbl[k] = x.nb[(int64_t)k * x.Nc + c];
    }
    for (int t = 0; t < 6; ++t) {
      const int32_t f = x.cf[t * x.Nc + c];
      const uint8_t fc = x.fcase[(int64_t)f * x.Sp + s];
      if (fc != 1 && fc != 2) continue;
      const double sg = (double)x.cfs[t * x.Nc + c];
      const int32_t ow = x.own[f], q = x.nei[f];
      { const int pq = find_sorted(nbl, 1, nn, q); if (pq >= 0) acc[pq] += sg * x.cd[f]; else atomicOr(err, 8); }
      { const int po = find_sorted(nbl, 1, nn, ow); if (po >= 0) acc[po] -= sg * x.cd[f]; else atomicOr(err, 8); }
      const int32_t v1 = x.fv[f], v2 = x.fv[x.Nf + f], v3 = x.fv[2 * x.Nf + f], v4 = x.fv[3 * x.Nf + f];
      const double ce = sg * x.ce[f], cz = sg * x.cz[f];
      b_vertex(x, nbl, s, nn, v3, ce, acc);
      b_vertex(x, nbl, s, nn, v1, -ce, acc);
      b_vertex(x, nbl, s, nn, v4, cz, acc);
      b_vertex(x, nbl, s, nn, v2, -cz, acc);
      if (fc == 2) {
        auto frac = [&](int32_t v) {
          return (double)x.nS[(int64_t)v * x.Sp + s] / (double)(x.vc_ptr[v + 1] - x.vc_ptr[v]);
        };
        const double sdel = ce * (frac(v3) - frac(v1)) + cz * (frac(v4) - frac(v2));
        const int nf = x.nfnb[f];
        int nrem = 0;
        for (int k = 0; k < nf; ++k) nrem += x.ppe[(int64_t)x.fnb[(int64_t)k * x.Nf + f] * x.Sp + s] ? 1 : 0;
        const double add = sdel / (double)nrem;
        for (int k = 0; k < nf; ++k) {
          const int32_t j = x.fnb[(int64_t)k * x.Nf + f];
          if (!x.ppe[(int64_t)j * x.Sp + s]) continue;
          const int p = find_sorted(nbl, 1, nn, j);
          if (p >= 0) acc[p] += add;
          else if (add != 0.0) atomicOr(err, 2);   // a zero share may miss a face-only stencil
        }
      }
    }
    double dg = 0.0;
    double* row = mval + (int64_t)o * x.W;
    for (int k = 0; k < x.W; ++k) {
      double v = 0.0;
      if (k < nn) {
        const int32_t j = x.nb[(int64_t)k * x.Nc + c];
        const double a = -acc[k] / x.rho;
        if (x.ppe[(int64_t)j * x.Sp + s]) v = a;
        else if (a != 0.0) atomicOr(err, 4);
        if (j == c) dg = v;
      }
      row[k] = v;
    }
    dinv[e] = dg != 0.0 ? 1.0 / dg : 0.0;
  }
}
// b = (1/dt) sum over flowing faces of sigma A n . (u*_C1 + u*_C2)/2; K rhs = -b
__global__ void kb_ppe_rhs(int64_t Nc, int64_t Nf, int Sp, const uint8_t* ppe, const int32_t* cf, const int8_t* cfs,
                           const uint8_t* fcase, const int32_t* own, const int32_t* nei, const double* A,
                           const double* nrm, const double* us, double dt, const double* p, double* rhs, double* x) {
  BSAMPLE;
  BROW(c, Nc) {
    const int64_t e = c * Sp + s;
    double b = 0.0;
    if (ppe[e]) {
      for (int t = 0; t < 6; ++t) {
        const int32_t f = cf[t * Nc + c];
        const uint8_t fc = fcase[(int64_t)f * Sp + s];
        if (fc != 1 && fc != 2) continue;
        const int32_t o = own[f], q = nei[f];
        double un = 0.0;
        for (int d = 0; d < 3; ++d)
          un += nrm[d * Nf + f] * 0.5 * (us[(d * Nc + o) * Sp + s] + us[(d * Nc + q) * Sp + s]);
        b += (double)cfs[t * Nc + c] * A[f] * un;
      }
      b /= dt;
    }
    rhs[e] = -b;
    x[e] = ppe[e] ? p[e] : 0.0;
  }
}

// 4. correction (Eq. 17 and the cell gradient of Section 2.4.3)
__global__ void kb_vertex_p(int64_t Nv, int Sp, const int32_t* vptr, const int32_t* vidx, const uint8_t* ppe,
                            const double* p, const int32_t* nS, double* pv, double* fS) {
  BSAMPLE;
  BROW(v, Nv) {
    const int32_t lo = vptr[v], hi = vptr[v + 1];
    double a = 0.0;
    for (int32_t e = lo; e < hi; ++e) {
      const int64_t j = (int64_t)vidx[e] * Sp + s;
      if (ppe[j]) a += p[j];
    }
    const double n = (double)(hi - lo);
    pv[v * Sp + s] = a / n;
    fS[v * Sp + s] = (double)nS[v * Sp + s] / n;
  }
}
__global__ void kb_face_correct(int64_t Nf, int64_t Nc, int Sp, const int32_t* own, const int32_t* nei,
                                const int32_t* fv, const uint8_t* fcase, const int32_t* fnb, const int32_t* nfnb,
                                const uint8_t* ppe, const double* p, const double* pv, const double* fS,
                                const double* A, const double* nrm, const double* cd, const double* ce,
                                const double* cz, const double* Jinv, const double* us, double dt, double rho,
                                const uint8_t* run, const double* F, double* Fnew, double* gradf) {
  BSAMPLE;
  const bool r = run[s] != 0;
  BROW(f, Nf) {
    const int64_t e = f * Sp + s;
    const uint8_t fc = fcase[e];
    if (!r || (fc != 1 && fc != 2)) {
      Fnew[e] = r ? 0.0 : F[e];
      for (int d = 0; d < 3; ++d) gradf[(d * Nf + f) * Sp + s] = 0.0;
      continue;
    }
    const int32_t o = own[f], q = nei[f];
    const int32_t v1 = fv[f], v2 = fv[Nf + f], v3 = fv[2 * Nf + f], v4 = fv[3 * Nf + f];
    const double dxi = p[(int64_t)q * Sp + s] - p[(int64_t)o * Sp + s];
    double deta = pv[(int64_t)v3 * Sp + s] - pv[(int64_t)v1 * Sp + s];
    double dzeta = pv[(int64_t)v4 * Sp + s] - pv[(int64_t)v2 * Sp + s];
    if (fc == 2) {
      const int nf = nfnb[f];
      double a = 0.0;
      int n = 0;
      for (int k = 0; k < nf; ++k) {
        const int64_t j = (int64_t)fnb[(int64_t)k * Nf + f] * Sp + s;
        if (ppe[j]) { a += p[j]; ++n; }
      }
      const double pbar = a / (double)n;
      deta += (fS[(int64_t)v3 * Sp + s] - fS[(int64_t)v1 * Sp + s]) * pbar;
      dzeta += (fS[(int64_t)v4 * Sp + s] - fS[(int64_t)v2 * Sp + s]) * pbar;
    }
    const double nd = cd[f] * dxi + ce[f] * deta + cz[f] * dzeta;
    double un = 0.0;
    for (int d = 0; d < 3; ++d)
      un += nrm[d * Nf + f] * 0.5 * (us[(d * Nc + o) * Sp + s] + us[(d * Nc + q) * Sp + s]);
    Fnew[e] = A[f] * un - dt / rho * nd;
    for (int d = 0; d < 3; ++d)
      gradf[(d * Nf + f) * Sp + s] = Jinv[(3 * d + 0) * Nf + f] * dxi + Jinv[(3 * d + 1) * Nf + f] * deta +
                                     Jinv[(3 * d + 2) * Nf + f] * dzeta;
  }
}
__global__ void kb_cell_correct(int64_t Nc, int64_t Nf, int Sp, const uint8_t* lm, const int32_t* cf,
                                const uint8_t* fcase, const double* gradf, const double* us, double dt, double rho,
                                const uint8_t* run, const double* u, double* unew) {
  BSAMPLE;
  const bool r = run[s] != 0;
  BROW(c, Nc) {
    const int64_t e = c * Sp + s;
    if (!r) {
      for (int d = 0; d < 3; ++d) unew[(d * Nc + c) * Sp + s] = u[(d * Nc + c) * Sp + s];
      continue;
    }
    if (!lm[e]) {
      for (int d = 0; d < 3; ++d) unew[(d * Nc + c) * Sp + s] = 0.0;
      continue;
    }
    double g[3] = {0, 0, 0};
    int n = 0;
    for (int t = 0; t < 6; ++t) {
      const int32_t f = cf[t * Nc + c];
      const uint8_t fc = fcase[(int64_t)f * Sp + s];
      if (fc != 1 && fc != 2) continue;
      ++n;
      for (int d = 0; d < 3; ++d) g[d] += gradf[(d * Nf + f) * Sp + s];
    }
    for (int d = 0; d < 3; ++d)
      unew[(d * Nc + c) * Sp + s] = us[(d * Nc + c) * Sp + s] - (n > 0 ? dt / rho * g[d] / (double)n : 0.0);
  }
}

// 5. energy (Eq. 4, Eq. 18-20) on all cells
__global__ void kb_energy_base(int64_t Nc, int Sp, int W, const int32_t* cf, const int8_t* cfs, const int32_t* own,
                               const int32_t* nei, const double* F, const double* Fold, const double* T,
                               const double* Told, const int32_t* Lcol, const double* Lval, const double* lT1,
                               const double* Twall, const double* V, BMat m, double dt, double* base) {
  BSAMPLE;
  const double tw = Twall[s];
  BROW(c, Nc) {
    double cn = 0.0, co = 0.0;
    for (int t = 0; t < 6; ++t) {
      const int32_t f = cf[t * Nc + c];
      const int32_t o = own[f], q = nei[f];
      if (q < 0) continue;
      const double sg = (double)cfs[t * Nc + c];
      cn += sg * F[(int64_t)f * Sp + s] * 0.5 * (T[(int64_t)o * Sp + s] + T[(int64_t)q * Sp + s]);
      co += sg * Fold[(int64_t)f * Sp + s] * 0.5 * (Told[(int64_t)o * Sp + s] + Told[(int64_t)q * Sp + s]);
    }
    double lt = 0.0;
    for (int k = 0; k < W; ++k)
      lt += Lval[(int64_t)k * Nc + c] * T[(int64_t)Lcol[(int64_t)k * Nc + c] * Sp + s];
    base[c * Sp + s] = m.rho * m.cp * V[c] / dt * T[c * Sp + s] - m.rho * m.cp * (1.5 * cn - 0.5 * co) +
                       0.5 * m.k * lt + m.k * lT1[c] * tw;
  }
}
// source linearisation at the current iterate (Eq. 20); Jacobi diagonal of the pass
__global__ void kb_energy_lin(int64_t Nc, int Sp, const double* V, BMat m, const double* Tliq, double dt,
                              const double* Tm, const double* fsm, const double* fsn, const double* base,
                              const double* kevd, double* dextra, double* rhs, double* x, double* jd) {
  BSAMPLE;
  const FsLaw law = b_law(m.law, Tliq[s]);
  BROW(c, Nc) {
    const int64_t e = c * Sp + s;
    const double t = Tm[e];
    const double dfs = fs_slope(law, t);
    const double a = m.rho * m.L * V[c] / dt;
    const double Sp_ = a * dfs;
    const double Sc = a * (fsm[e] - fsn[e] - dfs * t);
    const double dx = m.rho * m.cp * V[c] / dt - Sp_;
    dextra[e] = dx;
    rhs[e] = base[e] + Sc;
    x[e] = t;
    jd[e] = 1.0 / (kevd[c] + dx);
  }
}
// enthalpy-to-temperature inversion of the linearised update (samples that
// do not iterate keep their iterate)
__global__ void kb_energy_update(int64_t Nc, int Sp, BMat m, const double* Tliq, const uint8_t* take,
                                 const double* Tlin, const double* Tm, const double* fsm, double* Tnext,
                                 double* fsnext) {
  BSAMPLE;
  const FsLaw law = b_law(m.law, Tliq[s]);
  const bool go = take[s] != 0;
  BROW(c, Nc) {
    const int64_t e = c * Sp + s;
    if (!go) { Tnext[e] = Tm[e]; fsnext[e] = fsm[e]; continue; }
    const double t = Tm[e];
    const double dfs = fs_slope(law, t);
    const double H = m.cp * Tlin[e] + m.L * (1.0 - fsm[e] - dfs * (Tlin[e] - t));
    const double T = T_of_H(law, m.cp, m.L, H);
    Tnext[e] = T;
    fsnext[e] = fs_of(law, T);
  }
}
// first iterate of the latent-heat loop: T^n extrapolated linearly in time
// (samples that no longer run keep their state)
__global__ void kb_energy_guess(int64_t Nc, int Sp, const double* T, const double* Told, const double* fs,
                                FsLaw law0, const double* Tliq, const uint8_t* run, double* Tm, double* fsm) {
  BSAMPLE;
  const bool r = run[s] != 0;
  const FsLaw law = b_law(law0, Tliq[s]);
  BROW(c, Nc) {
    const int64_t e = c * Sp + s;
    if (!r) { Tm[e] = T[e]; fsm[e] = fs[e]; continue; }
    const double t = 2.0 * T[e] - Told[e];
    Tm[e] = t;
    fsm[e] = fs_of(law, t);
  }
}
// latent-heat loop bookkeeping per sample: stop rule and the next pass's
// inner tolerance; counts[0] samples still iterating
__global__ void kb_energy_check(int Sp, const double* sc, uint8_t* take, uint8_t* conv, double* ertol, double e_tol_T,
                                double e_rtol, int* counts) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Sp || !take[s]) return;
  const double dT = sc[B_T0 * Sp + s], dF = sc[B_T1 * Sp + s];
  if (dT <= e_tol_T && dF <= 1e-12 && ertol[s] <= e_rtol) {
    conv[s] = 1;
    take[s] = 0;
    return;
  }
  ertol[s] = fmax(e_rtol, fmin(1e-4, 1e-5 * dT));
  atomicAdd(&counts[0], 1);
}
__global__ void kb_energy_start(int Sp, const uint8_t* run, uint8_t* take, uint8_t* conv, double* ertol,
                                double e_rtol) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Sp) return;
  take[s] = run[s];
  conv[s] = run[s] ? 0 : 1;
  ertol[s] = fmax(e_rtol, 1e-4);
}

// 6. liquidus / solidus crossing times (Eq. 22-23 inputs)
__global__ void kb_crossings(int64_t Nc, int Sp, const double* Tn, const double* Tnew, double Ts, const double* Tliq,
                             const uint8_t* run, double time, double dt, double* tliq, double* tsol) {
  BSAMPLE;
  if (!run[s]) return;
  const double Tl = Tliq[s];
  BROW(c, Nc) {
    const int64_t e = c * Sp + s;
    const double a = Tn[e], b = Tnew[e];
    if (tliq[e] < 0.0 && a > Tl && b <= Tl) tliq[e] = time + dt * (a - Tl) / (a - b);
    if (tsol[e] < 0.0 && a > Ts && b <= Ts) tsol[e] = time + dt * (a - Ts) / (a - b);
  }
}
// grain growth (Eq. 24-26) per sample: d(r^2)/dt = lambda_s^2 D_s by the
// trapezoidal rule between the solid fractions at both ends of the step
__device__ __forceinline__ double b_grain_lambda(double fs, double kp) {
  if (!(fs > 0.0 && fs < 1.0)) return 0.0;
  const double S = 2.0 * (1.0 - pow(1.0 - fs, 1.0 - kp)) / (kp - 1.0);
  const double pi = 3.14159265358979323846;
  return -S / (2.0 * sqrt(pi)) + sqrt(fmax(S * S / (4.0 * pi) - S, 0.0));
}
__global__ void kb_grain(int64_t Nc, int Sp, const double* fsa, const double* fsb, const uint8_t* run, double kp,
                         double Ds, double dt, double* r2) {
  BSAMPLE;
  if (!run[s]) return;
  BROW(c, Nc) {
    const int64_t e = c * Sp + s;
    const double la = b_grain_lambda(fsa[e], kp), lb = b_grain_lambda(fsb[e], kp);
    r2[e] += dt * Ds * 0.5 * (la * la + lb * lb);
  }
}
__global__ void kb_fill(size_t n, double v, double* a) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) a[i] = v;
}
// the outputs of Section 5 per sample over the whole domain: latest solidus
// crossing, largest SDAS, smallest yield strength, largest grain radius, and
// the count of cells still above the solidus
__global__ void kb_qoi_ext_part(int64_t Nc, int Sp, const double* tliq, const double* tsol, double Ts,
                                const double* Tliq, const double* r2, double* part) {
  __shared__ double sh[5][8][33];
  BSAMPLE;
  const double Tl = Tliq[s];
  double a[5] = {-1.0, -1.0, 1e300, 0.0, 0.0};
  BROW(c, Nc) {
    const int64_t e = c * Sp + s;
    if (tsol[e] < 0.0) {
      a[4] += 1.0;
    } else {
      a[0] = fmax(a[0], tsol[e]);
      if (tliq[e] >= 0.0) {
        const double lam = 39.4 * pow((Tl - Ts) / (tsol[e] - tliq[e]), -0.317);   // Eq. 22
        a[1] = fmax(a[1], lam);
        a[2] = fmin(a[2], 59.0 / sqrt(lam) + 120.3);                            // Eq. 23
      }
    }
    if (r2) a[3] = fmax(a[3], sqrt(r2[e]));
  }
  for (int k = 0; k < 5; ++k) sh[k][threadIdx.y][threadIdx.x] = a[k];
  __syncthreads();
  if (threadIdx.y == 0) {
    double u[5] = {-1.0, -1.0, 1e300, 0.0, 0.0};
    for (int y = 0; y < 8; ++y) {
      u[0] = fmax(u[0], sh[0][y][threadIdx.x]);
      u[1] = fmax(u[1], sh[1][y][threadIdx.x]);
      u[2] = fmin(u[2], sh[2][y][threadIdx.x]);
      u[3] = fmax(u[3], sh[3][y][threadIdx.x]);
      u[4] += sh[4][y][threadIdx.x];
    }
    for (int k = 0; k < 5; ++k) part[((int64_t)k * Sp + s) * gridDim.x + blockIdx.x] = u[k];
  }
}
__global__ void kb_qoi_ext_final(int nb, int Sp, const double* part, double* out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Sp) return;
  double u[5] = {-1.0, -1.0, 1e300, 0.0, 0.0};
  for (int b = 0; b < nb; ++b) {
    u[0] = fmax(u[0], part[((int64_t)0 * Sp + s) * nb + b]);
    u[1] = fmax(u[1], part[((int64_t)1 * Sp + s) * nb + b]);
    u[2] = fmin(u[2], part[((int64_t)2 * Sp + s) * nb + b]);
    u[3] = fmax(u[3], part[((int64_t)3 * Sp + s) * nb + b]);
    u[4] += part[((int64_t)4 * Sp + s) * nb + b];
  }
  for (int k = 0; k < 5; ++k) out[k * Sp + s] = u[k];
}
// one sample's field in the caller's cell order: out[comps*to_in[c] + d] =
// src[(d*Nc + c)*Sp + s]
__global__ void kb_field_out(int64_t Nc, int Sp, int s, int comps, const int32_t* to_in, const double* src,
                             double* out) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < Nc; c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = to_in[c];
    for (int d = 0; d < comps; ++d) out[comps * o + d] = src[((int64_t)d * Nc + c) * Sp + s];
  }
}
// per-sample sums over solidified cells of t_f, cooling rate, SDAS, yield and the count
__global__ void kb_qoi_part(int64_t Nc, int Sp, const double* tliq, const double* tsol, double Ts, const double* Tliq,
                            double* part) {
  __shared__ double sh[5][8][33];
  BSAMPLE;
  const double Tl = Tliq[s];
  double a[5] = {0, 0, 0, 0, 0};
  BROW(c, Nc) {
    const int64_t e = c * Sp + s;
    if (tliq[e] >= 0.0 && tsol[e] >= 0.0) {
      const double tf = tsol[e] - tliq[e];
      const double cr = (Tl - Ts) / tf;
      const double lam = 39.4 * pow(cr, -0.317);      // Eq. 22
      a[0] += tf;
      a[1] += cr;
      a[2] += lam;
      a[3] += 59.0 / sqrt(lam) + 120.3;              // Eq. 23
      a[4] += 1.0;
    }
  }
  for (int k = 0; k < 5; ++k) sh[k][threadIdx.y][threadIdx.x] = a[k];
  __syncthreads();
  if (threadIdx.y == 0) {
    for (int k = 0; k < 5; ++k) {
      double u = 0.0;
      for (int y = 0; y < 8; ++y) u += sh[k][y][threadIdx.x];
      part[((int64_t)k * Sp + s) * gridDim.x + blockIdx.x] = u;
    }
  }
}
__global__ void kb_qoi_final(int nb, int Sp, const double* part, double* out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Sp) return;
  for (int k = 0; k < 5; ++k) {
    double u = 0.0;
    for (int b = 0; b < nb; ++b) u += part[((int64_t)k * Sp + s) * nb + b];
    out[k * Sp + s] = u;
  }
}
// initial state: T = melt temperature, at rest, no crossings yet; padding
// samples are solid and never run
__global__ void kb_init(int64_t Nc, int64_t Nf, int Sp, const double* Tmelt, const double* Tliq, FsLaw law0,
                        const uint8_t* run, double* T, double* Told, double* fs, double* u, double* uold, double* p,
                        double* tliq, double* tsol, double* F, double* Fold) {
  BSAMPLE;
  const double t0 = run[s] ? Tmelt[s] : law0.Ts - 1.0;
  BROW(c, Nc) {
    const int64_t e = c * Sp + s;
    T[e] = t0;
    Told[e] = t0;
    fs[e] = fs_of(b_law(law0, Tliq[s]), t0);
    p[e] = 0.0;
    tliq[e] = -1.0;
    tsol[e] = -1.0;
    for (int d = 0; d < 3; ++d) {
      u[(d * Nc + c) * Sp + s] = 0.0;
      uold[(d * Nc + c) * Sp + s] = 0.0;
    }
  }
  BROW(f, Nf) {
    F[f * Sp + s] = 0.0;
    Fold[f * Sp + s] = 0.0;
  }
}
__global__ void kb_shared_ops(int64_t Nc, int W, double mu, double k, const int32_t* Lcol, const double* Lval,
                              const double* LTval, const double* LTdiag, double* moff, double* kev, double* kevd) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < Nc; c += (int64_t)gridDim.x * blockDim.x) {
    for (int q = 0; q < W; ++q) {
      const int64_t e = (int64_t)q * Nc + c;
      moff[e] = Lcol[e] == (int32_t)c ? 0.0 : -0.5 * mu * Lval[e];
      kev[e] = -0.5 * k * LTval[e];
    }
    kevd[c] = -0.5 * k * LTdiag[c];
  }
}

// ---------------------------------------------------------------------------
// host: one step of every running sample, and the batch driver
// ---------------------------------------------------------------------------
static BMat bmat_of(const fvs_props& p) {
  const fvs_material& m = p.mat;
  return BMat{m.rho, m.k, m.cp, m.latent, m.T_sol, m.mu, m.beta, m.T_ref, m.g[0], m.g[1], m.g[2], m.darcy_C,
              m.darcy_eps, fs_law_of(m)};
}

struct JacobiB {
  Batch* B;
  const double* d;
  int64_t n;
  fvs_status operator()(const double* r, double* z) {
    kb_scale<<<bgrid(n, B->tiles), bblock(), 0, B->stream>>>(n, B->Sp, d, r, z); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    return FVS_OK;
  }
};
struct AmgB {
  Batch* B;
  fvs_status operator()(const double* r, double* z) {
    return B->fp32 ? bvcycle_mixed(*B, r, z) : bvcycle(*B, 0, r, z);
  }
};
struct ProjB {
  Batch* B;
  bool active() const { return true; }
  fvs_status operator()(double* v) const { return bproject(*B, v); }
};

static fvs_status batch_step(Batch& B, double dt, int& failures, int (&its)[4]) {
  fvs_mesh m = B.mesh;
  cudaStream_t st = B.stream;
  const int Sp = B.Sp;
  const int64_t Nc = m->Nc, Nf = m->Nf, Nv = m->Nv;
  const BMat mt = bmat_of(B.props);
  const dim3 blk = bblock();
  const dim3 gc = bgrid(Nc, B.tiles), gf = bgrid(Nf, B.tiles), gv = bgrid(Nv, B.tiles);
  failures = 0;
  its[0] = its[1] = its[2] = its[3] = 0;
  // phase times for FVS_DEBUG (waits for the stream at each phase end)
  const bool dbg = B.phase_ms != nullptr;
  auto t_last = std::chrono::steady_clock::now();
  auto tick = [&](int k) {
    if (!dbg) return;
    cudaStreamSynchronize(st);
    const auto now = std::chrono::steady_clock::now();
    B.phase_ms[k] += std::chrono::duration<double, std::milli>(now - t_last).count();
    t_last = now;
  };

  // 1. tags, open faces, pressure cells, face cases
  FVS_TRY(B.nlm.zero(st));
  kb_tag<<<gc, blk, 0, st>>>(Nc, Sp, B.T, mt.Ts, B.run, B.lm, B.u, B.uold, B.nlm); FVS_COUNT_LAUNCH();
  FVS_TRY(B.flow.zero(st));
  kb_faces_open<<<gf, blk, 0, st>>>(Nf, Sp, m->own, m->nei, B.lm, B.F, B.Fold, B.flow); FVS_COUNT_LAUNCH();
  kb_ppe_cells<<<gc, blk, 0, st>>>(Nc, Sp, B.lm, B.flow, B.ppe); FVS_COUNT_LAUNCH();
  kb_vertex_nonppe<<<gv, blk, 0, st>>>(Nv, Sp, m->vc_ptr, m->vc_idx, B.ppe, B.nS); FVS_COUNT_LAUNCH();
  kb_face_case<<<gf, blk, 0, st>>>(Nf, Sp, m->own, m->nei, m->fv, B.lm, B.nS, B.fcase); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();

  tick(0);
  const bool flow_on = !B.props.no_flow;
  if (flow_on) {
  // 2. momentum predictor, three components against the largest right side
  kb_mom_sys<<<gc, blk, 0, st>>>(Nc, Sp, m->W, m->Lu.col, m->Lu.val, m->V, B.fs, mt, dt, B.lm, m->cf, m->cfs,
                                 m->own, m->nei, B.F, B.Fold, B.u, B.uold, B.T, B.mdiag, B.jd, B.mrhs, B.mx);
  FVS_COUNT_LAUNCH();
  const size_t cs = (size_t)Nc * Sp;
  for (int d = 0; d < 3; ++d)
    FVS_TRY(bdot2(B, Nc, B.mrhs.p + d * cs, B.mrhs.p + d * cs, nullptr, nullptr, B_T0 + d, -1));
  kb_max3_floor<<<B.tiles, 32, 0, st>>>(Sp, B.sc, B.mfloor); FVS_COUNT_LAUNCH();
  {
    OpShared op{Nc, m->W, m->Lu.col.p, B.moff.p, B.mdiag.p, B.lm.p};
    JacobiB J{&B, B.jd.p, Nc};
    NoProj np;
    KrylovArgs a;
    a.rtol = B.props.mom_rtol;
    a.floor = B.mfloor;
    a.shape = &B.shp_mom;
    a.take = B.run;
    a.maxit = B.props.max_krylov_iters;
    for (int d = 0; d < 3; ++d) {
      int it = 0, fail = 0;
      FVS_TRY(bbicgstab(B, op, J, np, B.mrhs.p + d * cs, B.mx.p + d * cs, a, it, fail, &B.gmom[d]));
      failures += fail;
      its[0] += it;
    }
  }
  FVS_TRY(bcopy(B, 3 * cs, B.mx, B.ustar));

  tick(1);
  // 3. pressure rows, right side, per-sample hierarchy values, solve
  BPpe px;
  px.Nc = Nc; px.Nf = Nf; px.W = m->W; px.Sp = Sp;
  px.cf = m->cf; px.own = m->own; px.nei = m->nei; px.fv = m->fv; px.vc_ptr = m->vc_ptr; px.vc_idx = m->vc_idx;
  px.nb = m->nb; px.nnb = m->nnb; px.fnb = m->fnb; px.nfnb = m->nfnb; px.cfs = m->cfs;
  px.cd = m->cd; px.ce = m->ce; px.cz = m->cz; px.bdiag = B.K0.diag;
  px.ppe = B.ppe; px.fcase = B.fcase; px.nS = B.nS; px.rho = mt.rho;
  FVS_TRY(B.ocount.zero(st));
  kb_ppe_count<<<gc, blk, 0, st>>>(px, B.ocount); FVS_COUNT_LAUNCH();
  int nmod = 0;
  FVS_CUDA(cudaMemcpyAsync(&nmod, B.ocount.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  FVS_CUDA(cudaStreamSynchronize(st));
  if (nmod > B.ocap) {
    B.ocap = std::max<int64_t>(nmod, 2 * B.ocap);
    FVS_TRY(B.mval.alloc((size_t)B.ocap * m->W + 1));
    if (B.fp32) FVS_TRY(B.mvalf.alloc((size_t)B.ocap * m->W + 1));
    ++B.batch_version;   // captured solve loops hold the old row buffers
  }
  FVS_TRY(B.ocount.zero(st));
  FVS_TRY(B.err.zero(st));
  kb_ppe_rows<<<gc, blk, 0, st>>>(px, B.ovr, B.mval, B.lv[0]->dinv, B.ocount, B.ocap, B.err); FVS_COUNT_LAUNCH();
  kb_ppe_rhs<<<gc, blk, 0, st>>>(Nc, Nf, Sp, B.ppe, m->cf, m->cfs, B.fcase, m->own, m->nei, m->A, m->nrm, B.ustar,
                                 dt, B.p, B.prhs, B.px); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  {
    int e = 0;
    FVS_CUDA(cudaMemcpyAsync(&e, B.err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    FVS_CUDA(cudaStreamSynchronize(st));
    if (e) {
      set_error("batched pressure assembly failed (flags 0x%x)", e);
      return FVS_ERR_STATE;
    }
  }
  tick(2);
  if (B.fp32) {
    const int64_t nv = (int64_t)nmod * m->W;
    if (nv > 0) { kb_to_float<<<stride_grid(nv, 256), 256, 0, st>>>(nv, B.mval, B.mvalf); FVS_COUNT_LAUNCH(); }
    kb_to_float<<<stride_grid((int64_t)cs, 256), 256, 0, st>>>((int64_t)cs, B.lv[0]->dinv, B.lv[0]->dinvf);
    FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
  }
  FVS_TRY(batch_amg_values(B));
  tick(3);
  {
    OpPpe0 op = ppe_op(B);
    AmgB M{&B};
    ProjB P{&B};
    KrylovArgs a;
    a.rtol = B.props.p_rtol;
    a.take = B.run;
    a.shape = &B.lv[0]->shape;
    a.maxit = B.props.max_krylov_iters;
    int it = 0, fail = 0;
    if (m->orthogonal) FVS_TRY(bpcg(B, op, M, P, B.prhs, B.px, a, it, fail, &B.gp));
    else FVS_TRY(bbicgstab(B, op, M, P, B.prhs, B.px, a, it, fail, &B.gp));
    failures += fail;
    its[1] = it;
    FVS_TRY(bproject(B, B.px));
  }
  FVS_TRY(bcopy(B, cs, B.px, B.p));
  tick(4);

  // 4. flux and velocity correction
  kb_vertex_p<<<gv, blk, 0, st>>>(Nv, Sp, m->vc_ptr, m->vc_idx, B.ppe, B.p, B.nS, B.pv, B.fSv); FVS_COUNT_LAUNCH();
  kb_face_correct<<<gf, blk, 0, st>>>(Nf, Nc, Sp, m->own, m->nei, m->fv, B.fcase, m->fnb, m->nfnb, B.ppe, B.p,
                                      B.pv, B.fSv, m->A, m->nrm, m->cd, m->ce, m->cz, m->Jinv, B.ustar, dt, mt.rho,
                                      B.run, B.F, B.Fnew, B.gradf); FVS_COUNT_LAUNCH();
  kb_cell_correct<<<gc, blk, 0, st>>>(Nc, Nf, Sp, B.lm, m->cf, B.fcase, B.gradf, B.ustar, dt, mt.rho, B.run, B.u,
                                      B.unew); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  }   // flow_on: with natural convection off u, F and p stay zero

  tick(5);
  // 5. energy: linearised latent heat, inner solve, enthalpy inversion,
  // per-sample stop rule
  kb_energy_base<<<gc, blk, 0, st>>>(Nc, Sp, m->W, m->cf, m->cfs, m->own, m->nei, B.F, B.Fold, B.T, B.Told,
                                     B.LT.col, B.LT.val, B.lT1, B.Twall, m->V, mt, dt, B.ebase); FVS_COUNT_LAUNCH();
  kb_energy_guess<<<gc, blk, 0, st>>>(Nc, Sp, B.T, B.Told, B.fs, mt.law, B.Tliq, B.run, B.Tnew, B.fsnew);
  FVS_COUNT_LAUNCH();
  kb_energy_start<<<B.tiles, 32, 0, st>>>(Sp, B.run, B.etake, B.econv, B.ertol, B.props.e_rtol); FVS_COUNT_LAUNCH();
  {
    OpShared op{Nc, m->W, B.LT.col.p, B.kev.p, B.edx.p, nullptr};
    JacobiB J{&B, B.jd.p, Nc};
    NoProj np;
    KrylovArgs a;
    a.rtol_s = B.ertol;
    a.take = B.etake;
    a.shape = &B.shp_energy;
    a.maxit = B.props.max_krylov_iters;
    int left = 1;
    for (int it = 1; it <= B.props.max_e_iters && left > 0; ++it) {
      kb_energy_lin<<<gc, blk, 0, st>>>(Nc, Sp, m->V, mt, B.Tliq, dt, B.Tnew, B.fsnew, B.fs, B.ebase, B.kevd, B.edx,
                                        B.erhs, B.Tlin, B.jd); FVS_COUNT_LAUNCH();
      int it2 = 0, fail = 0;
      FVS_TRY(bbicgstab(B, op, J, np, B.erhs, B.Tlin, a, it2, fail, &B.ge));
      failures += fail;
      its[3] += it2;
      its[2] = it;
      kb_energy_update<<<gc, blk, 0, st>>>(Nc, Sp, mt, B.Tliq, B.etake, B.Tlin, B.Tnew, B.fsnew, B.Tit, B.fsit);
      FVS_COUNT_LAUNCH();
      FVS_TRY(bmaxdiff2(B, Nc, B.Tit, B.Tnew, B.fsit, B.fsnew, B_T0, B_T1));
      dswap_b(B.Tit, B.Tnew);
      dswap_b(B.fsit, B.fsnew);
      FVS_CUDA(cudaMemsetAsync(B.kcount.p, 0, 4 * sizeof(int), st));
      kb_energy_check<<<B.tiles, 32, 0, st>>>(Sp, B.sc, B.etake, B.econv, B.ertol, B.props.e_tol_T, B.props.e_rtol,
                                              B.kcount); FVS_COUNT_LAUNCH();
      FVS_LAUNCH_CHECK();
      int h[4];
      FVS_TRY(read_counts(B, h, 1));
      left = h[0];
    }
    if (left > 0) failures += left;
  }

  tick(6);
  // 6. crossing times, then rotate the time levels
  kb_crossings<<<gc, blk, 0, st>>>(Nc, Sp, B.T, B.Tnew, mt.Ts, B.Tliq, B.run, B.time, dt, B.tliq, B.tsol);
  FVS_COUNT_LAUNCH();
  if (B.grain_Ds > 0.0) {
    kb_grain<<<gc, blk, 0, st>>>(Nc, Sp, B.fs, B.fsnew, B.run, B.grain_kp, B.grain_Ds, dt, B.r2);
    FVS_COUNT_LAUNCH();
  }
  FVS_LAUNCH_CHECK();
  dswap_b(B.Told, B.T);
  dswap_b(B.T, B.Tnew);
  dswap_b(B.fs, B.fsnew);
  if (flow_on) {
    dswap_b(B.uold, B.u);
    dswap_b(B.u, B.unew);
    dswap_b(B.Fold, B.F);
    dswap_b(B.F, B.Fnew);
  }
  B.time += dt;
  return FVS_OK;
}

fvs_status batch_run(fvs_mesh mesh, const fvs_props* base, int64_t n, const double* inputs, double dt,
                     int max_steps, const UqSpec& spec, double* qoi, int64_t* steps) {
  if (base->n_k > 0) {
    set_error("the lockstep batch shares one conductivity operator; a k(T) table needs FVS_UQ_STREAMS");
    return FVS_ERR_ARG;
  }
  Batch B;
  B.mesh = mesh;
  FVS_CUDA(cudaStreamSynchronize(mesh->stream));
  FVS_CUDA(cudaStreamCreateWithFlags(&B.stream, cudaStreamNonBlocking));
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
  };
  fvs_status status = FVS_OK;
  {
    AllocStream as(B.stream);
    status = [&]() -> fvs_status {
      cudaStream_t st = B.stream;
      const int64_t Nc = mesh->Nc, Nf = mesh->Nf, Nv = mesh->Nv;
      const int W = mesh->W;
      B.S = n;
      B.Sp = (int)((n + 31) / 32 * 32);
      B.tiles = B.Sp / 32;
      B.props = *base;
      B.props.bc = nullptr;
      B.props.k_T = B.props.k_val = nullptr;
      B.grain_kp = spec.grain_kp;
      B.grain_Ds = spec.grain_Ds;
      B.aopt = AmgOptions();
      B.fp32 = base->precision == FVS_PREC_MIXED;
      const int Sp = B.Sp;
      // per-sample inputs
      std::vector<double> tl(Sp), tw(Sp), tm(Sp);
      std::vector<uint8_t> rn(Sp, 0);
      for (int s = 0; s < Sp; ++s) {
        if (s < n) {
          tm[s] = inputs[3 * s];
          tw[s] = inputs[3 * s + 1];
          tl[s] = spec.T_liq[s];
          if (!fs_law_valid(base->mat, tl[s])) {
            set_error("sample %d: liquidus %.3f K does not suit the solid-fraction law", s, tl[s]);
            return FVS_ERR_ARG;
          }
          rn[s] = 1;
        } else {
          tm[s] = base->mat.T_sol - 1.0;
          tw[s] = base->mat.T_sol - 1.0;
          tl[s] = base->mat.T_liq;
        }
      }
      FVS_TRY(upload(st, tl, B.Tliq));
      FVS_TRY(upload(st, tw, B.Twall));
      FVS_TRY(upload(st, tm, B.Tmelt));
      FVS_TRY(upload(st, rn, B.run));
      B.steps.assign(n, 0);
      // shared operators: temperature operator with every wall at T = 1
      {
        const int np = std::max(1, mesh->npatch);
        std::vector<int32_t> bt(np, FVS_BC_DIRICHLET);
        std::vector<double> bT(np, 1.0);
        DBuf<int32_t> dbt;
        DBuf<double> dbT;
        FVS_TRY(upload(st, bt, dbt));
        FVS_TRY(upload(st, bT, dbT));
        FVS_TRY(B.lT1.alloc(Nc + 1));
        FVS_TRY(assemble_temperature_operator(mesh, dbt, dbT, B.LT, B.lT1, st));
      }
      FVS_TRY(B.moff.alloc((size_t)Nc * W)); FVS_TRY(B.kev.alloc((size_t)Nc * W)); FVS_TRY(B.kevd.alloc(Nc));
      kb_shared_ops<<<stride_grid(Nc, 256), 256, 0, st>>>(Nc, W, base->mat.mu, base->mat.k, mesh->Lu.col, mesh->Lu.val,
                                                          B.LT.val, B.LT.diag, B.moff, B.kev, B.kevd);
      FVS_COUNT_LAUNCH();
      FVS_LAUNCH_CHECK();
      // state and work
      const size_t cs = (size_t)Nc * Sp, fsz = (size_t)Nf * Sp, vs = (size_t)Nv * Sp;
      for (DBuf<double>* b : {&B.T, &B.Told, &B.Tnew, &B.fs, &B.fsnew, &B.Tit, &B.fsit, &B.Tlin, &B.p, &B.tliq,
                              &B.tsol, &B.mdiag, &B.edx, &B.ebase, &B.erhs, &B.jd, &B.prhs, &B.px})
        FVS_TRY(b->alloc(cs + 1));
      for (DBuf<double>* b : {&B.u, &B.uold, &B.unew, &B.ustar, &B.mrhs, &B.mx}) FVS_TRY(b->alloc(3 * cs + 1));
      for (DBuf<double>* b : {&B.F, &B.Fold, &B.Fnew}) FVS_TRY(b->alloc(fsz + 1));
      FVS_TRY(B.gradf.alloc(3 * fsz + 1));
      FVS_TRY(B.pv.alloc(vs + 1)); FVS_TRY(B.fSv.alloc(vs + 1));
      FVS_TRY(B.lm.alloc(cs + 1)); FVS_TRY(B.flow.alloc(cs + 1)); FVS_TRY(B.ppe.alloc(cs + 1));
      FVS_TRY(B.fcase.alloc(fsz + 1)); FVS_TRY(B.nS.alloc(vs + 1)); FVS_TRY(B.ovr.alloc(cs + 1));
      FVS_TRY(B.mfloor.alloc(Sp)); FVS_TRY(B.econv.alloc(Sp)); FVS_TRY(B.etake.alloc(Sp)); FVS_TRY(B.ertol.alloc(Sp));
      FVS_TRY(B.nlm.alloc(Sp)); FVS_TRY(B.ocount.alloc(1)); FVS_TRY(B.err.alloc(1));
      FVS_TRY(B.sc.alloc((size_t)B_NSLOT * Sp)); FVS_TRY(B.sc.zero(st));
      FVS_TRY(B.kact.alloc(Sp)); FVS_TRY(B.krestart.alloc(Sp)); FVS_TRY(B.kcount.alloc(4));
      {
        const int64_t rows = std::max<int64_t>(std::max(Nc, Nf), Nv);
        const int nbm = red_blocks(rows, B.tiles);
        FVS_TRY(B.part.alloc((size_t)std::max(BATCH_NCM, 5) * Sp * nbm + 1));
        FVS_TRY(B.redcnt.alloc((size_t)Sp / 32 + 1));
        FVS_TRY(B.redcnt.zero(B.stream));
      }
      B.ocap = std::max<int64_t>(1024, Nc * Sp / 16);
      FVS_TRY(B.mval.alloc((size_t)B.ocap * W + 1));
      if (B.fp32) FVS_TRY(B.mvalf.alloc((size_t)B.ocap * W + 1));
      FVS_CUDA(cudaMallocHost((void**)&B.host, ((size_t)B_NSLOT * Sp + 64) * sizeof(double)));
      kb_init<<<bgrid(std::max(Nc, Nf), B.tiles), bblock(), 0, st>>>(Nc, Nf, Sp, B.Tmelt, B.Tliq, fs_law_of(base->mat),
                                                                      B.run, B.T, B.Told, B.fs, B.u, B.uold, B.p,
                                                                      B.tliq, B.tsol, B.F, B.Fold);
      FVS_COUNT_LAUNCH();
      FVS_LAUNCH_CHECK();
      if (spec.grain_Ds > 0.0) {
        FVS_TRY(B.r2.alloc(cs + 1));
        kb_fill<<<stride_grid((int64_t)cs, 256), 256, 0, st>>>(cs, spec.grain_r0 * spec.grain_r0, B.r2);
        FVS_COUNT_LAUNCH();
        FVS_LAUNCH_CHECK();
      }
      // natural convection off: no pressure system, so no hierarchy
      if (!base->no_flow) FVS_TRY(batch_amg_setup(B));
      {
        // launch shapes of the shared momentum and energy operators (FP64,
        // every row doing its full work)
        FVS_TRY(B.kw.ensure(cs));
        for (DBuf<double>* b : {&B.kw.r, &B.kw.p, &B.kw.v, &B.mdiag, &B.edx})
          FVS_CUDA(cudaMemsetAsync(b->p, 0, cs * sizeof(double), st));
        FVS_TRY(build_stage(st, Nc, W, mesh->Lu.col.p, 8, B.stage_m));
        FVS_TRY(build_stage(st, Nc, W, B.LT.col.p, 8, B.stage_e));
        FVS_TRY(tune_apply(B, OpShared{Nc, W, mesh->Lu.col.p, B.moff.p, B.mdiag.p, nullptr}, B.kw.r.p, B.kw.p.p,
                           B.kw.v.p, B.mdiag.p, B.shp_mom, &B.stage_m));
        FVS_TRY(tune_apply(B, OpShared{Nc, W, B.LT.col.p, B.kev.p, B.edx.p, nullptr}, B.kw.r.p, B.kw.p.p, B.kw.v.p,
                           B.edx.p, B.shp_energy, &B.stage_e));
        if (getenv("FVS_DEBUG"))
          fprintf(stderr, "[fvs batch] momentum shape %d x %d, energy shape %d x %d\n", B.shp_mom.rows,
                  B.shp_mom.per_sm, B.shp_energy.rows, B.shp_energy.per_sm);
      }
      // steps until every sample has taken the step that began fully solid
      std::vector<int> nlm(Sp);
      std::vector<uint8_t> runh = rn;
      int64_t left = n;
      int64_t total_fails = 0;
      const bool dbg = getenv("FVS_DEBUG") != nullptr;
      double phase[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      if (dbg) B.phase_ms = phase;
      for (int k = 0; k < max_steps && left > 0; ++k) {
        int fails = 0, its[4];
        FVS_TRY(batch_step(B, dt, fails, its));
        total_fails += fails;
        if (dbg)
          fprintf(stderr, "[fvs batch] step %d: momentum %d, pressure %d, energy passes %d (inner %d), "
                  "unconverged solves %d\n", k, its[0], its[1], its[2], its[3], fails);
        FVS_CUDA(cudaMemcpyAsync(nlm.data(), B.nlm.p, Sp * sizeof(int), cudaMemcpyDeviceToHost, st));
        FVS_CUDA(cudaStreamSynchronize(st));
        bool changed = false;
        for (int s = 0; s < n; ++s) {
          if (!runh[s]) continue;
          ++B.steps[s];
          if (nlm[s] == 0) { runh[s] = 0; changed = true; --left; }
        }
        if (changed) FVS_CUDA(cudaMemcpyAsync(B.run.p, runh.data(), Sp, cudaMemcpyHostToDevice, st));
      }
      if (dbg)
        fprintf(stderr, "[fvs batch] phase ms: tags %.1f momentum %.1f pressure rows %.1f amg values %.1f "
                "pressure solve %.1f correction %.1f energy %.1f\n", phase[0], phase[1], phase[2], phase[3],
                phase[4], phase[5], phase[6]);
      B.phase_ms = nullptr;
      // per-sample means over the solidified cells (Eq. 22-23), or the
      // domain extremes of Section 5
      const int nb = red_blocks(Nc, B.tiles);
      const bool ext = spec.qoi_kind == FVS_QOI_EXTREMES;
      DBuf<double> out;
      FVS_TRY(out.alloc((size_t)5 * Sp));
      if (ext) {
        kb_qoi_ext_part<<<dim3(nb, B.tiles), bblock(), 0, st>>>(Nc, Sp, B.tliq, B.tsol, base->mat.T_sol, B.Tliq,
                                                                 spec.grain_Ds > 0.0 ? B.r2.p : nullptr, B.part);
        FVS_COUNT_LAUNCH();
        kb_qoi_ext_final<<<B.tiles, 32, 0, st>>>(nb, Sp, B.part, out); FVS_COUNT_LAUNCH();
      } else {
        kb_qoi_part<<<dim3(nb, B.tiles), bblock(), 0, st>>>(Nc, Sp, B.tliq, B.tsol, base->mat.T_sol, B.Tliq, B.part);
        FVS_COUNT_LAUNCH();
        kb_qoi_final<<<B.tiles, 32, 0, st>>>(nb, Sp, B.part, out); FVS_COUNT_LAUNCH();
      }
      FVS_LAUNCH_CHECK();
      std::vector<double> h((size_t)5 * Sp);
      FVS_CUDA(cudaMemcpyAsync(h.data(), out.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
      FVS_CUDA(cudaStreamSynchronize(st));
      const double nan = std::nan("");
      for (int64_t i = 0; i < n; ++i) {
        if (ext) {
          const bool all_solid = h[(size_t)4 * Sp + i] == 0.0;
          const double tmax = h[i], lmax = h[(size_t)Sp + i];
          qoi[4 * i + 0] = all_solid && tmax >= 0.0 ? tmax : nan;
          qoi[4 * i + 1] = lmax >= 0.0 ? lmax : nan;
          qoi[4 * i + 2] = lmax >= 0.0 ? h[(size_t)2 * Sp + i] : nan;
          qoi[4 * i + 3] = h[(size_t)3 * Sp + i];
        } else {
          const double cnt = h[(size_t)4 * Sp + i];
          for (int q = 0; q < 4; ++q) qoi[4 * i + q] = cnt > 0 ? h[(size_t)q * Sp + i] / cnt : nan;
        }
        if (steps) steps[i] = B.steps[i];
      }
      // final fields of every sample in the caller's cell order
      if (spec.T_out || spec.p_out || spec.u_out) {
        DBuf<double> buf;
        FVS_TRY(buf.alloc((size_t)3 * Nc + 1));
        const int g = stride_grid(Nc, 256);
        struct Out { double* dst; const double* src; int comps; };
        const Out outs[3] = {{spec.T_out, B.T.p, 1}, {spec.p_out, B.p.p, 1}, {spec.u_out, B.u.p, 3}};
        for (const Out& o : outs) {
          if (!o.dst) continue;
          for (int64_t i = 0; i < n; ++i) {
            kb_field_out<<<g, 256, 0, st>>>(Nc, Sp, (int)i, o.comps, mesh->cell_in, o.src, buf.p);
            FVS_COUNT_LAUNCH();
            FVS_LAUNCH_CHECK();
            FVS_CUDA(cudaMemcpyAsync(o.dst + i * o.comps * Nc, buf.p, (size_t)o.comps * Nc * sizeof(double),
                                     cudaMemcpyDeviceToHost, st));
          }
        }
        FVS_CUDA(cudaStreamSynchronize(st));
      }
      if (total_fails > 0) {
        set_error("lockstep batch: %lld sample solves stayed above their tolerance", (long long)total_fails);
        return FVS_ERR_NOT_CONVERGED;
      }
      return FVS_OK;
    }();
    FVS_CUDA(cudaStreamSynchronize(B.stream));
  }
  StreamGuard g{B.stream};
  return status;
}

}  // namespace fvs
