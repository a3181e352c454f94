// Aggregation AMG: setup (strength, parallel MIS aggregation, Galerkin
// coarse operators, pinned dense coarsest inverse, component labels) and the
// V-cycle (damped Jacobi, piecewise-constant restriction / prolongation).
#include <algorithm>
#include <climits>
#include <cstdlib>

#include "amg.cuh"

namespace fvs {

#define GS(i, n) for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

static constexpr int GAL_CAP = 2048;   // entries gathered per coarse row

// ---------------------------------------------------------------------------
// strength of connection: j is strong for i if -a_ij >= theta max_k(-a_ik)
// (or the same holds with i and j exchanged, to keep the graph symmetric)
// ---------------------------------------------------------------------------
__global__ void k_maxoff(int64_t n, int w, const int32_t* col, const double* val, double* mo, double* dinv,
                         const double* diag) {
  GS(i, n) {
    double m = 0.0;
    for (int k = 0; k < w; ++k) {
      const int64_t e = (int64_t)k * n + i;
      if (col[e] != (int32_t)i) m = fmax(m, -val[e]);
    }
    mo[i] = m;
    dinv[i] = 1.0 / diag[i];
  }
}

__global__ void k_strong(int64_t n, int w, const int32_t* col, const double* val, const double* mo, double theta,
                         uint64_t* mask) {
  GS(i, n) {
    uint64_t msk = 0;
    for (int k = 0; k < w; ++k) {
      const int64_t e = (int64_t)k * n + i;
      const int32_t j = col[e];
      if (j == (int32_t)i) continue;
      const double a = -val[e];
      bool s = a > 0.0 && a >= theta * mo[i];
      if (!s) {
        for (int q = 0; q < w; ++q) {
          const int64_t ej = (int64_t)q * n + j;
          if (col[ej] == (int32_t)i) {
            const double b = -val[ej];
            s = b > 0.0 && b >= theta * mo[j];
            break;
          }
        }
      }
      if (s) msk |= (1ULL << k);
    }
    mask[i] = msk;
  }
}

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
  x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16;
  return x;
}
__device__ __forceinline__ bool beats(int32_t j, int32_t i) {
  const uint32_t hj = hash32((uint32_t)j), hi = hash32((uint32_t)i);
  return hj > hi || (hj == hi && j > i);
}

// Luby rounds of a maximal independent set on the strong graph:
// state 0 undecided, 1 root, 2 out
__global__ void k_mis_select(int64_t n, int w, const int32_t* col, const uint64_t* mask, const uint8_t* st,
                             uint8_t* st2) {
  GS(i, n) {
    uint8_t s = st[i];
    if (s == 0) {
      bool top = true;
      uint64_t m = mask[i];
      while (m) {
        const int k = __ffsll((long long)m) - 1;
        m &= m - 1;
        const int32_t j = col[(int64_t)k * n + i];
        if (st[j] == 0 && beats(j, (int32_t)i)) { top = false; break; }
      }
      if (top) s = 1;
    }
    st2[i] = s;
  }
}
__global__ void k_mis_remove(int64_t n, int w, const int32_t* col, const uint64_t* mask, const uint8_t* st2,
                             uint8_t* st, int* undecided) {
  int cnt = 0;
  GS(i, n) {
    uint8_t s = st2[i];
    if (s == 0) {
      uint64_t m = mask[i];
      while (m) {
        const int k = __ffsll((long long)m) - 1;
        m &= m - 1;
        if (st2[col[(int64_t)k * n + i]] == 1) { s = 2; break; }
      }
      if (s == 0) ++cnt;
    }
    st[i] = s;
  }
  if (cnt) atomicAdd(undecided, cnt);
}
__global__ void k_is_root(int64_t n, const uint8_t* st, int32_t* flag) {
  GS(i, n) flag[i] = st[i] == 1 ? 1 : 0;
}
// every non-root joins its strongest root neighbour (ties: lower index)
__global__ void k_assign(int64_t n, int w, const int32_t* col, const double* val, const uint64_t* mask,
                         const uint8_t* st, const int32_t* rid, int32_t* agg, int* err) {
  GS(i, n) {
    if (st[i] == 1) { agg[i] = rid[i]; continue; }
    double best = -1e300;
    int32_t bj = -1;
    uint64_t m = mask[i];
    while (m) {
      const int k = __ffsll((long long)m) - 1;
      m &= m - 1;
      const int64_t e = (int64_t)k * n + i;
      const int32_t j = col[e];
      if (st[j] != 1) continue;
      const double a = -val[e];
      if (a > best || (a == best && j < bj)) { best = a; bj = j; }
    }
    if (bj < 0) { atomicOr(err, 1); agg[i] = 0; } else agg[i] = rid[bj];
  }
}

__global__ void k_count_members(int64_t n, const int32_t* agg, int32_t* cnt) {
  GS(i, n) atomicAdd(&cnt[agg[i]], 1);
}
__global__ void k_fill_members(int64_t n, const int32_t* agg, const int32_t* ptr, int32_t* cur, int32_t* idx) {
  GS(i, n) {
    const int32_t a = agg[i];
    idx[ptr[a] + atomicAdd(&cur[a], 1)] = (int32_t)i;
  }
}
__global__ void k_sort_members(int64_t nc, const int32_t* ptr, int32_t* idx) {
  GS(I, nc) {
    const int32_t lo = ptr[I], hi = ptr[I + 1];
    for (int32_t a = lo + 1; a < hi; ++a)
      for (int32_t b = a; b > lo && idx[b - 1] > idx[b]; --b) {
        const int32_t t = idx[b]; idx[b] = idx[b - 1]; idx[b - 1] = t;
      }
  }
}

// ---------------------------------------------------------------------------
// Galerkin product with piecewise-constant transfers:
//   Ac[I][J] = sum_{i in I} sum_{j in J} a_ij
// one warp per coarse row: gather (agg[col], val) of all member rows into
// shared memory, bitonic-sort by key, reduce equal keys in a fixed order
// (deterministic).  Pass 1 counts entries, pass 2 writes the ELL rows.
// ---------------------------------------------------------------------------
template <bool FILL>
__global__ void __launch_bounds__(32) k_galerkin(int64_t nc, int64_t n, int w, const int32_t* col, const double* val,
                                                 const int32_t* agg, const int32_t* mptr, const int32_t* midx,
                                                 int32_t* rowlen, int wc, int32_t* ccol, double* cval, double* cdiag,
                                                 int* err) {
  __shared__ int32_t key[GAL_CAP];
  __shared__ double v[GAL_CAP];
  const int lane = threadIdx.x;
  for (int64_t I = blockIdx.x; I < nc; I += gridDim.x) {
    const int32_t lo = mptr[I], hi = mptr[I + 1];
    const int total = (hi - lo) * w;
    if (total > GAL_CAP) {
      if (lane == 0) { atomicOr(err, 2); if (!FILL) rowlen[I] = 0; }
      continue;
    }
    int P = 32;
    while (P < total) P <<= 1;
    for (int e = lane; e < P; e += 32) {
      if (e < total) {
        const int m = e / w, k = e - m * w;
        const int32_t i = midx[lo + m];
        const int64_t ei = (int64_t)k * n + i;
        const double a = val[ei];
        key[e] = a != 0.0 ? agg[col[ei]] : INT_MAX;
        v[e] = a;
      } else {
        key[e] = INT_MAX;
        v[e] = 0.0;
      }
    }
    __syncwarp();
    for (int size = 2; size <= P; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int e = lane; e < P; e += 32) {
          const int p = e ^ stride;
          if (p > e) {
            const bool up = (e & size) == 0;
            const int32_t ke = key[e], kp = key[p];
            if ((ke > kp) == up && ke != kp) {
              key[e] = kp; key[p] = ke;
              const double t = v[e]; v[e] = v[p]; v[p] = t;
            }
          }
        }
        __syncwarp();
      }
    }
    // segment heads
    int base = 0;
    for (int e0 = 0; e0 < P; e0 += 32) {
      const int e = e0 + lane;
      const bool head = key[e] != INT_MAX && (e == 0 || key[e - 1] != key[e]);
      const unsigned bal = __ballot_sync(0xffffffffu, head);
      if (FILL && head) {
        const int r = base + __popc(bal & ((1u << lane) - 1));
        double s = 0.0;
        for (int q = e; q < P && key[q] == key[e]; ++q) s += v[q];
        if (r < wc) {
          ccol[(int64_t)r * nc + I] = key[e];
          cval[(int64_t)r * nc + I] = s;
        } else {
          atomicOr(err, 4);
        }
        if (key[e] == (int32_t)I) cdiag[I] = s;
      }
      base += __popc(bal);
    }
    if (!FILL) {
      if (lane == 0) rowlen[I] = base;
    } else {
      for (int r = base + lane; r < wc; r += 32) {
        ccol[(int64_t)r * nc + I] = (int32_t)I;
        cval[(int64_t)r * nc + I] = 0.0;
      }
    }
    __syncwarp();
  }
}

__global__ void k_max_int(int64_t n, const int32_t* a, int* out) {
  int m = 0;
  GS(i, n) m = max(m, (int)a[i]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// ---------------------------------------------------------------------------
// coarsest level: dense copy, connected parts, pins, Gauss-Jordan inverse
// (one block; n <= AmgOptions::coarsest)
// ---------------------------------------------------------------------------
__global__ void k_coarsest(int n, int w, const int32_t* col, const double* val, double* M, double* Ainv,
                           int32_t* lab, uint8_t* sing, int* ncomp_out, int* err) {
  extern __shared__ double shd[];
  double* fac = shd;                 // [n]
  __shared__ int piv;
  __shared__ double pmax;
  const int n2 = 2 * n;
  // augmented [D | I]
  for (int e = threadIdx.x; e < n * n2; e += blockDim.x) M[e] = 0.0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    for (int k = 0; k < w; ++k) M[(int64_t)i * n2 + col[(int64_t)k * n + i]] += val[(int64_t)k * n + i];
    M[(int64_t)i * n2 + n + i] = 1.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // connected parts by breadth-first search over the symmetric pattern
    for (int i = 0; i < n; ++i) lab[i] = -1;
    int nc = 0;
    int* queue = (int*)(fac);       // reuse shared memory as a queue (n ints fit in n doubles)
    for (int s0 = 0; s0 < n; ++s0) {
      if (lab[s0] >= 0) continue;
      int qh = 0, qt = 0;
      queue[qt++] = s0;
      lab[s0] = nc;
      while (qh < qt) {
        const int i = queue[qh++];
        for (int j = 0; j < n; ++j)
          if (lab[j] < 0 && (M[(int64_t)i * n2 + j] != 0.0 || M[(int64_t)j * n2 + i] != 0.0)) {
            lab[j] = nc;
            queue[qt++] = j;
          }
      }
      ++nc;
    }
    // singular parts: row sums vanish; pin the first unknown of each
    for (int c = 0; c < nc; ++c) {
      double rs = 0.0, sc = 0.0;
      int first = -1;
      for (int i = 0; i < n; ++i) {
        if (lab[i] != c) continue;
        if (first < 0) first = i;
        for (int j = 0; j < n; ++j) rs += M[(int64_t)i * n2 + j];
        sc += fabs(M[(int64_t)i * n2 + i]);
      }
      const bool sg = fabs(rs) <= 1e-9 * sc;
      sing[c] = sg ? 1 : 0;
      if (sg) {
        for (int j = 0; j < n; ++j) M[(int64_t)first * n2 + j] = 0.0;
        M[(int64_t)first * n2 + first] = 1.0;
      }
    }
    *ncomp_out = nc;
  }
  __syncthreads();
  // Gauss-Jordan with partial pivoting
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      int p = k;
      double best = fabs(M[(int64_t)k * n2 + k]);
      for (int i = k + 1; i < n; ++i) {
        const double a = fabs(M[(int64_t)i * n2 + k]);
        if (a > best) { best = a; p = i; }
      }
      piv = p;
      pmax = best;
    }
    __syncthreads();
    if (!(pmax > 1e-300)) {
      if (threadIdx.x == 0) atomicOr(err, 8);
      return;
    }
    if (piv != k) {
      for (int j = threadIdx.x; j < n2; j += blockDim.x) {
        const double t = M[(int64_t)k * n2 + j];
        M[(int64_t)k * n2 + j] = M[(int64_t)piv * n2 + j];
        M[(int64_t)piv * n2 + j] = t;
      }
    }
    __syncthreads();
    const double inv = 1.0 / M[(int64_t)k * n2 + k];
    __syncthreads();
    for (int j = threadIdx.x; j < n2; j += blockDim.x) M[(int64_t)k * n2 + j] *= inv;
    for (int i = threadIdx.x; i < n; i += blockDim.x) fac[i] = M[(int64_t)i * n2 + k];
    __syncthreads();
    for (int e = threadIdx.x; e < n * n2; e += blockDim.x) {
      const int i = e / n2, j = e - i * n2;
      if (i != k) M[e] -= fac[i] * M[(int64_t)k * n2 + j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e - i * n;
    Ainv[e] = M[(int64_t)i * n2 + n + j];
  }
  __syncthreads();
  // fold the projections onto zero-mean parts into the inverse:
  // Ainv <- P Ainv P, P v = v - (mean of v on each singular part)
  int* order = (int*)fac;           // rows grouped by part (n ints)
  __shared__ int ncs;
  if (threadIdx.x == 0) {
    ncs = *ncomp_out;
    int pos = 0;
    for (int c = 0; c < ncs; ++c)
      for (int i = 0; i < n; ++i)
        if (lab[i] == c) order[pos++] = i;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {      // left: column j
    int pos = 0;
    for (int c = 0; c < ncs; ++c) {
      int cnt = 0;
      double sum = 0.0;
      for (int q = pos; q < n && lab[order[q]] == c; ++q, ++cnt) sum += Ainv[(int64_t)order[q] * n + j];
      if (sing[c]) {
        const double m = sum / (double)cnt;
        for (int q = pos; q < pos + cnt; ++q) Ainv[(int64_t)order[q] * n + j] -= m;
      }
      pos += cnt;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {      // right: row i
    int pos = 0;
    for (int c = 0; c < ncs; ++c) {
      int cnt = 0;
      double sum = 0.0;
      for (int q = pos; q < n && lab[order[q]] == c; ++q, ++cnt) sum += Ainv[(int64_t)i * n + order[q]];
      if (sing[c]) {
        const double m = sum / (double)cnt;
        for (int q = pos; q < pos + cnt; ++q) Ainv[(int64_t)i * n + order[q]] -= m;
      }
      pos += cnt;
    }
  }
}

// coarsest solve: y = Ainv b with the projections already folded into Ainv;
// one warp per row, FP64 arithmetic whatever the vector type
template <typename T>
__global__ void k_coarse_solve(int n, const double* __restrict__ Ainv, const T* __restrict__ b, T* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= n) return;
  double a = 0.0;
  for (int j = lane; j < n; j += 32) a = fma(Ainv[(int64_t)row * n + j], (double)b[j], a);
  a = warp_sum(a);
  if (lane == 0) y[row] = (T)a;
}

// ---------------------------------------------------------------------------
// V-cycle kernels
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_jac0(int64_t n, T omega, const T* dinv, const T* b, T* x) {
  GS(i, n) x[i] = omega * dinv[i] * b[i];
}
// y = x + omega D^-1 (b - A x)
template <typename T>
__global__ void k_jac(int64_t n, int w, const int32_t* __restrict__ col, const T* __restrict__ val, T omega,
                      const T* __restrict__ dinv, const T* __restrict__ b, const T* __restrict__ x,
                      T* __restrict__ y) {
  GS(i, n) {
    T acc = 0;
    for (int k = 0; k < w; ++k) {
      const int64_t e = (int64_t)k * n + i;
      acc = fma(val[e], x[col[e]], acc);
    }
    y[i] = x[i] + omega * dinv[i] * (b[i] - acc);
  }
}
template <typename T>
__global__ void k_resid(int64_t n, int w, const int32_t* __restrict__ col, const T* __restrict__ val,
                        const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ r) {
  GS(i, n) {
    T acc = 0;
    for (int k = 0; k < w; ++k) {
      const int64_t e = (int64_t)k * n + i;
      acc = fma(val[e], x[col[e]], acc);
    }
    r[i] = b[i] - acc;
  }
}
template <typename T>
__global__ void k_restrict(int64_t nc, const int32_t* mptr, const int32_t* midx, const T* r, T* bc) {
  GS(I, nc) {
    T s = 0;
    for (int32_t m = mptr[I]; m < mptr[I + 1]; ++m) s += r[midx[m]];
    bc[I] = s;
  }
}
template <typename T>
__global__ void k_prolong(int64_t n, const int32_t* agg, const T* yc, T scale, T* x) {
  GS(i, n) x[i] += scale * yc[agg[i]];
}
template <typename A, typename B>
__global__ void k_convert(int64_t n, const A* a, B* b) {
  GS(i, n) b[i] = (B)a[i];
}

// label propagation down the hierarchy and per-component counts
__global__ void k_pull_labels(int64_t n, const int32_t* agg, const int32_t* lab_c, int32_t* lab) {
  GS(i, n) lab[i] = lab_c[agg[i]];
}
__global__ void k_copy_i32(int64_t n, const int32_t* a, int32_t* b) {
  GS(i, n) b[i] = a[i];
}
__global__ void k_comp_count(int64_t n, const int32_t* lab, double* cnt) {
  GS(i, n) atomicAdd(&cnt[lab[i]], 1.0);
}
__global__ void k_comp_sum(int64_t n, const int32_t* lab, const double* v, double* s) {
  GS(i, n) atomicAdd(&s[lab[i]], v[i]);
}
__global__ void k_comp_sub(int64_t n, const int32_t* lab, const uint8_t* sing, const double* s, const double* cnt,
                           double* v) {
  GS(i, n) {
    const int32_t c = lab[i];
    if (sing[c]) v[i] -= s[c] / cnt[c];
  }
}
// single component: deterministic mean via block partials
__global__ void k_sum_part(int64_t n, const double* v, double* part) {
  __shared__ double sh[32];
  double a = 0.0;
  GS(i, n) a += v[i];
  a = block_sum(a, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = a;
}
__global__ void k_mean_final(int nb, const double* part, double cnt, double* mean) {
  __shared__ double sh[32];
  double a = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) a += part[b];
  a = block_sum(a, sh);
  if (threadIdx.x == 0) *mean = a / cnt;
}
__global__ void k_sub_scalar(int64_t n, const double* mean, double* v) {
  const double m = *mean;
  GS(i, n) v[i] -= m;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static fvs_status read_int(cudaStream_t s, const int* d, int* h) {
  FVS_CUDA(cudaMemcpyAsync(h, d, sizeof(int), cudaMemcpyDeviceToHost, s));
  FVS_CUDA(cudaStreamSynchronize(s));
  return FVS_OK;
}

static double env_num(const char* name, double dflt) {
  const char* v = getenv(name);
  return (v && *v) ? atof(v) : dflt;
}

fvs_status Amg::setup(cudaStream_t s, const Ell& A) {
  ready = false;
  lv.clear();
  opt.theta = env_num("FVS_AMG_THETA", opt.theta);
  opt.omega = env_num("FVS_AMG_OMEGA", opt.omega);
  opt.coarse_scale = env_num("FVS_AMG_SCALE", opt.coarse_scale);
  opt.npre = (int)env_num("FVS_AMG_NPRE", opt.npre);
  opt.npost = (int)env_num("FVS_AMG_NPOST", opt.npost);
  opt.coarsest = (int)env_num("FVS_AMG_COARSEST", opt.coarsest);
  if (opt.npre < 1) opt.npre = 1;
  if (opt.npost < 1) opt.npost = 1;
  DBuf<int> err, cnt;
  FVS_TRY(err.alloc(1));
  FVS_TRY(cnt.alloc(2));
  FVS_TRY(err.zero(s));
  {
    std::unique_ptr<AmgLevel> L0(new AmgLevel());
    L0->A = &A;
    lv.push_back(std::move(L0));
  }
  for (int l = 0;; ++l) {
    AmgLevel* L = lv[l].get();
    const Ell* cur = L->A;
    const int64_t n = cur->n;
    L->n = n;
    FVS_TRY(L->dinv.alloc(n + 1));
    FVS_TRY(L->b.alloc(n + 1)); FVS_TRY(L->x.alloc(n + 1)); FVS_TRY(L->y.alloc(n + 1)); FVS_TRY(L->r.alloc(n + 1));
    FVS_TRY(L->t.alloc(n + 1));
    DBuf<double> mo;
    FVS_TRY(mo.alloc(n + 1));
    if (n > 0) {
      k_maxoff<<<stride_grid(n, 256), 256, 0, s>>>(n, cur->w, cur->col, cur->val, mo, L->dinv, cur->diag); FVS_COUNT_LAUNCH();
      FVS_LAUNCH_CHECK();
    }
    if (n <= opt.coarsest || l + 1 >= opt.max_levels || cur->w > 64) break;
    // strength and aggregation
    DBuf<uint64_t> mask;
    DBuf<uint8_t> st, st2;
    FVS_TRY(mask.alloc(n)); FVS_TRY(st.alloc(n)); FVS_TRY(st2.alloc(n));
    FVS_TRY(st.zero(s));
    k_strong<<<stride_grid(n, 256), 256, 0, s>>>(n, cur->w, cur->col, cur->val, mo, opt.theta, mask); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    for (int round = 0;; ++round) {
      FVS_TRY(cnt.zero(s));
      k_mis_select<<<stride_grid(n, 256), 256, 0, s>>>(n, cur->w, cur->col, mask, st, st2); FVS_COUNT_LAUNCH();
      k_mis_remove<<<stride_grid(n, 256), 256, 0, s>>>(n, cur->w, cur->col, mask, st2, st, cnt); FVS_COUNT_LAUNCH();
      FVS_LAUNCH_CHECK();
      int und = 0;
      FVS_TRY(read_int(s, cnt, &und));
      if (und == 0) break;
      if (round == 63) {
        set_error("AMG aggregation did not finish");
        return FVS_ERR_NOT_CONVERGED;
      }
    }
    DBuf<int32_t> flag, rid;
    FVS_TRY(flag.alloc(n + 1)); FVS_TRY(rid.alloc(n + 1));
    FVS_TRY(flag.zero(s));
    k_is_root<<<stride_grid(n, 256), 256, 0, s>>>(n, st, flag); FVS_COUNT_LAUNCH();
    FVS_TRY(exclusive_scan(s, sw, n + 1, flag, rid));
    int nc = 0;
    FVS_CUDA(cudaMemcpyAsync(&nc, rid.p + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    FVS_CUDA(cudaStreamSynchronize(s));
    if (nc <= 0 || nc >= n || (double)nc > 0.85 * (double)n) break;  // stagnation: L is the coarsest
    FVS_TRY(L->agg.alloc(n));
    k_assign<<<stride_grid(n, 256), 256, 0, s>>>(n, cur->w, cur->col, cur->val, mask, st, rid, L->agg, err); FVS_COUNT_LAUNCH();
    DBuf<int32_t> mc;
    FVS_TRY(mc.alloc(nc + 1));
    FVS_TRY(mc.zero(s));
    FVS_TRY(L->mptr.alloc(nc + 1));
    FVS_TRY(L->midx.alloc(n));
    k_count_members<<<stride_grid(n, 256), 256, 0, s>>>(n, L->agg, mc); FVS_COUNT_LAUNCH();
    FVS_TRY(exclusive_scan(s, sw, nc + 1, mc, L->mptr));
    FVS_TRY(mc.zero(s));
    k_fill_members<<<stride_grid(n, 256), 256, 0, s>>>(n, L->agg, L->mptr, mc, L->midx); FVS_COUNT_LAUNCH();
    k_sort_members<<<stride_grid(nc, 256), 256, 0, s>>>(nc, L->mptr, L->midx); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    DBuf<int32_t> rowlen;
    FVS_TRY(rowlen.alloc(nc));
    const int gb = (int)std::min<int64_t>((int64_t)nc, (int64_t)sm_count() * 32);
    k_galerkin<false><<<gb, 32, 0, s>>>(nc, n, cur->w, cur->col, cur->val, L->agg, L->mptr, L->midx, rowlen, 0,
                                        nullptr, nullptr, nullptr, err); FVS_COUNT_LAUNCH();
    FVS_TRY(cnt.zero(s));
    k_max_int<<<stride_grid(nc, 256), 256, 0, s>>>(nc, rowlen, cnt); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    int wc = 0, e = 0;
    FVS_TRY(read_int(s, cnt, &wc));
    FVS_TRY(read_int(s, err, &e));
    if (e) {
      set_error("AMG setup failed (flags 0x%x) at level %d", e, l);
      return FVS_ERR_NOT_CONVERGED;
    }
    std::unique_ptr<AmgLevel> C(new AmgLevel());
    FVS_TRY(C->own.alloc(nc, wc));
    FVS_TRY(C->own.diag.zero(s));
    k_galerkin<true><<<gb, 32, 0, s>>>(nc, n, cur->w, cur->col, cur->val, L->agg, L->mptr, L->midx, rowlen, wc,
                                       C->own.col, C->own.val, C->own.diag, err); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    C->A = &C->own;
    lv.push_back(std::move(C));
  }
  {
    int e = 0;
    FVS_TRY(read_int(s, err, &e));
    if (e) {
      set_error("AMG setup failed (flags 0x%x)", e);
      return FVS_ERR_NOT_CONVERGED;
    }
  }
  FVS_TRY(coarsest_setup(s));
  if (opt.fp32) FVS_TRY(setup_fp32(s));
  if (getenv("FVS_DEBUG")) {
    fprintf(stderr, "[fvs amg] levels %d:", (int)lv.size());
    for (auto& L : lv) fprintf(stderr, " %lld(w%d)", (long long)L->n, L->A->w);
    fprintf(stderr, " coarsest %d parts %d\n", nc, ncomp);
  }
  ready = true;
  return FVS_OK;
}

fvs_status Amg::coarsest_setup(cudaStream_t s) {
  AmgLevel* L = lv.back().get();
  const Ell& A = *L->A;
  nc = (int)A.n;
  if (nc > 4 * opt.coarsest) {
    set_error("AMG coarsest level too large (%d rows)", nc);
    return FVS_ERR_NOT_CONVERGED;
  }
  DBuf<double> M;
  DBuf<int> err, ncd;
  FVS_TRY(M.alloc((size_t)2 * nc * nc + 1));
  FVS_TRY(Ainv.alloc((size_t)nc * nc + 1));
  FVS_TRY(clab.alloc(nc + 1));
  FVS_TRY(csing.alloc(nc + 1));
  FVS_TRY(err.alloc(1)); FVS_TRY(ncd.alloc(1));
  FVS_TRY(err.zero(s));
  if (nc > 0) {
    k_coarsest<<<1, 512, (size_t)nc * sizeof(double) + 64, s>>>(nc, A.w, A.col, A.val, M, Ainv, clab, csing, ncd, err); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
  }
  int e = 0, ncomp_c = 0;
  FVS_TRY(read_int(s, err, &e));
  if (nc > 0) FVS_TRY(read_int(s, ncd, &ncomp_c));
  if (e) {
    set_error("AMG coarsest inverse failed (zero pivot)");
    return FVS_ERR_NOT_CONVERGED;
  }
  ncomp = ncomp_c;
  sing_host.assign(ncomp, 0);
  if (ncomp > 0) FVS_CUDA(cudaMemcpyAsync(sing_host.data(), csing.p, ncomp, cudaMemcpyDeviceToHost, s));
  // labels of the fine rows through the aggregation chain
  const int64_t n0 = lv[0]->n;
  FVS_TRY(fine_lab.alloc(n0 + 1));
  DBuf<int32_t> tmp;
  FVS_TRY(tmp.alloc(n0 + 1));
  DBuf<int32_t> tmp2;
  FVS_TRY(tmp2.alloc(n0 + 1));
  if (lv.size() == 1) {
    k_copy_i32<<<stride_grid(n0 + 1, 256), 256, 0, s>>>(n0, clab, fine_lab); FVS_COUNT_LAUNCH();
  } else {
    // from the coarsest down: lab_l[i] = lab_{l+1}[agg_l[i]]
    const int32_t* up = clab;
    for (int l = (int)lv.size() - 2; l >= 0; --l) {
      int32_t* out = l == 0 ? fine_lab.p : ((l & 1) ? tmp.p : tmp2.p);
      k_pull_labels<<<stride_grid(lv[l]->n, 256), 256, 0, s>>>(lv[l]->n, lv[l]->agg, up, out); FVS_COUNT_LAUNCH();
      up = out;
    }
  }
  FVS_LAUNCH_CHECK();
  FVS_TRY(ccnt.alloc(ncomp + 1));
  FVS_TRY(csum.alloc(ncomp + 1));
  FVS_TRY(ccnt.zero(s));
  if (n0 > 0) { k_comp_count<<<stride_grid(n0, 256), 256, 0, s>>>(n0, fine_lab, ccnt); FVS_COUNT_LAUNCH(); }
  FVS_TRY(cpart.alloc(1025));
  FVS_LAUNCH_CHECK();
  FVS_CUDA(cudaStreamSynchronize(s));
  return FVS_OK;
}

fvs_status Amg::project(cudaStream_t s, double* v) {
  const int64_t n = lv[0]->n;
  if (n == 0 || ncomp == 0) return FVS_OK;
  if (ncomp == 1) {
    if (!sing_host[0]) return FVS_OK;
    const int nb = std::min(1024, 2 * sm_count());
    k_sum_part<<<nb, 256, 0, s>>>(n, v, cpart); FVS_COUNT_LAUNCH();
    k_mean_final<<<1, 1024, 0, s>>>(nb, cpart, (double)n, cpart.p + 1024); FVS_COUNT_LAUNCH();
    k_sub_scalar<<<stride_grid(n, 256), 256, 0, s>>>(n, cpart.p + 1024, v); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    return FVS_OK;
  }
  FVS_TRY(csum.zero(s));
  k_comp_sum<<<stride_grid(n, 256), 256, 0, s>>>(n, fine_lab, v, csum); FVS_COUNT_LAUNCH();
  k_comp_sub<<<stride_grid(n, 256), 256, 0, s>>>(n, fine_lab, csing, csum, ccnt, v); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

template <typename T>
fvs_status Amg::vcycle_t(cudaStream_t s, int l, const T* b, T* y) {
  AmgLevel* L = lv[l].get();
  const Ell& A = *L->A;
  const int64_t n = L->n;
  if (n == 0) return FVS_OK;
  if (l + 1 == (int)lv.size()) {
    k_coarse_solve<T><<<(nc + 7) / 8, 256, 0, s>>>(nc, Ainv.p, b, y); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    return FVS_OK;
  }
  AmgLevel* C = lv[l + 1].get();
  const bool f32 = sizeof(T) == 4;
  const T* val = f32 ? (const T*)L->valf.p : (const T*)A.val.p;
  const T* dinv = f32 ? (const T*)L->dinvf.p : (const T*)L->dinv.p;
  T* xa = f32 ? (T*)L->xf.p : (T*)L->x.p;
  T* xb = f32 ? (T*)L->tf.p : (T*)L->t.p;
  T* r = f32 ? (T*)L->rf.p : (T*)L->r.p;
  T* cb = f32 ? (T*)C->bf.p : (T*)C->b.p;
  T* cy = f32 ? (T*)C->yf.p : (T*)C->y.p;
  const double vb = (double)sizeof(T);
  const double jac_bytes = (double)n * ((4.0 + vb) * A.w + 4.0 * vb);
  const int g = stride_grid(n, 256);
  {
    ProfScope ps(L->A, f32 ? "jacobi0_f32" : "jacobi0", 3.0 * vb * (double)n, s);
    k_jac0<T><<<g, 256, 0, s>>>(n, (T)opt.omega, dinv, b, xa); FVS_COUNT_LAUNCH();
  }
  for (int k = 1; k < opt.npre; ++k) {
    ProfScope ps(L->A, f32 ? "jacobi_f32" : "jacobi", jac_bytes, s);
    k_jac<T><<<g, 256, 0, s>>>(n, A.w, A.col, val, (T)opt.omega, dinv, b, xa, xb); FVS_COUNT_LAUNCH();
    T* t = xa; xa = xb; xb = t;
  }
  {
    ProfScope ps(L->A, f32 ? "residual_f32" : "residual_vc", (double)n * ((4.0 + vb) * A.w + 3.0 * vb), s);
    k_resid<T><<<g, 256, 0, s>>>(n, A.w, A.col, val, xa, b, r); FVS_COUNT_LAUNCH();
  }
  k_restrict<T><<<stride_grid(C->n, 256), 256, 0, s>>>(C->n, L->mptr, L->midx, r, cb); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  FVS_TRY(vcycle_t<T>(s, l + 1, cb, cy));
  k_prolong<T><<<g, 256, 0, s>>>(n, L->agg, cy, (T)opt.coarse_scale, xa); FVS_COUNT_LAUNCH();
  for (int k = 0; k < opt.npost; ++k) {
    T* out = (k == opt.npost - 1) ? y : xb;
    ProfScope ps(L->A, f32 ? "jacobi_f32" : "jacobi", jac_bytes, s);
    k_jac<T><<<g, 256, 0, s>>>(n, A.w, A.col, val, (T)opt.omega, dinv, b, xa, out); FVS_COUNT_LAUNCH();
    xb = xa;
    xa = out;
  }
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

fvs_status Amg::apply(cudaStream_t s, const double* r, double* z) {
  if (!opt.fp32) return vcycle_t<double>(s, 0, r, z);
  // mixed precision: the V-cycle runs in FP32, the Krylov method around it in FP64
  AmgLevel* L = lv[0].get();
  const int64_t n = L->n;
  k_convert<double, float><<<stride_grid(n, 256), 256, 0, s>>>(n, r, L->bf.p); FVS_COUNT_LAUNCH();
  FVS_TRY(vcycle_t<float>(s, 0, L->bf.p, L->yf.p));
  k_convert<float, double><<<stride_grid(n, 256), 256, 0, s>>>(n, L->yf.p, z); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

// FP32 copies of the level operators and vectors (mixed precision)
fvs_status Amg::setup_fp32(cudaStream_t s) {
  for (auto& up : lv) {
    AmgLevel* L = up.get();
    const int64_t n = L->n;
    const int64_t nz = n * (int64_t)L->A->w;
    FVS_TRY(L->valf.alloc(nz + 1)); FVS_TRY(L->dinvf.alloc(n + 1));
    FVS_TRY(L->bf.alloc(n + 1)); FVS_TRY(L->xf.alloc(n + 1)); FVS_TRY(L->yf.alloc(n + 1)); FVS_TRY(L->rf.alloc(n + 1));
    FVS_TRY(L->tf.alloc(n + 1));
    if (n > 0) {
      k_convert<double, float><<<stride_grid(nz, 256), 256, 0, s>>>(nz, L->A->val.p, L->valf.p); FVS_COUNT_LAUNCH();
      k_convert<double, float><<<stride_grid(n, 256), 256, 0, s>>>(n, L->dinv.p, L->dinvf.p); FVS_COUNT_LAUNCH();
    }
  }
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

}  // namespace fvs
