// Aggregation AMG: setup (strength, parallel MIS aggregation, Galerkin
// coarse operators, pinned dense coarsest inverse, component labels) and the
// V-cycle (damped Jacobi, piecewise-constant restriction / prolongation).
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "amg.cuh"

namespace fvs {

#define GS(i, n) for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

static constexpr int GAL_CAP = 4096;   // entries gathered per coarse row (48 KB of shared memory)
static constexpr int GAL_SMALL = 256;  // rows up to this many entries: the many-warp kernel

// ---------------------------------------------------------------------------
// strength of connection: j is strong for i if -a_ij >= theta max_k(-a_ik)
// (or the same holds with i and j exchanged, to keep the graph symmetric)
// ---------------------------------------------------------------------------
__global__ void k_maxoff(int64_t n, int w, const int32_t* col, const double* val, double* mo, double* dinv,
                         const double* diag, const uint8_t* dirty = nullptr) {
  GS(i, n) {
    if (dirty && !dirty[i]) continue;
    double m = 0.0;
    for (int k = 0; k < w; ++k) {
      const int64_t e = (int64_t)k * n + i;
      if (col[e] != (int32_t)i) m = fmax(m, -val[e]);
    }
    mo[i] = m;
    dinv[i] = diag[i] != 0.0 ? 1.0 / diag[i] : 0.0;   // empty rows (refresh) stay untouched
  }
}

// strength masks: word q of row i (stored at [q*n + i]) flags slots
// 64q .. 64q + 63 of the row; slots beyond 64 * SMASK_WORDS are never strong
// (wider rows only occur on small coarse levels)
constexpr int SMASK_WORDS = 4;

__global__ void k_strong(int64_t n, int w, const int32_t* col, const double* val, const double* mo, double theta,
                         int absval, uint64_t* mask) {
  GS(i, n) {
    // judged from row i alone (the strength graph may be slightly
    // asymmetric; the independent-set rounds and the assignment only ever
    // look at a node's own mask, so that stays consistent)
    const int wk = w < 64 * SMASK_WORDS ? w : 64 * SMASK_WORDS;
    for (int q = 0; q < SMASK_WORDS; ++q) {
      uint64_t msk = 0;
      const int k1 = min(wk, 64 * (q + 1));
      for (int k = 64 * q; k < k1; ++k) {
        const int64_t e = (int64_t)k * n + i;
        const int32_t j = col[e];
        if (j == (int32_t)i) continue;
        const double a = absval ? fabs(val[e]) : -val[e];
        if (a > 0.0 && a >= theta * mo[i]) msk |= (1ULL << (k - 64 * q));
      }
      mask[(int64_t)q * n + i] = msk;
    }
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
      for (int q = 0; q < SMASK_WORDS && top; ++q) {
        uint64_t m = mask[(int64_t)q * n + i];
        while (m) {
          const int k = 64 * q + __ffsll((long long)m) - 1;
          m &= m - 1;
          const int32_t j = col[(int64_t)k * n + i];
          if (st[j] == 0 && beats(j, (int32_t)i)) { top = false; break; }
        }
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
      for (int q = 0; q < SMASK_WORDS && s == 0; ++q) {
        uint64_t m = mask[(int64_t)q * n + i];
        while (m) {
          const int k = 64 * q + __ffsll((long long)m) - 1;
          m &= m - 1;
          if (st2[col[(int64_t)k * n + i]] == 1) { s = 2; break; }
        }
      }
      if (s == 0) ++cnt;
    }
    st[i] = s;
  }
  if (cnt) atomicAdd(undecided, cnt);
}
__global__ void k_count_isolated(int64_t n, const uint64_t* mask, int* out) {
  int c = 0;
  GS(i, n) {
    uint64_t any = 0;
    for (int q = 0; q < SMASK_WORDS; ++q) any |= mask[(int64_t)q * n + i];
    c += any == 0 ? 1 : 0;
  }
  if (c) atomicAdd(out, c);
}
// fine rows without a nonzero coupling (identity rows of cells that carry no
// pressure: frozen or not yet melted cells of the numbering) take no part in
// the aggregation: state 3, no aggregate, no null-space label
__global__ void k_mark_decoupled(int64_t n, int w, const int32_t* col, const double* val, uint8_t* st) {
  GS(i, n) {
    bool any = false;
    for (int k = 0; k < w && !any; ++k) {
      const int64_t e = (int64_t)k * n + i;
      any = col[e] != (int32_t)i && val[e] != 0.0;
    }
    if (!any) st[i] = 3;
  }
}
__global__ void k_is_root(int64_t n, const uint8_t* st, int32_t* flag) {
  GS(i, n) flag[i] = st[i] == 1 ? 1 : 0;
}
// every non-root joins its strongest root neighbour (ties: lower index)
__global__ void k_assign(int64_t n, int w, const int32_t* col, const double* val, const uint64_t* mask,
                         const uint8_t* st, const int32_t* rid, int32_t* agg, int* err, int lenient = 0) {
  GS(i, n) {
    if (st[i] == 1) { agg[i] = rid[i]; continue; }
    if (st[i] == 3) { agg[i] = -1; continue; }
    double best = -1e300;
    int32_t bj = -1;
    for (int q = 0; q < SMASK_WORDS; ++q) {
      uint64_t m = mask[(int64_t)q * n + i];
      while (m) {
        const int k = 64 * q + __ffsll((long long)m) - 1;
        m &= m - 1;
        const int64_t e = (int64_t)k * n + i;
        const int32_t j = col[e];
        if (st[j] != 1) continue;
        const double a = -val[e];
        if (a > best || (a == best && j < bj)) { best = a; bj = j; }
      }
    }
    if (bj < 0) {
      if (lenient) agg[i] = -1;          // distance-2 set: joins a neighbour's aggregate next
      else { atomicOr(err, 1); agg[i] = 0; }
    } else {
      agg[i] = rid[bj];
    }
  }
}

// ---------------------------------------------------------------------------
// Distance-2 independent set (used where the distance-1 set coarsens a level
// by less than the accepted ratio: chains and star-like couplings of small
// coarse levels).  A node becomes a root when its key is the largest among
// the undecided nodes within two strong hops; nodes within two hops of a root
// drop out.  Keys: hash of the index, then the index (0 = not undecided).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t mis2_key(int64_t i, uint8_t st) {
  return st == 0 ? (((uint64_t)hash32((uint32_t)i) << 32) | (uint64_t)(i + 1)) : 0ULL;
}
// t1[i] = largest undecided key among i and its strong neighbours
__global__ void k_mis2_max1(int64_t n, const int32_t* col, const uint64_t* mask, const uint8_t* st, uint64_t* t1) {
  GS(i, n) {
    uint64_t best = mis2_key(i, st[i]);
    for (int q = 0; q < SMASK_WORDS; ++q) {
      uint64_t m = mask[(int64_t)q * n + i];
      while (m) {
        const int k = 64 * q + __ffsll((long long)m) - 1;
        m &= m - 1;
        const int32_t j = col[(int64_t)k * n + i];
        const uint64_t kj = mis2_key(j, st[j]);
        best = kj > best ? kj : best;
      }
    }
    t1[i] = best;
  }
}
// second hop; an undecided node holding the largest key within two hops is a root
__global__ void k_mis2_select(int64_t n, const int32_t* col, const uint64_t* mask, const uint8_t* st,
                              const uint64_t* t1, uint8_t* st2) {
  GS(i, n) {
    uint8_t s = st[i];
    if (s == 0) {
      uint64_t best = t1[i];
      for (int q = 0; q < SMASK_WORDS; ++q) {
        uint64_t m = mask[(int64_t)q * n + i];
        while (m) {
          const int k = 64 * q + __ffsll((long long)m) - 1;
          m &= m - 1;
          const uint64_t tj = t1[col[(int64_t)k * n + i]];
          best = tj > best ? tj : best;
        }
      }
      if (best == mis2_key(i, 0)) s = 1;
    }
    st2[i] = s;
  }
}
// r1[i] = 1 if i or a strong neighbour is a root
__global__ void k_mis2_near(int64_t n, const int32_t* col, const uint64_t* mask, const uint8_t* st2, uint8_t* r1) {
  GS(i, n) {
    uint8_t r = st2[i] == 1 ? 1 : 0;
    for (int q = 0; q < SMASK_WORDS && !r; ++q) {
      uint64_t m = mask[(int64_t)q * n + i];
      while (m) {
        const int k = 64 * q + __ffsll((long long)m) - 1;
        m &= m - 1;
        if (st2[col[(int64_t)k * n + i]] == 1) { r = 1; break; }
      }
    }
    r1[i] = r;
  }
}
// undecided nodes with a root within two hops drop out
__global__ void k_mis2_remove(int64_t n, const int32_t* col, const uint64_t* mask, const uint8_t* st2,
                              const uint8_t* r1, uint8_t* st, int* undecided) {
  int cnt = 0;
  GS(i, n) {
    uint8_t s = st2[i];
    if (s == 0) {
      bool near = r1[i] != 0;
      for (int q = 0; q < SMASK_WORDS && !near; ++q) {
        uint64_t m = mask[(int64_t)q * n + i];
        while (m) {
          const int k = 64 * q + __ffsll((long long)m) - 1;
          m &= m - 1;
          if (r1[col[(int64_t)k * n + i]]) { near = true; break; }
        }
      }
      if (near) s = 2;
      else ++cnt;
    }
    st[i] = s;
  }
  if (cnt) atomicAdd(undecided, cnt);
}
// nodes two hops from their root join the aggregate of their strongest
// assigned strong neighbour (reads one snapshot, writes another)
__global__ void k_assign_near(int64_t n, const int32_t* col, const double* val, const uint64_t* mask,
                              const uint8_t* st, const int32_t* agg_in, int32_t* agg_out, int* left) {
  int cnt = 0;
  GS(i, n) {
    int32_t a = agg_in[i];
    if (a < 0 && st[i] != 3) {
      double best = -1e300;
      int32_t bj = -1;
      for (int q = 0; q < SMASK_WORDS; ++q) {
        uint64_t m = mask[(int64_t)q * n + i];
        while (m) {
          const int k = 64 * q + __ffsll((long long)m) - 1;
          m &= m - 1;
          const int64_t e = (int64_t)k * n + i;
          const int32_t j = col[e];
          if (agg_in[j] < 0) continue;
          const double v = -val[e];
          if (v > best || (v == best && j < bj)) { best = v; bj = j; }
        }
      }
      if (bj >= 0) a = agg_in[bj];
      else ++cnt;
    }
    agg_out[i] = a;
  }
  if (cnt) atomicAdd(left, cnt);
}

// rows with agg < 0 (left out by a refresh) belong to no aggregate
__global__ void k_count_members(int64_t n, const int32_t* agg, int32_t* cnt) {
  GS(i, n) if (agg[i] >= 0) atomicAdd(&cnt[agg[i]], 1);
}
__global__ void k_fill_members(int64_t n, const int32_t* agg, const int32_t* ptr, int32_t* cur, int32_t* idx) {
  GS(i, n) {
    const int32_t a = agg[i];
    if (a >= 0) idx[ptr[a] + atomicAdd(&cur[a], 1)] = (int32_t)i;
  }
}
// refresh: a row carrying pressure without an aggregate (its cell melted
// again, or first melted in a margin row of the numbering) joins the
// aggregate of its most strongly coupled neighbour that has one; reads one
// snapshot, writes another
__global__ void k_join_agg(int64_t n, int w, const int32_t* col, const double* val, const int32_t* act,
                           const uint8_t* ppe, const int32_t* agg_in, int32_t* agg_out) {
  GS(i, n) {
    int32_t a = agg_in[i];
    if (a < 0 && ppe[act[i]]) {
      double best = 0.0;
      for (int k = 0; k < w; ++k) {
        const int64_t e = (int64_t)k * n + i;
        const int32_t j = col[e];
        if (j == (int32_t)i || val[e] == 0.0 || agg_in[j] < 0) continue;
        const double v = fabs(val[e]);
        if (v > best) { best = v; a = agg_in[j]; }
      }
    }
    agg_out[i] = a;
  }
}
// refresh: rows whose cells carry no pressure leave their aggregates; a row
// that carries pressure and found no aggregate stays outside every aggregate
// (smoothed on the fine level only, its couplings lumped into the coarse
// diagonals)
__global__ void k_mask_agg(int64_t n, const int32_t* act, const uint8_t* ppe, int32_t* agg) {
  GS(i, n) if (!ppe[act[i]]) agg[i] = -1;
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
// per coarse row: gather (agg[col], val) of all member rows into shared
// memory, bitonic-sort by key, reduce equal keys in a fixed order
// (deterministic).  The count pass gives the row lengths, the fill pass
// writes the ELL rows.  Rows of at most GAL_SMALL gathered entries take one
// warp each (many warps per block); larger rows take a whole block.  With a
// 'dirty' mask only the marked coarse rows are recomputed (refresh).
// ---------------------------------------------------------------------------
// a coupling to a row without an aggregate (a cell that carries pressure
// again since the aggregation was formed) lumps into the coarse diagonal, so
// coarse row sums -- and the constant null vectors -- are kept
__device__ __forceinline__ int32_t gal_key(int32_t a, int64_t I) { return a >= 0 ? a : (int32_t)I; }
// gather and zero-pad to P (a power of two), then sort; T threads, SYNC()
// the barrier among them
#define GAL_GATHER_SORT(T, t, SYNC)                                                \
  for (int e = (t); e < P; e += (T)) {                                            \
    if (e < total) {                                                              \
      const int m = e / w, k = e - m * w;                                         \
      const int32_t i = midx[lo + m];                                             \
      const int64_t ei = (int64_t)k * n + i;                                      \
      const double a = val[ei];                                                   \
      key[e] = a != 0.0 ? gal_key(agg[col[ei]], I) : INT_MAX;                     \
      v[e] = a;                                                                   \
    } else {                                                                      \
      key[e] = INT_MAX;                                                           \
      v[e] = 0.0;                                                                 \
    }                                                                             \
  }                                                                               \
  SYNC;                                                                           \
  GAL_SORT(T, t, SYNC)

// bitonic sort of key[0..P) (with v) by key; T threads, SYNC() the barrier
#define GAL_SORT(T, t, SYNC)                                                      \
  for (int size = 2; size <= P; size <<= 1) {                                     \
    for (int stride = size >> 1; stride > 0; stride >>= 1) {                      \
      for (int e = (t); e < P; e += (T)) {                                        \
        const int p = e ^ stride;                                                 \
        if (p > e) {                                                              \
          const bool up = (e & size) == 0;                                        \
          const int32_t ke = key[e], kp = key[p];                                 \
          if ((ke > kp) == up && ke != kp) {                                      \
            key[e] = kp; key[p] = ke;                                             \
            const double tv = v[e]; v[e] = v[p]; v[p] = tv;                       \
          }                                                                       \
        }                                                                         \
      }                                                                           \
      SYNC;                                                                       \
    }                                                                             \
  }

// one warp: segment heads of the sorted keys -> row I of the coarse ELL
template <bool FILL>
__device__ __forceinline__ void gal_emit(int lane, const int32_t* key, const double* v, int P, int64_t I, int64_t nc,
                                         int32_t* rowlen, int wc, int32_t* ccol, double* cval, double* cdiag,
                                         int* err) {
  if (FILL && lane == 0) cdiag[I] = 0.0;
  __syncwarp();
  int base = 0;
  for (int e0 = 0; e0 < P; e0 += 32) {
    const int e = e0 + lane;
    const bool head = key[e] != INT_MAX && (e == 0 || key[e - 1] != key[e]);
    const unsigned bal = __ballot_sync(0xffffffffu, head);
    if (FILL && head) {
      const int r = base + __popc(bal & ((1u << lane) - 1));
      double sum = 0.0;
      for (int q = e; q < P && key[q] == key[e]; ++q) sum += v[q];
      if (r < wc) {
        ccol[(int64_t)r * nc + I] = key[e];
        cval[(int64_t)r * nc + I] = sum;
      } else {
        atomicOr(err, 4);
      }
      if (key[e] == (int32_t)I) cdiag[I] = sum;
    }
    base += __popc(bal);
  }
  if (lane == 0 && rowlen) rowlen[I] = FILL ? min(base, wc) : base;
  if (FILL) {
    for (int r = base + lane; r < wc; r += 32) {
      ccol[(int64_t)r * nc + I] = (int32_t)I;
      cval[(int64_t)r * nc + I] = 0.0;
    }
  }
}

template <bool FILL, int WARPS>
__global__ void __launch_bounds__(32 * WARPS) k_galerkin(int64_t nc, int64_t n, int w, const int32_t* col,
                                                         const double* val, const int32_t* agg, const int32_t* mptr,
                                                         const int32_t* midx, int32_t* rowlen, int wc, int32_t* ccol,
                                                         double* cval, double* cdiag, int* err,
                                                         const uint8_t* dirty) {
  __shared__ int32_t key_s[WARPS * GAL_SMALL];
  __shared__ double v_s[WARPS * GAL_SMALL];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t* key = key_s + wid * GAL_SMALL;
  double* v = v_s + wid * GAL_SMALL;
  for (int64_t I = (int64_t)blockIdx.x * WARPS + wid; I < nc; I += (int64_t)gridDim.x * WARPS) {
    if (dirty && !dirty[I]) continue;
    const int32_t lo = mptr[I], hi = mptr[I + 1];
    const int total = (hi - lo) * w;
    if (total > GAL_SMALL) continue;     // the block-per-row kernel takes it
    int P = 32;
    while (P < total) P <<= 1;
    GAL_GATHER_SORT(32, lane, __syncwarp())
    gal_emit<FILL>(lane, key, v, P, I, nc, rowlen, wc, ccol, cval, cdiag, err);
    __syncwarp();
  }
}

template <bool FILL>
__global__ void __launch_bounds__(256) k_galerkin_big(int64_t nc, int64_t n, int w, const int32_t* col,
                                                      const double* val, const int32_t* agg, const int32_t* mptr,
                                                      const int32_t* midx, int32_t* rowlen, int wc, int32_t* ccol,
                                                      double* cval, double* cdiag, int* err, const uint8_t* dirty) {
  __shared__ int32_t key[GAL_CAP];
  __shared__ double v[GAL_CAP];
  for (int64_t I = blockIdx.x; I < nc; I += gridDim.x) {
    if (dirty && !dirty[I]) continue;
    const int32_t lo = mptr[I], hi = mptr[I + 1];
    const int total = (hi - lo) * w;
    if (total <= GAL_SMALL || total > GAL_CAP) continue;   // the warp / wide kernels take these
    int P = 32;
    while (P < total) P <<= 1;
    GAL_GATHER_SORT(256, (int)threadIdx.x, __syncthreads())
    if (threadIdx.x < 32) gal_emit<FILL>((int)threadIdx.x, key, v, P, I, nc, rowlen, wc, ccol, cval, cdiag, err);
    __syncthreads();
  }
}

// coarse rows whose members' padded rows exceed GAL_CAP entries (wide, short
// rows of small coarse levels): gather only the stored entries of each member
// row (rlen; null: every slot), members in order
template <bool FILL>
__global__ void __launch_bounds__(256) k_galerkin_wide(int64_t nc, int64_t n, int w, const int32_t* col,
                                                       const double* val, const int32_t* rlen_in,
                                                       const int32_t* agg, const int32_t* mptr,
                                                       const int32_t* midx, int32_t* rowlen, int wc, int32_t* ccol,
                                                       double* cval, double* cdiag, int* err, const uint8_t* dirty) {
  __shared__ int32_t key[GAL_CAP];
  __shared__ double v[GAL_CAP];
  for (int64_t I = blockIdx.x; I < nc; I += gridDim.x) {
    if (dirty && !dirty[I]) continue;
    const int32_t lo = mptr[I], hi = mptr[I + 1];
    if ((hi - lo) * w <= GAL_CAP) continue;
    int total = 0;
    for (int32_t m = lo; m < hi; ++m) total += rlen_in ? rlen_in[midx[m]] : w;
    if (total > GAL_CAP) {
      if (threadIdx.x == 0) { atomicOr(err, 2); if (!FILL) rowlen[I] = 0; }
      continue;
    }
    int P = 32;
    while (P < total) P <<= 1;
    int base = 0;
    for (int32_t m = lo; m < hi; ++m) {
      const int32_t i = midx[m];
      const int len = rlen_in ? rlen_in[i] : w;
      for (int k = threadIdx.x; k < len; k += blockDim.x) {
        const int64_t ei = (int64_t)k * n + i;
        const double a = val[ei];
        key[base + k] = a != 0.0 ? gal_key(agg[col[ei]], I) : INT_MAX;
        v[base + k] = a;
      }
      base += len;
    }
    for (int e = total + threadIdx.x; e < P; e += blockDim.x) {
      key[e] = INT_MAX;
      v[e] = 0.0;
    }
    __syncthreads();
    GAL_SORT(256, (int)threadIdx.x, __syncthreads())
    if (threadIdx.x < 32) gal_emit<FILL>((int)threadIdx.x, key, v, P, I, nc, rowlen, wc, ccol, cval, cdiag, err);
    __syncthreads();
  }
}

__global__ void k_sum_i32(int64_t n, const int32_t* a, unsigned long long* out) {
  unsigned long long t = 0;
  GS(i, n) t += (unsigned long long)(a[i] > 0 ? a[i] : 0);
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0 && t) atomicAdd(out, t);
}

__global__ void k_max_int(int64_t n, const int32_t* a, int* out) {
  int m = 0;
  GS(i, n) m = max(m, (int)a[i]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// ---------------------------------------------------------------------------
// coarsest level: dense copy, connected parts, pins, Gauss-Jordan inverse.
// Larger coarsest levels (n > SMEM_COARSEST) are inverted in place in global
// memory by the whole GPU: one small pivot launch and one elimination launch
// per column (FP64 arithmetic is scarce on this part, so the O(n^3) work is
// spread over every SM instead of one block).
// ---------------------------------------------------------------------------
__global__ void k_dense_fill(int n, int w, const int32_t* col, const double* val, double* M) {
  GS(i, n) {
    for (int k = 0; k < w; ++k) M[(int64_t)i * n + col[(int64_t)k * n + i]] += val[(int64_t)k * n + i];
  }
}
// Connected parts of the symmetric pattern of M: the block builds a bit
// matrix of the pattern and the row sums in shared memory, then one thread
// runs a breadth-first search over 32-bit words.  Each singular part (zero
// row sums) gets its first (lowest) row pinned.  'order' lists the rows
// grouped by part, parts in order of discovery.
static constexpr int DENSE_PARTS_MAX = 1024;
static size_t dense_parts_smem(int n) {
  const size_t nw = (size_t)(n + 31) / 32;
  return 2 * (size_t)n * sizeof(double) + ((size_t)n * nw + nw + (size_t)n) * sizeof(uint32_t);
}
__global__ void __launch_bounds__(1024) k_dense_parts(int n, double* M, int32_t* lab, uint8_t* sing, int32_t* order,
                                                      int* ncomp_out) {
  extern __shared__ double psm[];
  const int nw = (n + 31) / 32;
  double* rs = psm;                                   // [n] row sums
  double* dg = rs + n;                                // [n] |diagonal|
  uint32_t* adj = (uint32_t*)(dg + n);                // [n][nw]
  uint32_t* vis = adj + (size_t)n * nw;               // [nw]
  int* queue = (int*)(vis + nw);                      // [n]
  for (int e = threadIdx.x; e < n * nw; e += blockDim.x) adj[e] = 0u;
  for (int e = threadIdx.x; e < nw; e += blockDim.x) vis[e] = 0u;
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e - i * n;
    if (M[e] != 0.0) {
      atomicOr(&adj[i * nw + (j >> 5)], 1u << (j & 31));
      atomicOr(&adj[j * nw + (i >> 5)], 1u << (i & 31));
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double a = 0.0;
    for (int j = 0; j < n; ++j) a += M[(int64_t)i * n + j];
    rs[i] = a;
    dg[i] = fabs(M[(int64_t)i * n + i]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int nc = 0, qt = 0;
    for (int s0 = 0; s0 < n; ++s0) {
      if ((vis[s0 >> 5] >> (s0 & 31)) & 1u) continue;
      const int start = qt;
      int qh = qt;
      queue[qt++] = s0;
      vis[s0 >> 5] |= 1u << (s0 & 31);
      while (qh < qt) {
        const int i = queue[qh++];
        lab[i] = nc;
        for (int w = 0; w < nw; ++w) {
          uint32_t c = adj[i * nw + w] & ~vis[w];
          vis[w] |= c;
          while (c) {
            const int b = __ffs(c) - 1;
            c &= c - 1u;
            queue[qt++] = w * 32 + b;
          }
        }
      }
      double r = 0.0, sc = 0.0;
      for (int q = start; q < qt; ++q) {
        r += rs[queue[q]];
        sc += dg[queue[q]];
      }
      const bool sg = fabs(r) <= 1e-9 * sc;
      sing[nc] = sg ? 1 : 0;
      if (sg)   // pin the first row of the part: p = 0 there
        for (int j = 0; j < n; ++j) M[(int64_t)s0 * n + j] = (j == s0) ? 1.0 : 0.0;
      ++nc;
    }
    *ncomp_out = nc;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < n; q += blockDim.x) order[q] = queue[q];
}
// column k: partial pivot (largest |M[i][k]|, i >= k, lowest index on ties),
// row swap, scaling of the pivot row, elimination factors
__global__ void __launch_bounds__(256) k_gj_pivot(int n, int k, double* M, double* fac, int32_t* perm, int* err) {
  __shared__ double bv[256];
  __shared__ int bi[256];
  if (*err) return;
  double best = -1.0;
  int arg = n;
  for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
    const double a = fabs(M[(int64_t)i * n + k]);
    if (a > best) { best = a; arg = i; }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = arg;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double b2 = bv[threadIdx.x + o];
      const int i2 = bi[threadIdx.x + o];
      if (b2 > bv[threadIdx.x] || (b2 == bv[threadIdx.x] && i2 < bi[threadIdx.x])) {
        bv[threadIdx.x] = b2;
        bi[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  const int p = bi[0];
  if (!(bv[0] > 1e-300)) {
    if (threadIdx.x == 0) atomicOr(err, 8);
    return;
  }
  if (threadIdx.x == 0) perm[k] = p;
  if (p != k)
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const double t = M[(int64_t)k * n + j];
      M[(int64_t)k * n + j] = M[(int64_t)p * n + j];
      M[(int64_t)p * n + j] = t;
    }
  __syncthreads();
  const double inv = 1.0 / M[(int64_t)k * n + k];
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (i == k) {
      fac[i] = 0.0;
    } else {
      fac[i] = M[(int64_t)i * n + k];
      M[(int64_t)i * n + k] = 0.0;
    }
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    M[(int64_t)k * n + j] = (j == k ? 1.0 : M[(int64_t)k * n + j]) * inv;
}
// rows i != k: M[i][:] -= fac[i] * M[k][:]  (one block per row)
__global__ void __launch_bounds__(128) k_gj_elim(int n, int k, double* M, const double* fac, const int* err) {
  if (*err) return;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const double f = fac[i];
    if (i == k || f == 0.0) continue;
    double* Mi = M + (int64_t)i * n;
    const double* Mk = M + (int64_t)k * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) Mi[j] -= f * Mk[j];
  }
}
// undo the row swaps as column swaps, last first (one thread per row)
__global__ void k_gj_unswap(int n, double* M, const int32_t* perm, const int* err) {
  if (*err) return;
  GS(i, n) {
    double* Mi = M + (int64_t)i * n;
    for (int k = n - 1; k >= 0; --k) {
      const int p = perm[k];
      if (p != k) { const double t = Mi[k]; Mi[k] = Mi[p]; Mi[p] = t; }
    }
  }
}
// M <- P M (LEFT) or M P (!LEFT), P v = v - (mean of v on each singular part)
template <bool LEFT>
__global__ void k_dense_fold(int n, double* M, const int32_t* lab, const uint8_t* sing, const int32_t* order,
                             const int* ncomp, const int* err) {
  if (*err) return;
  const int ncs = *ncomp;
  GS(t, n) {
    int pos = 0;
    for (int c = 0; c < ncs; ++c) {
      int cnt = 0;
      double sum = 0.0;
      for (int q = pos; q < n && lab[order[q]] == c; ++q, ++cnt)
        sum += LEFT ? M[(int64_t)order[q] * n + t] : M[(int64_t)t * n + order[q]];
      if (sing[c]) {
        const double m = sum / (double)cnt;
        for (int q = pos; q < pos + cnt; ++q) {
          if (LEFT) M[(int64_t)order[q] * n + t] -= m;
          else M[(int64_t)t * n + order[q]] -= m;
        }
      }
      pos += cnt;
    }
  }
}

// Small coarsest levels (n <= SMEM_COARSEST): the same pinned inverse, but
// in place in shared memory (one block), which is an order of magnitude
// faster than the global-memory version above.
static constexpr int SMEM_COARSEST = 160;

__global__ void __launch_bounds__(1024) k_coarsest_smem(int n, int w, const int32_t* col, const double* val,
                                                        double* Ainv, int32_t* lab, uint8_t* sing,
                                                        int* ncomp_out, int* err, int vs) {
  // one block per sample s = blockIdx.x; values and outputs of sample s sit
  // at stride vs (vs = 1, one block: a single system)
  const int smp = blockIdx.x;
  extern __shared__ double smem[];
  double* M = smem;                          // [n*n] in-place inverse
  double* fac = M + n * n;                   // [n]
  int* perm = (int*)(fac + n);               // [n] row swaps
  int* lb = perm + n;                        // [n] labels
  int* order = lb + n;                       // [n] rows grouped by part
  __shared__ int piv, ncs;
  __shared__ double pval;
  __shared__ uint8_t sg[SMEM_COARSEST];
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) M[e] = 0.0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    for (int k = 0; k < w; ++k) M[i * n + col[(int64_t)k * n + i]] += val[((int64_t)k * n + i) * vs + smp];
  __syncthreads();
  // connected parts of the symmetric pattern: every row starts with its own
  // index as label and takes the smallest label among the rows it couples
  // to, one warp per row, until no label changes (at most n rounds)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int i = threadIdx.x; i < n; i += blockDim.x) lb[i] = i;
  __syncthreads();
  for (int round = 0; round < n; ++round) {
    if (threadIdx.x == 0) ncs = 0;
    __syncthreads();
    for (int i = wid; i < n; i += nwarp) {
      int m = lb[i];
      for (int j = lane; j < n; j += 32)
        if (M[i * n + j] != 0.0 || M[j * n + i] != 0.0) m = min(m, lb[j]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0 && m < lb[i]) { lb[i] = m; ncs = 1; }
    }
    __syncthreads();
    const int changed = ncs;
    __syncthreads();
    if (!changed) break;
  }
  // row sums and diagonals for the singular test
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double rs = 0.0;
    for (int j = 0; j < n; ++j) rs += M[i * n + j];
    fac[i] = rs;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // parts numbered by their smallest row; a singular part (zero row sums)
    // pins its first row
    int nc = 0;
    for (int i = 0; i < n; ++i) {
      if (lb[i] == i) perm[i] = nc++;
    }
    for (int i = 0; i < n; ++i) lb[i] = perm[lb[i]];
    for (int c = 0; c < nc; ++c) {
      double rs = 0.0, sc = 0.0;
      int first = -1;
      for (int i = 0; i < n; ++i) {
        if (lb[i] != c) continue;
        if (first < 0) first = i;
        rs += fac[i];
        sc += fabs(M[i * n + i]);
      }
      const bool sgl = fabs(rs) <= 1e-9 * sc;
      sg[c] = sgl ? 1 : 0;
      if (sgl) {
        for (int j = 0; j < n; ++j) M[first * n + j] = 0.0;
        M[first * n + first] = 1.0;
      }
    }
    int pos = 0;
    for (int c = 0; c < nc; ++c)
      for (int i = 0; i < n; ++i)
        if (lb[i] == c) order[pos++] = i;
    ncs = nc;
    ncomp_out[smp] = nc;
  }
  __syncthreads();
  // in-place Gauss-Jordan with partial (row) pivoting; the pivot search is
  // one warp's, the update a 32 x 32 tiling of the matrix
  for (int k = 0; k < n; ++k) {
    if (wid == 0) {
      int p = k;
      double best = -1.0;
      for (int i = k + lane; i < n; i += 32) {
        const double a = fabs(M[i * n + k]);
        if (a > best) { best = a; p = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, p, o);
        if (ob > best || (ob == best && op < p)) { best = ob; p = op; }
      }
      if (lane == 0) {
        piv = p;
        perm[k] = p;
        pval = best;
      }
    }
    __syncthreads();
    if (!(pval > 1e-300)) {
      if (threadIdx.x == 0) atomicOr(err, 8);
      return;
    }
    if (piv != k)
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double t = M[k * n + j];
        M[k * n + j] = M[piv * n + j];
        M[piv * n + j] = t;
      }
    __syncthreads();
    const double inv = 1.0 / M[k * n + k];
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) M[k * n + j] = (j == k ? 1.0 : M[k * n + j]) * inv;
    for (int i = threadIdx.x; i < n; i += blockDim.x) fac[i] = (i == k) ? 0.0 : M[i * n + k];
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      if (i != k) M[i * n + k] = 0.0;
    __syncthreads();
    for (int i = wid; i < n; i += nwarp) {
      if (i == k) continue;
      const double f = fac[i];
      for (int j = lane; j < n; j += 32) M[i * n + j] -= f * M[k * n + j];
    }
    __syncthreads();
  }
  // undo the row swaps as column swaps, last first
  for (int k = n - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k)
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double t = M[i * n + k];
        M[i * n + k] = M[i * n + p];
        M[i * n + p] = t;
      }
    __syncthreads();
  }
  // fold the projections onto zero-mean parts: M <- P M P
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    int pos = 0;
    for (int c = 0; c < ncs; ++c) {
      int cnt = 0;
      double sum = 0.0;
      for (int q = pos; q < n && lb[order[q]] == c; ++q, ++cnt) sum += M[order[q] * n + j];
      if (sg[c]) {
        const double m = sum / (double)cnt;
        for (int q = pos; q < pos + cnt; ++q) M[order[q] * n + j] -= m;
      }
      pos += cnt;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int pos = 0;
    for (int c = 0; c < ncs; ++c) {
      int cnt = 0;
      double sum = 0.0;
      for (int q = pos; q < n && lb[order[q]] == c; ++q, ++cnt) sum += M[i * n + order[q]];
      if (sg[c]) {
        const double m = sum / (double)cnt;
        for (int q = pos; q < pos + cnt; ++q) M[i * n + order[q]] -= m;
      }
      pos += cnt;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) Ainv[(int64_t)e * vs + smp] = M[e];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    lab[(int64_t)i * vs + smp] = lb[i];
  }
  for (int c = threadIdx.x; c < ncs; c += blockDim.x) sing[(int64_t)c * vs + smp] = sg[c];
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
// Fine level: (A x)_i over every slot of the row (one thread per row; the
// coarse levels have their own kernels below)
template <typename T>
__device__ __forceinline__ T fine_row(int64_t n, int w, const int32_t* __restrict__ col, const T* __restrict__ val,
                                      const T* __restrict__ x, int64_t i) {
  return ell_row(n, w, col, val, x, i, (T)0);
}

// y = x + omega D^-1 (b - A x)
template <typename T>
__global__ void k_jac(int64_t n, int w, const int32_t* __restrict__ col, const T* __restrict__ val, T omega,
                      const T* __restrict__ dinv, const T* __restrict__ b, const T* __restrict__ x,
                      T* __restrict__ y) {
  GS(i, n) {
    const T acc = fine_row(n, w, col, val, x, i);
    y[i] = x[i] + omega * dinv[i] * (b[i] - acc);
  }
}
template <typename T>
__global__ void k_resid(int64_t n, int w, const int32_t* __restrict__ col, const T* __restrict__ val,
                        const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ r) {
  GS(i, n) {
    const T acc = fine_row(n, w, col, val, x, i);
    r[i] = b[i] - acc;
  }
}

// Coarse levels, G lanes per row (1, 2, 4 or 8 by the level's size and row
// length): lane q of a row sums the stored entries q, q + G,
// q + 2G, ... (four loads in flight), then the row's lanes add their partial
// sums by shuffles.  The 32 / G rows of a warp are consecutive, so with
// slot-major storage every slot's values and columns of those rows fill
// whole 32-byte sectors; several lanes per row idle fewer lanes on rows of
// uneven length and shorten the serial chain of gathers on wide rows.
template <typename T, int G, class X>
__device__ __forceinline__ T coarse_part(int64_t n, const int32_t* __restrict__ col, const T* __restrict__ val,
                                         const X& x, int len, int64_t i, int q) {
  T acc = 0;
  int k = q;
  for (; k + 3 * G < len; k += 4 * G) {
    const int64_t e0 = (int64_t)k * n + i, e1 = e0 + (int64_t)G * n, e2 = e1 + (int64_t)G * n,
                  e3 = e2 + (int64_t)G * n;
    const int32_t c0 = col[e0], c1 = col[e1], c2 = col[e2], c3 = col[e3];
    const T v0 = val[e0], v1 = val[e1], v2 = val[e2], v3 = val[e3];
    const T x0 = x(c0), x1 = x(c1), x2 = x(c2), x3 = x(c3);
    acc = fma(v0, x0, acc);
    acc = fma(v1, x1, acc);
    acc = fma(v2, x2, acc);
    acc = fma(v3, x3, acc);
  }
  for (; k < len; k += G) {
    const int64_t e = (int64_t)k * n + i;
    acc = fma(val[e], x(col[e]), acc);
  }
  return acc;
}
// x of a sweep, gathered by column
template <typename T>
struct XVec {
  const T* __restrict__ x;
  __device__ __forceinline__ T operator()(int32_t c) const { return x[c]; }
};
template <typename T, int G>
__device__ __forceinline__ T lanes_sum(T v) {
#pragma unroll
  for (int o = 1; o < G; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// r = b - A x on a coarse level (warp-uniform loop over groups of rows)
template <typename T, int G>
__global__ void k_resid_g(int64_t n, const int32_t* __restrict__ col, const T* __restrict__ val,
                          const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ r,
                          const int32_t* __restrict__ rlen) {
  const int lane = threadIdx.x & 31, q = lane & (G - 1);
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i0 = warp * (32 / G); i0 < n; i0 += nw * (32 / G)) {
    const int64_t i = i0 + lane / G;
    const bool ok = i < n;
    T acc = ok ? coarse_part<T, G>(n, col, val, XVec<T>{x}, rlen[i], i, q) : (T)0;
    acc = lanes_sum<T, G>(acc);
    if (ok && q == 0) r[i] = b[i] - acc;
  }
}
// y = x + omega D^-1 (b - A x) on a coarse level
template <typename T, int G>
__global__ void k_jac_g(int64_t n, const int32_t* __restrict__ col, const T* __restrict__ val, T omega,
                        const T* __restrict__ dinv, const T* __restrict__ b, const T* __restrict__ x,
                        T* __restrict__ y, const int32_t* __restrict__ rlen) {
  const int lane = threadIdx.x & 31, q = lane & (G - 1);
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i0 = warp * (32 / G); i0 < n; i0 += nw * (32 / G)) {
    const int64_t i = i0 + lane / G;
    const bool ok = i < n;
    T acc = ok ? coarse_part<T, G>(n, col, val, XVec<T>{x}, rlen[i], i, q) : (T)0;
    acc = lanes_sum<T, G>(acc);
    if (ok && q == 0) y[i] = x[i] + omega * dinv[i] * (b[i] - acc);
  }
}
// Chebyshev sweep (three-term recurrence of the Chebyshev polynomials in
// D^-1 A): y = x + beta (x - xp) + alpha D^-1 (b - A x), xp the iterate
// before x (nullptr: zero).  xp and y may be the same array (each row reads
// its own xp entry before writing y); x is gathered and must differ from y.
template <typename T>
__global__ void k_cheb(int64_t n, int w, const int32_t* __restrict__ col, const T* __restrict__ val, T alpha,
                       T beta, const T* __restrict__ dinv, const T* __restrict__ b, const T* __restrict__ x,
                       const T* xp, T* y) {
  GS(i, n) {
    const T acc = fine_row(n, w, col, val, x, i);
    const T xi = x[i];
    const T d = xp ? xi - xp[i] : xi;
    y[i] = xi + beta * d + alpha * dinv[i] * (b[i] - acc);
  }
}
template <typename T, int G>
__global__ void k_cheb_g(int64_t n, const int32_t* __restrict__ col, const T* __restrict__ val, T alpha, T beta,
                         const T* __restrict__ dinv, const T* __restrict__ b, const T* __restrict__ x, const T* xp,
                         T* y, const int32_t* __restrict__ rlen) {
  const int lane = threadIdx.x & 31, q = lane & (G - 1);
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i0 = warp * (32 / G); i0 < n; i0 += nw * (32 / G)) {
    const int64_t i = i0 + lane / G;
    const bool ok = i < n;
    T acc = ok ? coarse_part<T, G>(n, col, val, XVec<T>{x}, rlen[i], i, q) : (T)0;
    acc = lanes_sum<T, G>(acc);
    if (ok && q == 0) {
      const T xi = x[i];
      const T d = xp ? xi - xp[i] : xi;
      y[i] = xi + beta * d + alpha * dinv[i] * (b[i] - acc);
    }
  }
}
// Gershgorin bound of the spectrum of D^-1 A: every eigenvalue lies in a disc
// about 1 of radius sum_{j != i} |a_ij| / |a_ii|, so the largest real part is
// at most max_i |D^-1_ii| sum_j |a_ij|.  The stored slots of a row are summed
// (padding holds zeros); one atomic per warp, on the bit patterns, which order
// non-negative doubles as their values.
__global__ void k_gershgorin(int64_t n, int w, const double* __restrict__ val, const double* __restrict__ dinv,
                             const int32_t* __restrict__ rlen, unsigned long long* out) {
  double m = 0.0;
  GS(i, n) {
    const int len = rlen ? rlen[i] : w;
    double s = 0.0;
    for (int k = 0; k < len; ++k) s += fabs(val[(int64_t)k * n + i]);
    m = fmax(m, s * fabs(dinv[i]));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// lanes per row of a coarse level from its mean stored row length
// (FVS_AMG_LANES forces one count)
static int coarse_lanes(const AmgLevel& L) {
  static const int forced = [] {
    const char* e = getenv("FVS_AMG_LANES");
    const int v = e ? atoi(e) : 0;
    return (v == 1 || v == 2 || v == 4 || v == 8) ? v : 0;
  }();
  if (forced) return forced;
  // large levels are bandwidth-bound: two lanes keep whole sectors per slot
  // and most lanes busy; small levels are latency-bound: more lanes per row
  // shorten each lane's chain of dependent gathers (128^3 cavity, cold
  // launches: 905k-row level 37/43 us with two lanes against 47/69 us with
  // four; 6k-row level 12 us with two against 8 us with four)
  const double mean = L.n > 0 ? L.stored / (double)L.n : 0.0;
  if (mean < 6.0) return 1;
  return L.n >= 65536 ? 2 : (L.n >= 8192 ? 4 : 8);
}

template <typename T>
__global__ void k_restrict(int64_t nc, const int32_t* mptr, const int32_t* midx, const T* r, T* bc) {
  GS(I, nc) {
    T s = 0;
    for (int32_t m = mptr[I]; m < mptr[I + 1]; ++m) s += r[midx[m]];
    bc[I] = s;
  }
}
// restriction and the next level's first Jacobi iterate: bc = R r,
// xc = omega Dc^-1 bc
template <typename T>
__global__ void k_restrict_jac0(int64_t nc, const int32_t* mptr, const int32_t* midx, const T* r, T* bc, T omega,
                                const T* dinvc, T* xc) {
  GS(I, nc) {
    T s = 0;
    for (int32_t m = mptr[I]; m < mptr[I + 1]; ++m) s += r[midx[m]];
    bc[I] = s;
    xc[I] = omega * dinvc[I] * s;
  }
}
template <typename T>
__global__ void k_prolong(int64_t n, const int32_t* agg, const T* yc, T scale, T* x) {
  GS(i, n) {
    const int32_t a = agg[i];
    if (a >= 0) x[i] += scale * yc[a];
  }
}
template <typename A, typename B>
__global__ void k_convert(int64_t n, const A* a, B* b) {
  GS(i, n) b[i] = (B)a[i];
}

// label propagation down the hierarchy and per-component counts
__global__ void k_pull_labels(int64_t n, const int32_t* agg, const int32_t* lab_c, int32_t* lab) {
  GS(i, n) lab[i] = agg[i] >= 0 ? lab_c[agg[i]] : -1;
}
__global__ void k_copy_i32(int64_t n, const int32_t* a, int32_t* b) {
  GS(i, n) b[i] = a[i];
}
// rows with a negative label (cells frozen since the hierarchy was built)
// take no part in the projection
__global__ void k_comp_count(int64_t n, const int32_t* lab, double* cnt) {
  // lanes with the same label add once (one part usually holds every row)
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = b + threadIdx.x;
    const int32_t c = i < n ? lab[i] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    if (c >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&cnt[c], (double)__popc(peers));
  }
}
// per-part sums; a warp whose rows all lie in one part adds once
__global__ void k_comp_sum(int64_t n, const int32_t* lab, const double* v, double* s) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = b + threadIdx.x;
    const int32_t c = i < n ? lab[i] : -1;
    double x = c >= 0 ? v[i] : 0.0;
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    if (peers == 0xffffffffu) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) == 0 && c >= 0) atomicAdd(&s[c], x);
    } else if (c >= 0) {
      atomicAdd(&s[c], x);
    }
  }
}
__global__ void k_comp_sub(int64_t n, const int32_t* lab, const uint8_t* sing, const double* s, const double* cnt,
                           double* v) {
  GS(i, n) {
    const int32_t c = lab[i];
    if (c >= 0 && sing[c]) v[i] -= s[c] / cnt[c];
  }
}
// single component: deterministic mean via block partials (lab, when given,
// masks rows out; cnt_dev, when given, holds the row count)
// (want >= 0: only the rows labelled want)
__device__ __forceinline__ bool in_part(const int32_t* lab, int want, int64_t i) {
  return !lab || (want < 0 ? lab[i] >= 0 : lab[i] == want);
}
__global__ void k_sum_part(int64_t n, const double* v, const int32_t* lab, int want, double* part) {
  __shared__ double sh[32];
  double a = 0.0;
  GS(i, n) if (in_part(lab, want, i)) a += v[i];
  a = block_sum(a, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = a;
}
__global__ void k_mean_final(int nb, const double* part, double cnt, const double* cnt_dev, double* mean) {
  __shared__ double sh[32];
  double a = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) a += part[b];
  a = block_sum(a, sh);
  if (threadIdx.x == 0) {
    const double c = cnt_dev ? *cnt_dev : cnt;
    *mean = c > 0.0 ? a / c : 0.0;
  }
}
__global__ void k_sub_scalar(int64_t n, const double* mean, const int32_t* lab, int want, double* v) {
  const double m = *mean;
  GS(i, n) if (in_part(lab, want, i)) v[i] -= m;
}
// refresh: rows whose cells no longer carry pressure leave the null-space labels
__global__ void k_mask_labels(int64_t n, const int32_t* act, const uint8_t* ppe, int32_t* lab) {
  GS(i, n) if (!ppe[act[i]]) lab[i] = -1;
}
// refresh: a row carrying pressure without a label takes the label of the
// labelled rows it couples to; left[0] counts rows still without one,
// left[1] rows that took one; two different labels flag err (the row joins
// two parts)
__global__ void k_adopt_labels(int64_t n, int w, const int32_t* col, const double* val, const int32_t* act,
                               const uint8_t* ppe, const int32_t* lab_in, int32_t* lab_out, int* left, int* err) {
  int still = 0, took = 0;
  GS(i, n) {
    int32_t l = lab_in[i];
    if (l < 0 && ppe[act[i]]) {
      for (int k = 0; k < w; ++k) {
        const int64_t e = (int64_t)k * n + i;
        const int32_t j = col[e];
        if (j == (int32_t)i || val[e] == 0.0) continue;
        const int32_t lj = lab_in[j];
        if (lj < 0) continue;
        if (l < 0) l = lj;
        else if (l != lj) atomicOr(err, 16);
      }
      if (l < 0) ++still;
      else ++took;
    }
    lab_out[i] = l;
  }
  if (still) atomicAdd(left, still);
  if (took) atomicAdd(left + 1, took);
}
// a coupling between two labelled rows of different parts flags err
__global__ void k_label_conflicts(int64_t n, int w, const int32_t* col, const double* val, const int32_t* lab,
                                  int* err) {
  GS(i, n) {
    const int32_t l = lab[i];
    if (l < 0) continue;
    for (int k = 0; k < w; ++k) {
      const int64_t e = (int64_t)k * n + i;
      const int32_t j = col[e];
      if (j == (int32_t)i || val[e] == 0.0) continue;
      const int32_t lj = lab[j];
      if (lj >= 0 && lj != l) { atomicOr(err, 32); break; }
    }
  }
}
// 64-bit fingerprint of each ELL row (columns and value bits); with 'old'
// given, rows whose fingerprint changed are marked dirty
__device__ __forceinline__ uint64_t smix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
__global__ void k_row_hash(int64_t n, int w, const int32_t* col, const double* val, uint64_t* hash,
                           uint8_t* dirty, int compare) {
  GS(i, n) {
    uint64_t h = 0x6a09e667f3bcc909ULL;
    for (int k = 0; k < w; ++k) {
      const int64_t e = (int64_t)k * n + i;
      h = smix64(h ^ (uint64_t)(uint32_t)col[e]);
      h = smix64(h + (uint64_t)__double_as_longlong(val[e]));
    }
    if (compare) dirty[i] = hash[i] != h ? 1 : 0;
    hash[i] = h;
  }
}
// a coarse row is dirty when any of its member rows is
__global__ void k_dirty_up(int64_t n, const int32_t* agg, const uint8_t* dirty, uint8_t* dirty_c) {
  GS(i, n) if (dirty[i] && agg[i] >= 0) dirty_c[agg[i]] = 1;
}
// FP32 copies of the dirty rows
__global__ void k_convert_rows(int64_t n, int w, const double* val, const double* dinv, const uint8_t* dirty,
                               float* valf, float* dinvf) {
  GS(i, n) {
    if (!dirty[i]) continue;
    for (int k = 0; k < w; ++k) valf[(int64_t)k * n + i] = (float)val[(int64_t)k * n + i];
    dinvf[i] = (float)dinv[i];
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static fvs_status read_int(cudaStream_t s, const int* d, int* h) {
  FVS_CUDA(cudaMemcpyAsync(h, d, sizeof(int), cudaMemcpyDeviceToHost, s));
  FVS_CUDA(cudaStreamSynchronize(s));
  return FVS_OK;
}

// one Galerkin pass (count or fill) over all coarse rows (or the dirty ones)
static void galerkin_pass(cudaStream_t s, bool fill, int64_t nc, const Ell& A, const int32_t* rlen_in,
                          const int32_t* agg, const int32_t* mptr, const int32_t* midx, int32_t* rowlen, int wc,
                          int32_t* ccol, double* cval, double* cdiag, int* err, const uint8_t* dirty = nullptr) {
  if (nc <= 0) return;
  const int64_t n = A.n;
  const int gs = (int)std::min<int64_t>((nc + 3) / 4, (int64_t)sm_count() * 16);
  const int gb = (int)std::min<int64_t>(nc, (int64_t)sm_count() * 8);
  if (fill) {
    k_galerkin<true, 4><<<gs, 128, 0, s>>>(nc, n, A.w, A.col, A.val, agg, mptr, midx, rowlen, wc, ccol, cval, cdiag,
                                           err, dirty); FVS_COUNT_LAUNCH();
    k_galerkin_big<true><<<gb, 256, 0, s>>>(nc, n, A.w, A.col, A.val, agg, mptr, midx, rowlen, wc, ccol, cval,
                                            cdiag, err, dirty); FVS_COUNT_LAUNCH();
    k_galerkin_wide<true><<<gb, 256, 0, s>>>(nc, n, A.w, A.col, A.val, rlen_in, agg, mptr, midx, rowlen, wc, ccol,
                                             cval, cdiag, err, dirty); FVS_COUNT_LAUNCH();
  } else {
    k_galerkin<false, 4><<<gs, 128, 0, s>>>(nc, n, A.w, A.col, A.val, agg, mptr, midx, rowlen, wc, ccol, cval,
                                            cdiag, err, dirty); FVS_COUNT_LAUNCH();
    k_galerkin_big<false><<<gb, 256, 0, s>>>(nc, n, A.w, A.col, A.val, agg, mptr, midx, rowlen, wc, ccol, cval,
                                             cdiag, err, dirty); FVS_COUNT_LAUNCH();
    k_galerkin_wide<false><<<gb, 256, 0, s>>>(nc, n, A.w, A.col, A.val, rlen_in, agg, mptr, midx, rowlen, wc, ccol,
                                              cval, cdiag, err, dirty); FVS_COUNT_LAUNCH();
  }
}

static double env_num(const char* name, double dflt) {
  const char* v = getenv(name);
  return (v && *v) ? atof(v) : dflt;
}

// entries per level that one smoother or residual sweep reads: every slot on
// the fine level, the stored entries of each row on the coarse levels (for
// the algorithmic bytes of the kernel timing)
fvs_status Amg::count_stored(cudaStream_t s) {
  DBuf<unsigned long long> acc;
  FVS_TRY(acc.alloc(1));
  for (auto& up : lv) {
    AmgLevel* L = up.get();
    if (!L->rlen.n || L->n == 0) {
      L->stored = (double)L->n * (double)(L->A ? L->A->w : 0);
      continue;
    }
    FVS_CUDA(cudaMemsetAsync(acc.p, 0, sizeof(unsigned long long), s));
    k_sum_i32<<<stride_grid(L->n, 256), 256, 0, s>>>(L->n, L->rlen, acc); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    unsigned long long h = 0;
    FVS_CUDA(cudaMemcpyAsync(&h, acc.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    FVS_CUDA(cudaStreamSynchronize(s));
    L->stored = (double)h;
  }
  return FVS_OK;
}

fvs_status Amg::setup(cudaStream_t s, const Ell& A) {
  ready = false;
  masked = false;
  refreshes = 0;
  ++version;
  lv.clear();
  opt.theta = env_num("FVS_AMG_THETA", opt.theta);
  opt.omega = env_num("FVS_AMG_OMEGA", opt.omega);
  opt.coarse_scale = env_num("FVS_AMG_SCALE", opt.coarse_scale);
  opt.npre = (int)env_num("FVS_AMG_NPRE", opt.npre);
  opt.npost = (int)env_num("FVS_AMG_NPOST", opt.npost);
  opt.coarsest = (int)env_num("FVS_AMG_COARSEST", opt.coarsest);
  opt.mis2_ratio = env_num("FVS_AMG_MIS2_RATIO", opt.mis2_ratio);
  opt.mis2_from = (int)env_num("FVS_AMG_MIS2_FROM", opt.mis2_from);
  opt.smoother = (int)env_num("FVS_AMG_SMOOTHER", opt.smoother);
  opt.cheb_ratio = env_num("FVS_AMG_CHEB_RATIO", opt.cheb_ratio);
  if (opt.smoother != 1) opt.smoother = 0;
  if (!(opt.cheb_ratio > 1.0)) opt.cheb_ratio = 4.0;
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
  // phase timing for FVS_DEBUG (waits for the stream at each phase end)
  const bool dbg = getenv("FVS_DEBUG") != nullptr;
  double tph[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  auto t_last = std::chrono::steady_clock::now();
  auto tick = [&](int k) {
    if (!dbg) return;
    cudaStreamSynchronize(s);
    const auto now = std::chrono::steady_clock::now();
    tph[k] += std::chrono::duration<double, std::milli>(now - t_last).count();
    t_last = now;
  };
  for (int l = 0;; ++l) {
    tick(0);
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
    if (n <= opt.coarsest || l + 1 >= opt.max_levels) break;
    // strength and aggregation; if the strong graph coarsens too little (small
    // coarse levels of anisotropic problems), retry with every negative
    // coupling counted as strong, then with every nonzero coupling (coarse
    // Galerkin operators of skewed meshes carry many positive ones)
    DBuf<uint64_t> mask;
    DBuf<uint8_t> st, st2;
    DBuf<int32_t> flag, rid;
    FVS_TRY(mask.alloc((size_t)SMASK_WORDS * n)); FVS_TRY(st.alloc(n)); FVS_TRY(st2.alloc(n));
    FVS_TRY(flag.alloc(n + 1)); FVS_TRY(rid.alloc(n + 1));
    int nc = 0;
    bool mis2 = false;
    DBuf<uint64_t> t1;
    DBuf<uint8_t> r1;
    // attempts 0-2: distance-1 independent sets on ever wider strength
    // graphs; attempt 3, only where those would stall the coarsening: the
    // distance-2 set on the first graph
    const int first = l >= opt.mis2_from ? 3 : 0;
    for (int attempt = first; attempt < 4; ++attempt) {
      if (first == 0 && attempt == 3 && (double)nc <= opt.mis2_ratio * (double)n) break;   // keep the distance-1 result
      mis2 = attempt == 3;
      const double theta = (attempt == 0 || mis2) ? opt.theta : 0.0;
      const int absval = attempt == 2 ? 1 : 0;
      FVS_TRY(st.zero(s));
      if (l == 0) {
        k_mark_decoupled<<<stride_grid(n, 256), 256, 0, s>>>(n, cur->w, cur->col, cur->val, st);
        FVS_COUNT_LAUNCH();
      }
      k_strong<<<stride_grid(n, 256), 256, 0, s>>>(n, cur->w, cur->col, cur->val, mo, theta, absval, mask);
      FVS_COUNT_LAUNCH();
      FVS_LAUNCH_CHECK();
      tick(1);
      if (mis2) { FVS_TRY(t1.alloc(n)); FVS_TRY(r1.alloc(n)); }
      for (int round = 0;; round += 2) {
        // two independent-set rounds per check (rounds after completion change nothing)
        FVS_TRY(cnt.zero(s));
        for (int q = 0; q < 2; ++q) {
          int* cq = q == 1 ? cnt.p : cnt.p + 1;
          if (mis2) {
            k_mis2_max1<<<stride_grid(n, 256), 256, 0, s>>>(n, cur->col, mask, st, t1); FVS_COUNT_LAUNCH();
            k_mis2_select<<<stride_grid(n, 256), 256, 0, s>>>(n, cur->col, mask, st, t1, st2); FVS_COUNT_LAUNCH();
            k_mis2_near<<<stride_grid(n, 256), 256, 0, s>>>(n, cur->col, mask, st2, r1); FVS_COUNT_LAUNCH();
            k_mis2_remove<<<stride_grid(n, 256), 256, 0, s>>>(n, cur->col, mask, st2, r1, st, cq); FVS_COUNT_LAUNCH();
          } else {
            k_mis_select<<<stride_grid(n, 256), 256, 0, s>>>(n, cur->w, cur->col, mask, st, st2); FVS_COUNT_LAUNCH();
            k_mis_remove<<<stride_grid(n, 256), 256, 0, s>>>(n, cur->w, cur->col, mask, st2, st, cq);
            FVS_COUNT_LAUNCH();
          }
        }
        FVS_LAUNCH_CHECK();
        int und = 0;
        FVS_TRY(read_int(s, cnt, &und));
        if (und == 0) break;
        if (round >= 62) {
          set_error("AMG aggregation did not finish");
          return FVS_ERR_NOT_CONVERGED;
        }
      }
      FVS_TRY(flag.zero(s));
      k_is_root<<<stride_grid(n, 256), 256, 0, s>>>(n, st, flag); FVS_COUNT_LAUNCH();
      FVS_TRY(exclusive_scan(s, sw, n + 1, flag, rid));
      FVS_CUDA(cudaMemcpyAsync(&nc, rid.p + n, sizeof(int), cudaMemcpyDeviceToHost, s));
      FVS_CUDA(cudaStreamSynchronize(s));
      if ((double)nc <= 0.6 * (double)n) break;
    }
    if (dbg) {
      // rows without a strong coupling in the last attempt become singletons
      FVS_TRY(cnt.zero(s));
      k_count_isolated<<<stride_grid(n, 256), 256, 0, s>>>(n, mask, cnt); FVS_COUNT_LAUNCH();
      int iso = 0;
      FVS_TRY(read_int(s, cnt, &iso));
      fprintf(stderr, "[fvs amg] level %d: %lld rows (w%d) -> %d aggregates%s, %d rows without strong couplings\n",
              l, (long long)n, cur->w, nc, mis2 ? " (distance-2 set)" : "", iso);
    }
    if (nc <= 0 || nc >= n || (double)nc > 0.85 * (double)n) break;  // stagnation: L is the coarsest
    tick(2);
    FVS_TRY(L->agg.alloc(n));
    k_assign<<<stride_grid(n, 256), 256, 0, s>>>(n, cur->w, cur->col, cur->val, mask, st, rid, L->agg, err,
                                                 mis2 ? 1 : 0);
    FVS_COUNT_LAUNCH();
    if (mis2) {
      // nodes two hops from a root: up to three passes of joining an
      // assigned neighbour's aggregate; any left over is a setup failure
      DBuf<int32_t> agg2;
      FVS_TRY(agg2.alloc(n));
      int left = 0;
      for (int pass = 0; pass < 3; ++pass) {
        FVS_TRY(cnt.zero(s));
        k_assign_near<<<stride_grid(n, 256), 256, 0, s>>>(n, cur->col, cur->val, mask, st, L->agg, agg2, cnt);
        FVS_COUNT_LAUNCH();
        FVS_CUDA(cudaMemcpyAsync(L->agg.p, agg2.p, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        FVS_TRY(read_int(s, cnt, &left));
        if (left == 0) break;
      }
      if (left) {
        set_error("AMG aggregation left %d rows without an aggregate at level %d", left, l);
        return FVS_ERR_NOT_CONVERGED;
      }
    }
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
    std::unique_ptr<AmgLevel> C(new AmgLevel());
    DBuf<int32_t>& rowlen = C->rlen;   // kept: the V-cycle walks only the stored entries of each row
    FVS_TRY(rowlen.alloc(nc + 1));
    galerkin_pass(s, false, nc, *cur, L->rlen.p, L->agg, L->mptr, L->midx, rowlen, 0, nullptr, nullptr, nullptr,
                  err);
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
    tick(3);
    FVS_TRY(C->own.alloc(nc, wc));
    FVS_TRY(C->own.diag.zero(s));
    galerkin_pass(s, true, nc, *cur, L->rlen.p, L->agg, L->mptr, L->midx, rowlen, wc, C->own.col, C->own.val,
                  C->own.diag, err);
    FVS_LAUNCH_CHECK();
    C->A = &C->own;
    lv.push_back(std::move(C));
    tick(4);
  }
  {
    int e = 0;
    FVS_TRY(read_int(s, err, &e));
    if (e) {
      set_error("AMG setup failed (flags 0x%x)", e);
      return FVS_ERR_NOT_CONVERGED;
    }
  }
  tick(0);
  FVS_TRY(coarsest_setup(s));
  tick(5);
  if (opt.fp32) FVS_TRY(setup_fp32(s));
  if (lv[0]->n > 0) {
    const Ell& A0 = *lv[0]->A;
    FVS_TRY(rowhash.alloc(A0.n + 1));
    k_row_hash<<<stride_grid(A0.n, 256), 256, 0, s>>>(A0.n, A0.w, A0.col, A0.val, rowhash, nullptr, 0);
    FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
  }
  tick(6);
  if (dbg) {
    fprintf(stderr, "[fvs amg] levels %d:", (int)lv.size());
    for (auto& L : lv) fprintf(stderr, " %lld(w%d)", (long long)L->n, L->A->w);
    fprintf(stderr, " coarsest %d parts %d | ms: misc %.2f strength %.2f mis %.2f members %.2f galerkin %.2f "
            "coarsest %.2f fp32 %.2f\n", nc, ncomp, tph[0], tph[1], tph[2], tph[3], tph[4], tph[5], tph[6]);
  }
  FVS_TRY(count_stored(s));
  if (opt.smoother == 1) FVS_TRY(cheb_bounds(s));
  ready = true;
  return FVS_OK;
}

fvs_status Amg::cheb_bounds(cudaStream_t s) {
  const int nl = (int)lv.size();
  FVS_TRY(gbound.alloc(nl + 1));
  FVS_CUDA(cudaMemsetAsync(gbound.p, 0, sizeof(unsigned long long) * nl, s));
  for (int l = 0; l + 1 < nl; ++l) {   // the coarsest level is solved, not smoothed
    AmgLevel* L = lv[l].get();
    if (L->n == 0) continue;
    k_gershgorin<<<stride_grid(L->n, 256), 256, 0, s>>>(L->n, L->A->w, L->A->val, L->dinv,
                                                       L->rlen.n ? L->rlen.p : nullptr, gbound.p + l);
    FVS_COUNT_LAUNCH();
  }
  FVS_LAUNCH_CHECK();
  std::vector<unsigned long long> h(nl, 0ULL);
  FVS_CUDA(cudaMemcpyAsync(h.data(), gbound.p, sizeof(unsigned long long) * nl, cudaMemcpyDeviceToHost, s));
  FVS_CUDA(cudaStreamSynchronize(s));
  for (int l = 0; l < nl; ++l) {
    double v;
    memcpy(&v, &h[l], sizeof(v));
    lv[l]->cheb_b = std::isfinite(v) ? v : 0.0;
  }
  ++bound_epoch;
  return FVS_OK;
}

// the first sweep from a given iterate: weighted Jacobi, or the first step
// of the Chebyshev recurrence (weight 1 / theta, theta the interval's centre)
double Amg::first_weight(const AmgLevel& L) const {
  if (opt.smoother != 1 || !(L.cheb_b > 0.0)) return opt.omega;
  return 2.0 / (L.cheb_b * (1.0 + 1.0 / opt.cheb_ratio));
}

fvs_status Amg::coarsest_setup(cudaStream_t s) {
  AmgLevel* L = lv.back().get();
  const Ell& A = *L->A;
  nc = (int)A.n;
  if (nc > 4 * opt.coarsest || nc > DENSE_PARTS_MAX) {
    set_error("AMG coarsest level too large (%d rows)", nc);
    return FVS_ERR_NOT_CONVERGED;
  }
  DBuf<int>& err = c_err;
  DBuf<int>& ncd = c_ncd;
  FVS_TRY(Ainv.alloc((size_t)nc * nc + 1));
  FVS_TRY(clab.alloc(nc + 1));
  FVS_TRY(csing.alloc(nc + 1));
  FVS_TRY(err.alloc(1)); FVS_TRY(ncd.alloc(1));
  FVS_TRY(err.zero(s));
  if (nc > 0) {
    if (nc <= SMEM_COARSEST) {
      const size_t sh = (size_t)nc * nc * sizeof(double) + (size_t)nc * sizeof(double) + 3 * (size_t)nc * sizeof(int);
      // the attribute is per function, shared by every thread: set it once to
      // the largest size any launch uses (concurrent solvers launch smaller ones)
      static bool attr_set[64] = {false};
      int dev = 0;
      cudaGetDevice(&dev);
      if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        const size_t shmax = (size_t)SMEM_COARSEST * SMEM_COARSEST * sizeof(double) +
                             (size_t)SMEM_COARSEST * sizeof(double) + 3 * (size_t)SMEM_COARSEST * sizeof(int);
        FVS_CUDA(cudaFuncSetAttribute(k_coarsest_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmax));
        attr_set[dev] = true;
      }
      k_coarsest_smem<<<1, 1024, sh, s>>>(nc, A.w, A.col, A.val, Ainv, clab, csing, ncd, err, 1);
      FVS_COUNT_LAUNCH();
    } else {
      DBuf<double>& fac = gj_fac;
      DBuf<int32_t>& perm = gj_perm;
      DBuf<int32_t> order;
      FVS_TRY(fac.alloc(nc)); FVS_TRY(perm.alloc(nc)); FVS_TRY(order.alloc(nc));
      FVS_CUDA(cudaMemsetAsync(Ainv.p, 0, (size_t)nc * nc * sizeof(double), s));
      k_dense_fill<<<stride_grid(nc, 128), 128, 0, s>>>(nc, A.w, A.col, A.val, Ainv); FVS_COUNT_LAUNCH();
      static bool parts_attr[64] = {false};
      int dev = 0;
      cudaGetDevice(&dev);
      if (dev >= 0 && dev < 64 && !parts_attr[dev]) {
        FVS_CUDA(cudaFuncSetAttribute(k_dense_parts, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)dense_parts_smem(DENSE_PARTS_MAX)));
        parts_attr[dev] = true;
      }
      k_dense_parts<<<1, 1024, dense_parts_smem(nc), s>>>(nc, Ainv, clab, csing, order, ncd); FVS_COUNT_LAUNCH();
      const int eb = std::min(nc, 4 * sm_count());
      // 2 nc launches whose cost is mostly launch latency: capture them once
      // per level size and buffer set, then replay the graph
      const uint64_t key = ((uint64_t)nc << 40) ^ (uint64_t)(uintptr_t)Ainv.p ^ ((uint64_t)(uintptr_t)fac.p << 1) ^
                           ((uint64_t)(uintptr_t)perm.p << 2) ^ ((uint64_t)(uintptr_t)err.p << 3) ^ (uint64_t)eb;
      bool replayed = false;
      if (graphs_enabled() && s != nullptr) {
        if (!gj_exec || gj_key != key) {
          if (gj_exec) cudaGraphExecDestroy(gj_exec);
          gj_exec = nullptr;
          gj_key = 0;
          cudaGraph_t g = nullptr;
          if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            for (int k = 0; k < nc; ++k) {
              k_gj_pivot<<<1, 256, 0, s>>>(nc, k, Ainv, fac, perm, err);
              k_gj_elim<<<eb, 128, 0, s>>>(nc, k, Ainv, fac, err);
            }
            if (cudaStreamEndCapture(s, &g) == cudaSuccess && g) {
              if (cudaGraphInstantiate(&gj_exec, g, 0) != cudaSuccess) gj_exec = nullptr;
              cudaGraphDestroy(g);
            }
          }
          cudaGetLastError();   // a failed capture leaves the eager launches below
          if (gj_exec) gj_key = key;
        }
        if (gj_exec && cudaGraphLaunch(gj_exec, s) == cudaSuccess) {
          replayed = true;
          __atomic_add_fetch(&g_launches, 2ULL * (unsigned long long)nc, __ATOMIC_RELAXED);
        }
      }
      if (!replayed) {
        for (int k = 0; k < nc; ++k) {
          k_gj_pivot<<<1, 256, 0, s>>>(nc, k, Ainv, fac, perm, err); FVS_COUNT_LAUNCH();
          k_gj_elim<<<eb, 128, 0, s>>>(nc, k, Ainv, fac, err); FVS_COUNT_LAUNCH();
        }
      }
      k_gj_unswap<<<stride_grid(nc, 128), 128, 0, s>>>(nc, Ainv, perm, err); FVS_COUNT_LAUNCH();
      k_dense_fold<true><<<stride_grid(nc, 128), 128, 0, s>>>(nc, Ainv, clab, csing, order, ncd, err);
      FVS_COUNT_LAUNCH();
      k_dense_fold<false><<<stride_grid(nc, 128), 128, 0, s>>>(nc, Ainv, clab, csing, order, ncd, err);
      FVS_COUNT_LAUNCH();
    }
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
  masked = true;   // decoupled rows (label -1) stay out of the projection
  return FVS_OK;
}

fvs_status Amg::refresh(cudaStream_t s, const int32_t* act, const uint8_t* ppe) {
  if (!ready || lv.empty()) {
    set_error("AMG refresh without a hierarchy");
    return FVS_ERR_STATE;
  }
  const int64_t n0 = lv[0]->n;
  if (lv[0]->A->n != n0) {
    set_error("AMG refresh: operator has %lld rows, hierarchy %lld", (long long)lv[0]->A->n, (long long)n0);
    return FVS_ERR_STATE;
  }
  ready = false;
  ++version;
  const bool dbg = getenv("FVS_DEBUG") != nullptr;
  double tph[4] = {0, 0, 0, 0};
  auto t_last = std::chrono::steady_clock::now();
  auto tick = [&](int k) {
    if (!dbg) return;
    cudaStreamSynchronize(s);
    const auto now = std::chrono::steady_clock::now();
    tph[k] += std::chrono::duration<double, std::milli>(now - t_last).count();
    t_last = now;
  };
  DBuf<int> err, cnt2;
  DBuf<double> mo;
  FVS_TRY(err.alloc(1));
  FVS_TRY(err.zero(s));
  FVS_TRY(cnt2.alloc(2));
  FVS_TRY(mo.alloc(n0 + 1));
  for (auto& L : lv) {
    FVS_TRY(L->dirty.alloc(L->n + 1));
    FVS_TRY(L->dirty.zero(s));
  }
  // fine rows that changed since the hierarchy was last formed
  if (n0 > 0) {
    const Ell& A = *lv[0]->A;
    k_row_hash<<<stride_grid(n0, 256), 256, 0, s>>>(n0, A.w, A.col, A.val, rowhash, lv[0]->dirty, 1);
    FVS_COUNT_LAUNCH();
  }
  if (lv.size() > 1 && n0 > 0) {
    // level 0: mark the aggregates of changed rows (before the rows of cells
    // without pressure leave them), then rebuild the member lists
    AmgLevel* L = lv[0].get();
    const int64_t nc = lv[1]->n;
    {
      // rows that carry pressure again join the aggregate of the row they
      // couple to most strongly (two passes for chains of such rows); the
      // Galerkin pass below checks that the coarse rows still fit
      const Ell& A = *L->A;
      DBuf<int32_t> agg2;
      FVS_TRY(agg2.alloc(n0 + 1));
      for (int pass = 0; pass < 2; ++pass) {
        k_join_agg<<<stride_grid(n0, 256), 256, 0, s>>>(n0, A.w, A.col, A.val, act, ppe, L->agg, agg2);
        FVS_COUNT_LAUNCH();
        FVS_CUDA(cudaMemcpyAsync(L->agg.p, agg2.p, n0 * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
      }
    }
    k_dirty_up<<<stride_grid(n0, 256), 256, 0, s>>>(n0, L->agg, L->dirty, lv[1]->dirty); FVS_COUNT_LAUNCH();
    k_mask_agg<<<stride_grid(n0, 256), 256, 0, s>>>(n0, act, ppe, L->agg); FVS_COUNT_LAUNCH();
    DBuf<int32_t> mc;
    FVS_TRY(mc.alloc(nc + 1));
    FVS_TRY(mc.zero(s));
    k_count_members<<<stride_grid(n0, 256), 256, 0, s>>>(n0, L->agg, mc); FVS_COUNT_LAUNCH();
    FVS_TRY(exclusive_scan(s, sw, nc + 1, mc, L->mptr));
    FVS_TRY(mc.zero(s));
    k_fill_members<<<stride_grid(n0, 256), 256, 0, s>>>(n0, L->agg, L->mptr, mc, L->midx); FVS_COUNT_LAUNCH();
    k_sort_members<<<stride_grid(nc, 256), 256, 0, s>>>(nc, L->mptr, L->midx); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
  }
  tick(0);
  // Galerkin rows of the dirty aggregates, level by level on the kept
  // aggregation; a coarse row that no longer fits its level's width (a row
  // that joined an aggregate brought new couplings) flags a new setup
  for (size_t l = 0; l < lv.size(); ++l) {
    AmgLevel* L = lv[l].get();
    const Ell* cur = L->A;
    const int64_t n = L->n;
    if (n > 0) {
      k_maxoff<<<stride_grid(n, 256), 256, 0, s>>>(n, cur->w, cur->col, cur->val, mo, L->dinv, cur->diag, L->dirty);
      FVS_COUNT_LAUNCH();
      if (opt.fp32) {
        k_convert_rows<<<stride_grid(n, 256), 256, 0, s>>>(n, cur->w, cur->val, L->dinv, L->dirty, L->valf,
                                                           L->dinvf); FVS_COUNT_LAUNCH();
      }
    }
    if (l + 1 == lv.size()) break;
    AmgLevel* C = lv[l + 1].get();
    if (l > 0 && n > 0) {
      k_dirty_up<<<stride_grid(n, 256), 256, 0, s>>>(n, L->agg, L->dirty, C->dirty); FVS_COUNT_LAUNCH();
    }
    galerkin_pass(s, true, C->n, *cur, L->rlen.p, L->agg, L->mptr, L->midx, C->rlen, C->own.w, C->own.col,
                  C->own.val, C->own.diag, err, C->dirty);
    FVS_LAUNCH_CHECK();
  }
  {
    int e = 0;
    FVS_TRY(read_int(s, err, &e));
    if (e) {
      set_error("AMG refresh needs a new aggregation (flags 0x%x)", e);
      return FVS_ERR_NOT_CONVERGED;
    }
  }
  // the coarsest inverse (a dense O(n^3) factorisation) is kept from the last
  // full setup: the coarse rows above it are exact Galerkin products, and a
  // refreshed solve that slows down rebuilds the hierarchy (redoing the
  // inverse on every fourth refresh measured slower at 128^3: 52.0 against
  // 50.2 ms a step over 20 steps with freezing).  FVS_AMG_COARSEST_EVERY=k
  // redoes it on every k-th refresh.
  tick(1);
  const int every = (int)env_num("FVS_AMG_COARSEST_EVERY", 0);
  if (every > 0 && ++refreshes % every == 0) FVS_TRY(coarsest_setup(s));
  tick(2);
  if (n0 > 0) {
    k_mask_labels<<<stride_grid(n0, 256), 256, 0, s>>>(n0, act, ppe, fine_lab); FVS_COUNT_LAUNCH();
    // rows that carry pressure again take the label of the rows they couple
    // to (a few passes for chains of such rows); a row between two parts, or
    // one left without a label, needs a new setup
    const Ell& A = *lv[0]->A;
    DBuf<int32_t> lab2;
    FVS_TRY(lab2.alloc(n0 + 1));
    int left = 0;
    for (int pass = 0; pass < 4; ++pass) {
      FVS_TRY(cnt2.zero(s));
      k_adopt_labels<<<stride_grid(n0, 256), 256, 0, s>>>(n0, A.w, A.col, A.val, act, ppe, fine_lab, lab2, cnt2,
                                                          err);
      FVS_COUNT_LAUNCH();
      FVS_CUDA(cudaMemcpyAsync(fine_lab.p, lab2.p, n0 * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
      int h[2] = {0, 0};
      FVS_CUDA(cudaMemcpyAsync(h, cnt2.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
      FVS_CUDA(cudaStreamSynchronize(s));
      left = h[0];
      if (left == 0 || h[1] == 0) break;   // done, or no progress
    }
    // rows labelled in the same pass from different sides may now couple two parts
    k_label_conflicts<<<stride_grid(n0, 256), 256, 0, s>>>(n0, A.w, A.col, A.val, fine_lab, err); FVS_COUNT_LAUNCH();
    int e = 0;
    FVS_TRY(read_int(s, err, &e));
    if (e || left) {
      set_error("AMG refresh: rows carrying pressure again need a new setup (flags 0x%x, %d unlabelled)", e, left);
      return FVS_ERR_NOT_CONVERGED;
    }
    FVS_TRY(ccnt.zero(s));
    k_comp_count<<<stride_grid(n0, 256), 256, 0, s>>>(n0, fine_lab, ccnt); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
  }
  tick(3);
  if (dbg)
    fprintf(stderr, "[fvs amg] refresh ms: fingerprints+members %.2f galerkin %.2f coarsest %.2f labels+fp32 %.2f\n",
            tph[0], tph[1], tph[2], tph[3]);
  masked = true;
  FVS_TRY(count_stored(s));
  if (opt.smoother == 1) FVS_TRY(cheb_bounds(s));
  ready = true;
  return FVS_OK;
}

fvs_status Amg::project(cudaStream_t s, double* v) {
  const int64_t n = lv[0]->n;
  if (n == 0 || ncomp == 0) return FVS_OK;
  int nsing = 0, first = -1;
  for (int c = 0; c < ncomp; ++c)
    if (sing_host[c]) { ++nsing; if (first < 0) first = c; }
  if (nsing == 0) return FVS_OK;
  if (nsing == 1) {
    // one singular part (the usual case; the other parts, if any, are rows
    // without pressure): deterministic mean through block partials
    const int nb = std::min(1024, 2 * sm_count());
    const int32_t* mask = (masked || ncomp > 1) ? fine_lab.p : nullptr;
    const int want = ncomp > 1 ? first : -1;
    k_sum_part<<<nb, 256, 0, s>>>(n, v, mask, want, cpart); FVS_COUNT_LAUNCH();
    k_mean_final<<<1, 1024, 0, s>>>(nb, cpart, (double)n, mask ? ccnt.p + first : nullptr, cpart.p + 1024);
    FVS_COUNT_LAUNCH();
    k_sub_scalar<<<stride_grid(n, 256), 256, 0, s>>>(n, cpart.p + 1024, mask, want, v); FVS_COUNT_LAUNCH();
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
fvs_status Amg::vcycle_t(cudaStream_t s, int l, const T* b, T* y, bool x0_ready) {
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
  T* cbv = f32 ? (T*)C->bf.p : (T*)C->b.p;
  T* cy = f32 ? (T*)C->yf.p : (T*)C->y.p;
  const double vb = (double)sizeof(T);
  // kernel timing: every level is credited to the hierarchy's fine operator,
  // coarse levels under their own class names; algorithmic bytes from the
  // entries a sweep reads (value + column per entry) and its vectors
  const void* pkey = lv[0]->A;
  const bool cl = l > 0;
  const double ent = L->stored > 0.0 ? L->stored : (double)n * A.w;
  const double jac_bytes = (4.0 + vb) * ent + 4.0 * vb * (double)n;
  const double res_bytes = (4.0 + vb) * ent + 3.0 * vb * (double)n;
  const int32_t* rl = L->rlen.n ? L->rlen.p : nullptr;   // coarse levels: stored row lengths
  const int g = stride_grid(n, 256);
  const char* n_jac0 = f32 ? (cl ? "jacobi0_f32_coarse" : "jacobi0_f32") : (cl ? "jacobi0_coarse" : "jacobi0");
  const char* n_jac = f32 ? (cl ? "jacobi_f32_coarse" : "jacobi_f32") : (cl ? "jacobi_coarse" : "jacobi");
  const char* n_res = f32 ? (cl ? "residual_f32_coarse" : "residual_f32") : (cl ? "residual_vc_coarse" : "residual_vc");
  const int G = rl ? coarse_lanes(*L) : 1;   // coarse levels: G lanes per row
  const int gg = stride_grid(n * G, 256);
  const T w0 = (T)first_weight(*L);
  auto jac = [&](T* xin, T* xout) {
    ProfScope ps(pkey, n_jac, jac_bytes, s);
    if (!rl) k_jac<T><<<g, 256, 0, s>>>(n, A.w, A.col, val, w0, dinv, b, xin, xout);
    else if (G == 1) k_jac_g<T, 1><<<gg, 256, 0, s>>>(n, A.col, val, w0, dinv, b, xin, xout, rl);
    else if (G == 2) k_jac_g<T, 2><<<gg, 256, 0, s>>>(n, A.col, val, w0, dinv, b, xin, xout, rl);
    else if (G == 4) k_jac_g<T, 4><<<gg, 256, 0, s>>>(n, A.col, val, w0, dinv, b, xin, xout, rl);
    else k_jac_g<T, 8><<<gg, 256, 0, s>>>(n, A.col, val, w0, dinv, b, xin, xout, rl);
    FVS_COUNT_LAUNCH();
  };
  // Chebyshev smoother: interval [cb / ratio, cb], centre th, half-width de;
  // step k >= 1 of the recurrence has rho_k = 1 / (2 th / de - rho_{k-1}),
  // rho_0 = de / th, alpha = 2 rho_k / de, beta = rho_k rho_{k-1}
  const bool cheb = opt.smoother == 1 && L->cheb_b > 0.0;
  const double cb = L->cheb_b, th = 0.5 * (cb + cb / opt.cheb_ratio), de = 0.5 * (cb - cb / opt.cheb_ratio);
  auto cheb_step = [&](T* xin, const T* xprev, T* xout, double& rho) {
    const double rn = 1.0 / (2.0 * th / de - rho);
    const T alpha = (T)(2.0 * rn / de), beta = (T)(rn * rho);
    rho = rn;
    ProfScope ps(pkey, n_jac, jac_bytes + vb * (double)n, s);
    if (!rl) k_cheb<T><<<g, 256, 0, s>>>(n, A.w, A.col, val, alpha, beta, dinv, b, xin, xprev, xout);
    else if (G == 1) k_cheb_g<T, 1><<<gg, 256, 0, s>>>(n, A.col, val, alpha, beta, dinv, b, xin, xprev, xout, rl);
    else if (G == 2) k_cheb_g<T, 2><<<gg, 256, 0, s>>>(n, A.col, val, alpha, beta, dinv, b, xin, xprev, xout, rl);
    else if (G == 4) k_cheb_g<T, 4><<<gg, 256, 0, s>>>(n, A.col, val, alpha, beta, dinv, b, xin, xprev, xout, rl);
    else k_cheb_g<T, 8><<<gg, 256, 0, s>>>(n, A.col, val, alpha, beta, dinv, b, xin, xprev, xout, rl);
    FVS_COUNT_LAUNCH();
  };
  if (!x0_ready) {
    ProfScope ps(pkey, n_jac0, 3.0 * vb * (double)n, s);
    k_jac0<T><<<g, 256, 0, s>>>(n, w0, dinv, b, xa); FVS_COUNT_LAUNCH();
  }
  {
    double rho = cheb ? de / th : 0.0;
    const T* xprev = nullptr;   // the pre-smoothing starts from zero
    for (int k = 1; k < opt.npre; ++k) {
      if (cheb) {
        cheb_step(xa, xprev, xb, rho);
        xprev = xa;
      } else {
        jac(xa, xb);
      }
      T* t = xa; xa = xb; xb = t;
    }
  }
  {
    ProfScope ps(pkey, n_res, res_bytes, s);
    if (!rl) k_resid<T><<<g, 256, 0, s>>>(n, A.w, A.col, val, xa, b, r);
    else if (G == 1) k_resid_g<T, 1><<<gg, 256, 0, s>>>(n, A.col, val, xa, b, r, rl);
    else if (G == 2) k_resid_g<T, 2><<<gg, 256, 0, s>>>(n, A.col, val, xa, b, r, rl);
    else if (G == 4) k_resid_g<T, 4><<<gg, 256, 0, s>>>(n, A.col, val, xa, b, r, rl);
    else k_resid_g<T, 8><<<gg, 256, 0, s>>>(n, A.col, val, xa, b, r, rl);
    FVS_COUNT_LAUNCH();
  }
  // restriction; above a level that is not the coarsest it also forms that
  // level's first Jacobi iterate from zero (row by row, no second launch)
  const bool next_sweeps = l + 2 < (int)lv.size();
  if (next_sweeps) {
    T* cx = f32 ? (T*)C->xf.p : (T*)C->x.p;
    const T* cdinv = f32 ? (const T*)C->dinvf.p : (const T*)C->dinv.p;
    k_restrict_jac0<T><<<stride_grid(C->n, 256), 256, 0, s>>>(C->n, L->mptr, L->midx, r, cbv,
                                                             (T)first_weight(*C), cdinv, cx);
  } else {
    k_restrict<T><<<stride_grid(C->n, 256), 256, 0, s>>>(C->n, L->mptr, L->midx, r, cbv);
  }
  FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  FVS_TRY(vcycle_t<T>(s, l + 1, cbv, cy, next_sweeps));
  k_prolong<T><<<g, 256, 0, s>>>(n, L->agg, cy, (T)opt.coarse_scale, xa); FVS_COUNT_LAUNCH();
  {
    double rho = cheb ? de / th : 0.0;
    for (int k = 0; k < opt.npost; ++k) {
      T* out = (k == opt.npost - 1) ? y : xb;
      if (cheb && k > 0) cheb_step(xa, xb, out, rho);   // xb holds the iterate before xa
      else jac(xa, out);
      xb = xa;
      xa = out;
    }
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

int amg_smem_coarsest() { return SMEM_COARSEST; }

fvs_status amg_coarsest_batched(cudaStream_t s, int n, int w, const int32_t* col, const double* val, int Sp,
                                double* Ainv, int32_t* lab, uint8_t* sing, int* ncomp, int* err) {
  if (n <= 0) return FVS_OK;
  if (n > SMEM_COARSEST) {
    set_error("batched coarsest level has %d rows (at most %d)", n, SMEM_COARSEST);
    return FVS_ERR_NOT_CONVERGED;
  }
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    const size_t shmax = (size_t)SMEM_COARSEST * SMEM_COARSEST * sizeof(double) +
                         (size_t)SMEM_COARSEST * sizeof(double) + 3 * (size_t)SMEM_COARSEST * sizeof(int);
    FVS_CUDA(cudaFuncSetAttribute(k_coarsest_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmax));
    attr_set[dev] = true;
  }
  const size_t sh = (size_t)n * n * sizeof(double) + (size_t)n * sizeof(double) + 3 * (size_t)n * sizeof(int);
  k_coarsest_smem<<<Sp, 1024, sh, s>>>(n, w, col, val, Ainv, lab, sing, ncomp, err, Sp);
  FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

}  // namespace fvs
