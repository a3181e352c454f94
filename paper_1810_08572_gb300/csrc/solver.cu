// The fractional step of Section 2.2 on the GPU:
//  1. tags from T^n (S / LM, Section 2.4), compaction of the LM cells
//  2. momentum predictor u* on LM cells (Eq. 6; rows and columns of solid
//     cells deleted, Section 2.4.1)
//  3. pressure Poisson equation on the flowing LM cells (Eq. 9) with face
//     cases 1/2/3 and smeared gradient coefficients (Section 2.4.2, Eq. 15-16),
//     solved by AMG-preconditioned CG/BiCGStab (Section 2.5)
//  4. face flux and cell velocity correction (Eq. 8, Eq. 17)
//  5. energy with latent heat on all cells (Eq. 4, Eq. 18-20, Section 2.4.4)
//  6. liquidus/solidus crossing times for the microstructure relations (Eq. 22-23)
#include <algorithm>
#include <chrono>
#include <cmath>

#include "fslaw.cuh"
#include "solver.cuh"

extern "C" const char* fvs_last_error(void);

namespace fvs {

#define GS(i, n) for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

struct Mat {
  double rho, k, cp, L, Ts, Tl, mu, beta, Tref, g0, g1, g2, C, eps;
  FsLaw law;    // solid fraction (linear or Eq. 21)
};
constexpr int SOLVER_COARSEST = 1000;   // coarsest AMG level of the single solver (dense inverse)

static Mat mat_of(const fvs_props& p) {
  const fvs_material& m = p.mat;
  return Mat{m.rho, m.k, m.cp, m.latent, m.T_sol, m.T_liq, m.mu, m.beta, m.T_ref, m.g[0], m.g[1], m.g[2],
             m.darcy_C, m.darcy_eps, fs_law_of(m)};
}

// ---------------------------------------------------------------------------
// 1. tags and compaction
// ---------------------------------------------------------------------------
// counts: [1] cells whose tag changed, [2] LM cells outside the current
// system numbering (melted), [3] numbered cells that are no longer LM, [4] LM cells
__global__ void k_tag(int64_t Nc, const double* T, double Ts, uint8_t* lm, int32_t* flag, double* u, double* uold,
                      int* counts, const int32_t* map, int numbered, const uint8_t* metal) {
  int ch = 0, melted = 0, dead = 0, nlm = 0;
  GS(c, Nc) {
    const bool l = metal[c] && T[c] > Ts;   // mold cells are never liquid/mushy
    ch += (lm[c] != (uint8_t)l) ? 1 : 0;
    if (numbered) {
      const bool in = map[c] >= 0;
      melted += (l && !in) ? 1 : 0;
      dead += (!l && in) ? 1 : 0;
    }
    nlm += l ? 1 : 0;
    lm[c] = l;
    flag[c] = l;
    if (!l) {
      for (int d = 0; d < 3; ++d) {
        u[d * Nc + c] = 0.0;
        uold[d * Nc + c] = 0.0;
      }
    }
  }
  if (ch) atomicAdd(counts + 1, ch);
  if (melted) atomicAdd(counts + 2, melted);
  if (dead) atomicAdd(counts + 3, dead);
  if (nlm) atomicAdd(counts + 4, nlm);
}
// a numbering also takes the metal cells across a face from an LM cell: a
// solid cell at the front that melts again then already has a row (an
// identity row until it carries pressure) and the numbering and the AMG
// hierarchy built for it stay in use
__global__ void k_margin(int64_t Nc, const int32_t* cf, const int32_t* own, const int32_t* nei, const uint8_t* lm,
                         const uint8_t* metal, int32_t* flag) {
  GS(c, Nc) {
    if (lm[c] || !metal[c]) continue;
    for (int s = 0; s < 6; ++s) {
      const int32_t f = cf[s * Nc + c];
      const int32_t o = own[f], q = nei[f];
      const int32_t j = o == c ? q : o;
      if (j >= 0 && lm[j]) { flag[c] = 1; break; }
    }
  }
}
__global__ void k_compact(int64_t Nc, const int32_t* flag, const int32_t* excl, int32_t* map, int32_t* act) {
  GS(c, Nc) {
    if (flag[c]) {
      map[c] = excl[c];
      act[excl[c]] = (int32_t)c;
    } else {
      map[c] = -1;
    }
  }
}
// faces with a solid owner (and walls) carry no flux; mark cells with a flowing face
__global__ void k_faces_open(int64_t Nf, const int32_t* own, const int32_t* nei, const uint8_t* lm, double* F,
                             double* Fold, uint8_t* flow) {
  GS(f, Nf) {
    const int32_t o = own[f], q = nei[f];
    const bool open = q >= 0 && lm[o] && lm[q];
    if (!open) {
      F[f] = 0.0;
      Fold[f] = 0.0;
    } else {
      flow[o] = 1;
      flow[q] = 1;
    }
  }
}
__global__ void k_ppe_cells(int64_t Nc, const uint8_t* lm, const uint8_t* flow, uint8_t* ppe) {
  GS(c, Nc) ppe[c] = lm[c] && flow[c];
}
__global__ void k_vertex_nonppe(int64_t Nv, const int32_t* vptr, const int32_t* vidx, const uint8_t* ppe, int32_t* nS) {
  GS(v, Nv) {
    int n = 0;
    for (int32_t e = vptr[v]; e < vptr[v + 1]; ++e) n += ppe[vidx[e]] ? 0 : 1;
    nS[v] = n;
  }
}
// Section 2.4.2: 0 wall, 1 no solid neighbour, 2 solid neighbour only, 3 solid owner
__global__ void k_face_case(int64_t Nf, const int32_t* own, const int32_t* nei, const int32_t* fv, const uint8_t* lm,
                            const int32_t* nS, uint8_t* fcase) {
  GS(f, Nf) {
    const int32_t o = own[f], q = nei[f];
    uint8_t c;
    if (q < 0) c = 0;
    else if (!(lm[o] && lm[q])) c = 3;
    else {
      int s = 0;
      for (int k = 0; k < 4; ++k) s += nS[fv[k * Nf + f]];
      c = s > 0 ? 2 : 1;
    }
    fcase[f] = c;
  }
}

// ---------------------------------------------------------------------------
// 2. momentum predictor (Eq. 6)
// ---------------------------------------------------------------------------
__global__ void k_mom_matrix(int64_t nact, int64_t Nc, int W, const int32_t* act, const int32_t* map,
                             const uint8_t* lm, const int32_t* Lcol, const double* Lval, const double* V,
                             const double* fs, Mat m, double dt, int32_t* col, double* val, double* diag) {
  GS(r, nact) {
    const int32_t c = act[r];
    if (!lm[c]) {
      // a numbered cell that has frozen since the numbering was made: u* = 0
      for (int k = 0; k < W; ++k) {
        col[(int64_t)k * nact + r] = (int32_t)r;
        val[(int64_t)k * nact + r] = k == 0 ? 1.0 : 0.0;
      }
      diag[r] = 1.0;
      continue;
    }
    const double f = fs[c];
    const double D = m.C * f * f / ((1.0 - f) * (1.0 - f) * (1.0 - f) + m.eps);
    const double dterm = (m.rho / dt + D) * V[c];
    bool seen_diag = false;   // padding slots also carry col = c (value 0)
    for (int k = 0; k < W; ++k) {
      const int32_t j = Lcol[(int64_t)k * Nc + c];
      const double a = Lval[(int64_t)k * Nc + c];
      int32_t cc = (int32_t)r;
      double v = 0.0;
      if (j == c) {
        if (!seen_diag) {
          v = dterm - 0.5 * m.mu * a;
          diag[r] = v;
          seen_diag = true;
        }
      } else if (map[j] >= 0 && lm[j]) {
        cc = map[j];
        v = -0.5 * m.mu * a;
      }
      col[(int64_t)k * nact + r] = cc;
      val[(int64_t)k * nact + r] = v;
    }
  }
}

__global__ void k_mom_rhs(int64_t nact, int64_t Nc, int W, const int32_t* act, const uint8_t* lm, const int32_t* cf,
                          const int8_t* cfs, const int32_t* own, const int32_t* nei, const double* F,
                          const double* Fold, const double* u, const double* uold, const int32_t* Lcol,
                          const double* Lval, const double* V, const double* T, Mat m, double dt, double* rhs,
                          double* x) {
  GS(r, nact) {
    const int32_t c = act[r];
    if (!lm[c]) {
      for (int d = 0; d < 3; ++d) {
        rhs[d * nact + r] = 0.0;
        x[d * nact + r] = 0.0;
      }
      continue;
    }
    double cn[3] = {0, 0, 0}, co[3] = {0, 0, 0};
    for (int s = 0; s < 6; ++s) {
      const int32_t f = cf[s * Nc + c];
      const int32_t o = own[f], q = nei[f];
      if (q < 0) continue;
      const double sg = (double)cfs[s * Nc + c];
      const double fn = sg * F[f], fo = sg * Fold[f];
      for (int d = 0; d < 3; ++d) {
        cn[d] += fn * 0.5 * (u[d * Nc + o] + u[d * Nc + q]);
        co[d] += fo * 0.5 * (uold[d * Nc + o] + uold[d * Nc + q]);
      }
    }
    double lu[3] = {0, 0, 0};
    for (int k = 0; k < W; ++k) {
      const int32_t j = Lcol[(int64_t)k * Nc + c];
      const double a = Lval[(int64_t)k * Nc + c];
      for (int d = 0; d < 3; ++d) lu[d] += a * u[d * Nc + j];
    }
    const double Vc = V[c];
    const double bf = -m.rho * m.beta * (T[c] - m.Tref) * Vc;
    const double g[3] = {m.g0, m.g1, m.g2};
    for (int d = 0; d < 3; ++d) {
      rhs[d * nact + r] = m.rho * Vc / dt * u[d * Nc + c] - m.rho * (1.5 * cn[d] - 0.5 * co[d]) +
                          0.5 * m.mu * lu[d] + bf * g[d];
      x[d * nact + r] = u[d * Nc + c];
    }
  }
}

__global__ void k_scatter3(int64_t Nc, int64_t nact, const int32_t* map, const uint8_t* lm, const double* x,
                           double* full) {
  GS(c, Nc) {
    const int32_t r = map[c];
    for (int d = 0; d < 3; ++d) full[d * Nc + c] = (r >= 0 && lm[c]) ? x[d * nact + r] : 0.0;
  }
}

// ---------------------------------------------------------------------------
// 3. pressure system K = -A on LM cells (Eq. 9, Section 2.4.2)
// ---------------------------------------------------------------------------
struct PpeCtx {
  int64_t Nc, Nf, nact;
  int W;
  const int32_t *act, *map, *cf, *own, *nei, *fv, *vc_ptr, *vc_idx, *nb, *nnb, *fnb, *nfnb, *nS;
  const int8_t* cfs;
  const uint8_t *ppe, *fcase;
  const double *cd, *ce, *cz, *Pbval;
  const int32_t* Pbcol;
  double rho;
  int WF;
};

// nbl: the row's sorted neighbour list, copied to thread-local memory once
__device__ __forceinline__ void ppe_vertex(const PpeCtx& x, const int32_t* nbl, int nn, int32_t v, double coef,
                                           double* acc) {
  const int32_t lo = x.vc_ptr[v], hi = x.vc_ptr[v + 1];
  const double share = coef / (double)(hi - lo);
  for (int32_t e = lo; e < hi; ++e) {
    const int32_t j = x.vc_idx[e];
    if (!x.ppe[j]) continue;            // deleted column (solid or non-flowing)
    const int p = find_sorted(nbl, 1, nn, j);
    if (p >= 0) acc[p] += share;
  }
}

__global__ void k_ppe_matrix(PpeCtx x, int32_t* col, double* val, double* diag, int* err) {
  double acc[FVS_MAX_NB];
  GS(r, x.nact) {
    const int32_t c = x.act[r];
    const int nn = x.nnb[c];
    if (!x.ppe[c]) {
      // an LM cell with no flowing face: p = 0 (identity row)
      for (int k = 0; k < x.W; ++k) {
        col[(int64_t)k * x.nact + r] = (int32_t)r;
        val[(int64_t)k * x.nact + r] = k == 0 ? 1.0 : 0.0;
      }
      diag[r] = 1.0;
      continue;
    }
    bool modified = false;
    for (int s = 0; s < 6; ++s) {
      const uint8_t fc = x.fcase[x.cf[s * x.Nc + c]];
      modified |= (fc == 2 || fc == 3);
    }
    if (!modified) {
      // unchanged row: the base coefficients, renumbered
      double dg = 0.0;
      for (int k = 0; k < x.W; ++k) {
        const int32_t j = x.Pbcol[(int64_t)k * x.Nc + c];
        const double a = -x.Pbval[(int64_t)k * x.Nc + c] / x.rho;
        const int32_t mj = x.map[j];
        int32_t cc = (int32_t)r;
        double v = 0.0;
        if (k < nn) {
          if (mj >= 0 && x.ppe[j]) { cc = mj; v = a; }
          else if (a != 0.0) atomicOr(err, 1);
          if (j == c) dg = v;
        }
        col[(int64_t)k * x.nact + r] = cc;
        val[(int64_t)k * x.nact + r] = v;
      }
      diag[r] = dg;
      continue;
    }
    // re-assembly from the faces (Section 2.4.2, step 3)
    int32_t nbl[FVS_MAX_NB];
    for (int k = 0; k < nn; ++k) {
      acc[k] = 0.0;
      nbl[k] = x.nb[(int64_t)k * x.Nc + c];
    }
    for (int s = 0; s < 6; ++s) {
      const int32_t f = x.cf[s * x.Nc + c];
      const uint8_t fc = x.fcase[f];
      if (fc != 1 && fc != 2) continue;
      const double sg = (double)x.cfs[s * x.Nc + c];
      const int32_t o = x.own[f], q = x.nei[f];
      { const int pq = find_sorted(nbl, 1, nn, q); if (pq >= 0) acc[pq] += sg * x.cd[f]; else atomicOr(err, 8); }
      { const int po = find_sorted(nbl, 1, nn, o); if (po >= 0) acc[po] -= sg * x.cd[f]; else atomicOr(err, 8); }
      const int32_t v1 = x.fv[f], v2 = x.fv[x.Nf + f], v3 = x.fv[2 * x.Nf + f], v4 = x.fv[3 * x.Nf + f];
      const double ce = sg * x.ce[f], cz = sg * x.cz[f];
      ppe_vertex(x, nbl, nn, v3, ce, acc);
      ppe_vertex(x, nbl, nn, v1, -ce, acc);
      ppe_vertex(x, nbl, nn, v4, cz, acc);
      ppe_vertex(x, nbl, nn, v2, -cz, acc);
      if (fc == 2) {
        // Eq. 16: the deleted neighbours' coefficients, spread equally over
        // the remaining members of N(f)
        auto frac = [&](int32_t v) {
          return (double)x.nS[v] / (double)(x.vc_ptr[v + 1] - x.vc_ptr[v]);
        };
        const double sdel = ce * (frac(v3) - frac(v1)) + cz * (frac(v4) - frac(v2));
        const int nf = x.nfnb[f];
        int nrem = 0;
        for (int k = 0; k < nf; ++k) nrem += x.ppe[x.fnb[(int64_t)k * x.Nf + f]] ? 1 : 0;
        const double add = sdel / (double)nrem;
        for (int k = 0; k < nf; ++k) {
          const int32_t j = x.fnb[(int64_t)k * x.Nf + f];
          if (!x.ppe[j]) continue;
          const int p = find_sorted(nbl, 1, nn, j);
          if (p >= 0) acc[p] += add;
          else if (add != 0.0) atomicOr(err, 2);   // a zero share may miss a face-only stencil
        }
      }
    }
    double dg = 0.0;
    for (int k = 0; k < x.W; ++k) {
      int32_t cc = (int32_t)r;
      double v = 0.0;
      if (k < nn) {
        const int32_t j = x.nb[(int64_t)k * x.Nc + c];
        const double a = -acc[k] / x.rho;
        const int32_t mj = x.map[j];
        if (mj >= 0 && x.ppe[j]) { cc = mj; v = a; }
        else if (a != 0.0) atomicOr(err, 4);
        if (j == c) dg = v;
      }
      col[(int64_t)k * x.nact + r] = cc;
      val[(int64_t)k * x.nact + r] = v;
    }
    diag[r] = dg;
  }
}

// Operator the pressure preconditioner is built on: each row of K keeps its
// diagonal and its couplings to the cells across its six faces; the
// couplings that the vertex interpolation of the non-orthogonal face
// gradients adds (the other 20 of a 27-point row) are lumped into the
// diagonal.  Row sums are unchanged, so every liquid pocket keeps the
// constant as its null vector.  Slot 0 holds the diagonal, slot 1 + s the
// neighbour across face s (the row itself with a zero where there is none).
__global__ void k_ppe_compact(int64_t nact, int64_t Nc, int W, const int32_t* act, const int32_t* map,
                              const uint8_t* ppe, const int32_t* cf, const int32_t* own, const int32_t* nei,
                              const int32_t* col, const double* val, int32_t* ccol, double* cval, double* cdiag) {
  GS(r, nact) {
    const int32_t c = act[r];
    int32_t fcol[6];
    double fval[6];
    double d = 0.0;
    for (int s = 0; s < 6; ++s) {
      const int32_t f = cf[s * Nc + c];
      const int32_t o = own[f], q = nei[f];
      const int32_t j = o == c ? q : o;
      fcol[s] = (ppe[c] && j >= 0 && map[j] >= 0 && ppe[j]) ? map[j] : -1;
      fval[s] = 0.0;
    }
    for (int k = 0; k < W; ++k) {
      const int32_t cc = col[(int64_t)k * nact + r];
      const double v = val[(int64_t)k * nact + r];
      int hit = -1;
      if (cc != (int32_t)r)
        for (int s = 0; s < 6; ++s)
          if (hit < 0 && fcol[s] == cc) hit = s;
      if (hit >= 0) fval[hit] += v;
      else d += v;
    }
    ccol[r] = (int32_t)r;
    cval[r] = d;
    for (int s = 0; s < 6; ++s) {
      ccol[(int64_t)(1 + s) * nact + r] = fcol[s] >= 0 ? fcol[s] : (int32_t)r;
      cval[(int64_t)(1 + s) * nact + r] = fval[s];
    }
    cdiag[r] = d;
  }
}

// b = (1/dt) sum over flowing faces of sigma A n . (u*_C1 + u*_C2)/2;  K rhs = -b
__global__ void k_ppe_rhs(int64_t nact, int64_t Nc, int64_t Nf, const int32_t* act, const uint8_t* ppe,
                          const int32_t* cf, const int8_t* cfs, const uint8_t* fcase, const int32_t* own,
                          const int32_t* nei, const double* A, const double* nrm, const double* us, double dt,
                          const double* p, double* rhs, double* x) {
  GS(r, nact) {
    const int32_t c = act[r];
    double b = 0.0;
    if (ppe[c]) {
      for (int s = 0; s < 6; ++s) {
        const int32_t f = cf[s * Nc + c];
        const uint8_t fc = fcase[f];
        if (fc != 1 && fc != 2) continue;
        const int32_t o = own[f], q = nei[f];
        double un = 0.0;
        for (int d = 0; d < 3; ++d) un += nrm[d * Nf + f] * 0.5 * (us[d * Nc + o] + us[d * Nc + q]);
        b += (double)cfs[s * Nc + c] * A[f] * un;
      }
      b /= dt;
    }
    rhs[r] = -b;
    x[r] = ppe[c] ? p[c] : 0.0;
  }
}

__global__ void k_scatter1(int64_t Nc, const int32_t* map, const uint8_t* ppe, const double* x, double* full) {
  GS(c, Nc) {
    const int32_t r = map[c];
    full[c] = (r >= 0 && ppe[c]) ? x[r] : 0.0;
  }
}

// ---------------------------------------------------------------------------
// 4. correction (Eq. 17 and the cell-centred gradient of Section 2.4.3)
// ---------------------------------------------------------------------------
__global__ void k_vertex_p(int64_t Nv, const int32_t* vptr, const int32_t* vidx, const uint8_t* ppe, const double* p,
                           const int32_t* nS, double* pv, double* fS) {
  GS(v, Nv) {
    const int32_t lo = vptr[v], hi = vptr[v + 1];
    double s = 0.0;
    for (int32_t e = lo; e < hi; ++e) {
      const int32_t j = vidx[e];
      if (ppe[j]) s += p[j];
    }
    const double n = (double)(hi - lo);
    pv[v] = s / n;
    fS[v] = (double)nS[v] / n;
  }
}

__global__ void k_face_correct(int64_t Nf, int64_t Nc, const int32_t* own, const int32_t* nei, const int32_t* fv,
                               const uint8_t* fcase, const int32_t* fnb, const int32_t* nfnb, const uint8_t* ppe,
                               const double* p, const double* pv, const double* fS, const double* A,
                               const double* nrm, const double* cd, const double* ce, const double* cz,
                               const double* Jinv, const double* us, double dt, double rho, double* Fnew,
                               double* gradf) {
  GS(f, Nf) {
    const uint8_t fc = fcase[f];
    if (fc != 1 && fc != 2) {
      Fnew[f] = 0.0;
      for (int d = 0; d < 3; ++d) gradf[d * Nf + f] = 0.0;
      continue;
    }
    const int32_t o = own[f], q = nei[f];
    const int32_t v1 = fv[f], v2 = fv[Nf + f], v3 = fv[2 * Nf + f], v4 = fv[3 * Nf + f];
    const double dxi = p[q] - p[o];
    double deta = pv[v3] - pv[v1];
    double dzeta = pv[v4] - pv[v2];
    if (fc == 2) {
      // deleted neighbours take the mean of the remaining ones (Eq. 16)
      const int nf = nfnb[f];
      double s = 0.0;
      int n = 0;
      for (int k = 0; k < nf; ++k) {
        const int32_t j = fnb[(int64_t)k * Nf + f];
        if (ppe[j]) { s += p[j]; ++n; }
      }
      const double pbar = s / (double)n;
      deta += (fS[v3] - fS[v1]) * pbar;
      dzeta += (fS[v4] - fS[v2]) * pbar;
    }
    const double nd = cd[f] * dxi + ce[f] * deta + cz[f] * dzeta;   // A (n . grad p)
    double un = 0.0;
    for (int d = 0; d < 3; ++d) un += nrm[d * Nf + f] * 0.5 * (us[d * Nc + o] + us[d * Nc + q]);
    Fnew[f] = A[f] * un - dt / rho * nd;
    for (int d = 0; d < 3; ++d)
      gradf[d * Nf + f] = Jinv[(3 * d + 0) * Nf + f] * dxi + Jinv[(3 * d + 1) * Nf + f] * deta +
                          Jinv[(3 * d + 2) * Nf + f] * dzeta;
  }
}

__global__ void k_cell_correct(int64_t Nc, int64_t Nf, const uint8_t* lm, const int32_t* cf, const uint8_t* fcase,
                               const double* gradf, const double* us, double dt, double rho, double* unew) {
  GS(c, Nc) {
    if (!lm[c]) {
      for (int d = 0; d < 3; ++d) unew[d * Nc + c] = 0.0;
      continue;
    }
    double g[3] = {0, 0, 0};
    int n = 0;
    for (int s = 0; s < 6; ++s) {
      const int32_t f = cf[s * Nc + c];
      const uint8_t fc = fcase[f];
      if (fc != 1 && fc != 2) continue;
      ++n;
      for (int d = 0; d < 3; ++d) g[d] += gradf[d * Nf + f];
    }
    for (int d = 0; d < 3; ++d)
      unew[d * Nc + c] = us[d * Nc + c] - (n > 0 ? dt / rho * g[d] / (double)n : 0.0);
  }
}

// ---------------------------------------------------------------------------
// 5. energy with latent heat (Eq. 4, Eq. 18-20)
// ---------------------------------------------------------------------------
// Lval / lT: the conductive operator (conductivities inside); rcp = rho cp per cell
__global__ void k_energy_base(int64_t Nc, int W, const int32_t* cf, const int8_t* cfs, const int32_t* own,
                              const int32_t* nei, const double* F, const double* Fold, const double* T,
                              const double* Told, const int32_t* Lcol, const double* Lval, const double* lT,
                              const double* V, const double* rcp, double dt, double* base) {
  GS(c, Nc) {
    double cn = 0.0, co = 0.0;
    for (int s = 0; s < 6; ++s) {
      const int32_t f = cf[s * Nc + c];
      const int32_t o = own[f], q = nei[f];
      if (q < 0) continue;
      const double sg = (double)cfs[s * Nc + c];
      cn += sg * F[f] * 0.5 * (T[o] + T[q]);
      co += sg * Fold[f] * 0.5 * (Told[o] + Told[q]);
    }
    double lt = 0.0;
    for (int k = 0; k < W; ++k) lt += Lval[(int64_t)k * Nc + c] * T[Lcol[(int64_t)k * Nc + c]];
    base[c] = rcp[c] * V[c] / dt * T[c] - rcp[c] * (1.5 * cn - 0.5 * co) + 0.5 * lt + lT[c];
  }
}

// source linearisation at the current iterate (Eq. 20): S_p, S_c
__global__ void k_energy_lin(int64_t Nc, const double* V, Mat m, double dt, const double* Tm, const double* fsm,
                             const double* fsn, const double* base, double* dextra, double* rhs, double* x,
                             const double* rcp, const double* rL, const uint8_t* metal, const double* kdiag,
                             double* jinv) {
  GS(c, Nc) {
    const double t = Tm[c];
    const double dfs = metal[c] ? fs_slope(m.law, t) : 0.0;
    const double a = rL[c] * V[c] / dt;
    const double Sp = a * dfs;
    const double Sc = a * (fsm[c] - fsn[c] - dfs * t);
    const double dx = rcp[c] * V[c] / dt - Sp;
    dextra[c] = dx;
    jinv[c] = 1.0 / (kdiag[c] + dx);   // Jacobi preconditioner of the pass
    rhs[c] = base[c] + Sc;
    x[c] = t;
  }
}

__global__ void k_inverse(int64_t n, const double* a, double* inv) {
  GS(i, n) inv[i] = 1.0 / a[i];
}

// enthalpy-to-temperature inversion of the linearised update:
// H = cp T_lin + L (1 - fs^m - dfs (T_lin - T^m)), T = H^-1(H), fs = fs(T)
__global__ void k_energy_update(int64_t Nc, Mat m, const double* Tlin, const double* Tm, const double* fsm,
                                double* Tnext, double* fsnext, const uint8_t* metal) {
  GS(c, Nc) {
    if (!metal[c]) {      // mold: no latent heat
      Tnext[c] = Tlin[c];
      fsnext[c] = 0.0;
      continue;
    }
    const double t = Tm[c];
    const double dfs = fs_slope(m.law, t);
    const double H = m.cp * Tlin[c] + m.L * (1.0 - fsm[c] - dfs * (Tlin[c] - t));
    const double T = T_of_H(m.law, m.cp, m.L, H);
    Tnext[c] = T;
    fsnext[c] = fs_of(m.law, T);
  }
}

__global__ void k_count_u8(int64_t n, const uint8_t* a, int* out) {
  int c = 0;
  GS(i, n) c += a[i] ? 1 : 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// first iterate of the latent-heat loop: T^n extrapolated linearly in time
// (the loop converges to the same discrete solution from any start, within
// its stop rule; this start is closer)
__global__ void k_energy_guess(int64_t Nc, const double* T, const double* Told, FsLaw law, double* Tm,
                               double* fsm, const uint8_t* metal) {
  GS(c, Nc) {
    const double t = 2.0 * T[c] - Told[c];
    Tm[c] = t;
    fsm[c] = metal[c] ? fs_of(law, t) : 0.0;
  }
}
__global__ void k_crossings(int64_t Nc, const double* Tn, const double* Tnew, double Ts, double Tl, double time,
                            double dt, double* tliq, double* tsol, const uint8_t* metal) {
  GS(c, Nc) {
    if (!metal[c]) continue;
    const double a = Tn[c], b = Tnew[c];
    if (tliq[c] < 0.0 && a > Tl && b <= Tl) tliq[c] = time + dt * (a - Tl) / (a - b);
    if (tsol[c] < 0.0 && a > Ts && b <= Ts) tsol[c] = time + dt * (a - Ts) / (a - b);
  }
}

// grain growth (Eq. 24-26): lambda_s of the invariant-size approximation for
// the Scheil interface contents (C_0 / C_l = (1 - fs)^(1 - kp)), zero outside
// the mushy range
__device__ __forceinline__ double grain_lambda(double fs, double kp) {
  if (!(fs > 0.0 && fs < 1.0)) return 0.0;
  const double S = 2.0 * (1.0 - pow(1.0 - fs, 1.0 - kp)) / (kp - 1.0);
  const double pi = 3.14159265358979323846;
  return -S / (2.0 * sqrt(pi)) + sqrt(fmax(S * S / (4.0 * pi) - S, 0.0));
}
// d(r^2)/dt = lambda_s^2 D_s, trapezoidal over the step
__global__ void k_grain(int64_t Nc, const double* fsa, const double* fsb, const uint8_t* metal, double kp, double Ds,
                        double dt, double* r2) {
  GS(c, Nc) {
    if (!metal[c]) continue;
    const double la = grain_lambda(fsa[c], kp), lb = grain_lambda(fsb[c], kp);
    r2[c] += dt * Ds * 0.5 * (la * la + lb * lb);
  }
}
__global__ void k_grain_init(int64_t Nc, const uint8_t* metal, double r0, double* r2) {
  GS(c, Nc) r2[c] = metal[c] ? r0 * r0 : 0.0;
}
__global__ void k_sqrt_out(int64_t n, const int32_t* to_in, const double* a, double* out) {
  GS(c, n) out[to_in[c]] = sqrt(a[c]);
}

// ---------------------------------------------------------------------------
// state set-up and queries
// ---------------------------------------------------------------------------
__global__ void k_init_state(int64_t Nc, const int32_t* cell_in, const double* Tin, double Tuni, const double* uin,
                             Mat m, double* T, double* Told, double* fs, double* u, double* uold, double* p,
                             double* tliq, double* tsol, const uint8_t* metal, double T_mold) {
  GS(c, Nc) {
    const int32_t o = cell_in[c];
    const bool me = metal[c] != 0;
    const double t = Tin ? Tin[o] : (me ? Tuni : T_mold);
    T[c] = t;
    Told[c] = t;
    fs[c] = me ? fs_of(m.law, t) : 0.0;
    const bool solid = !(me && t > m.Ts);
    for (int d = 0; d < 3; ++d) {
      const double v = (uin && !solid) ? uin[3 * (int64_t)o + d] : 0.0;
      u[d * Nc + c] = v;
      uold[d * Nc + c] = v;
    }
    p[c] = 0.0;
    tliq[c] = me && t <= m.Tl ? 0.0 : -1.0;
    tsol[c] = me && t <= m.Ts ? 0.0 : -1.0;
  }
}

// materials per cell and conductance per face (metal and, with a mold
// material, mold zones; Section 2.4.4 energy equation on all cells)
struct MoldMat {
  int on;
  double rho_cp, k, rho_L;
  double mold_rho_cp, mold_k, h;
  MoldMat(int on_, double rho, double cp, double k_, double rhoL, double mrho, double mcp, double mk, double h_)
      : on(on_), rho_cp(rho * cp), k(k_), rho_L(rhoL), mold_rho_cp(mrho * mcp), mold_k(mk), h(h_) {}
};
// piecewise-linear k(T) of the metal, constant outside the table (n = 0:
// the constant k of the material)
struct KTable {
  int n = 0;
  double T[16], k[16];
};
__device__ __forceinline__ double k_metal(const KTable& t, double k0, double T) {
  if (t.n == 0) return k0;
  if (T <= t.T[0]) return t.k[0];
  for (int i = 1; i < t.n; ++i)
    if (T <= t.T[i]) return t.k[i - 1] + (t.k[i] - t.k[i - 1]) * (T - t.T[i - 1]) / (t.T[i] - t.T[i - 1]);
  return t.k[t.n - 1];
}
__global__ void k_cell_materials(int64_t Nc, const uint8_t* zone, MoldMat mm, uint8_t* metal, double* rcp,
                                 double* rL) {
  GS(c, Nc) {
    const bool me = !mm.on || zone[c] == 0;
    metal[c] = me ? 1 : 0;
    rcp[c] = me ? mm.rho_cp : mm.mold_rho_cp;
    rL[c] = me ? mm.rho_L : 0.0;
  }
}
// kf: conductivity of the face (metal: k at the mean of the two cells' T, or
// of the cell and a fixed wall value, when k depends on T; the mold: its
// constant k); gint > 0 on a face between a metal and a mold cell:
// A / (d_own/k_own + 1/h + d_nei/k_nei), and on a convective wall:
// A / (d_own/k_own + 1/h_wall).  T may be null when k is constant.
__global__ void k_face_conductance(int64_t Nf, const int32_t* own, const int32_t* nei, const int32_t* patch,
                                   const int32_t* bc_type, const double* bc_T, const double* bc_h,
                                   const uint8_t* metal, const double* A, const double* dof, const double* dnf,
                                   MoldMat mm, KTable kt, const double* T, double* kf, double* gint) {
  GS(f, Nf) {
    const int32_t o = own[f], q = nei[f];
    const double To = T ? T[o] : 0.0;
    const double ko = metal[o] ? k_metal(kt, mm.k, To) : mm.mold_k;
    double k = ko, g = 0.0;
    if (q >= 0) {
      if (metal[o] != metal[q]) {
        const double kq = metal[q] ? k_metal(kt, mm.k, T ? T[q] : 0.0) : mm.mold_k;
        g = A[f] / (dof[f] / ko + 1.0 / mm.h + dnf[f] / kq);
      } else if (metal[o] && T) {
        k = k_metal(kt, mm.k, 0.5 * (To + T[q]));
      }
    } else {
      const int32_t b = patch[f];
      if (bc_type[b] == FVS_BC_CONVECTIVE) g = A[f] / (dof[f] / ko + 1.0 / bc_h[b]);
      else if (bc_type[b] == FVS_BC_DIRICHLET && metal[o] && T) k = k_metal(kt, mm.k, 0.5 * (To + bc_T[b]));
    }
    kf[f] = k;
    gint[f] = g;
  }
}

__global__ void k_gather_out(int64_t n, int comps, const int32_t* to_in, const double* src, double* dst) {
  GS(i, n) {
    const int64_t o = to_in[i];
    for (int d = 0; d < comps; ++d) dst[comps * o + d] = src[d * n + i];
  }
}
__global__ void k_gather_u8(int64_t n, const int32_t* to_in, const uint8_t* src, double* dst) {
  GS(i, n) dst[to_in[i]] = (double)src[i];
}
__global__ void k_qoi(int64_t Nc, const int32_t* to_in, const double* tliq, const double* tsol, double Ts, double Tl,
                      double* dst) {
  GS(c, Nc) {
    const int64_t o = to_in[c];
    double tf = __longlong_as_double(0x7ff8000000000000LL), cr = tf, lam = tf, ys = tf;
    if (tliq[c] >= 0.0 && tsol[c] >= 0.0) {
      tf = tsol[c] - tliq[c];
      cr = (Tl - Ts) / tf;
      lam = 39.4 * pow(cr, -0.317);          // Eq. 22 (micrometres)
      ys = 59.0 / sqrt(lam) + 120.3;         // Eq. 23 (MPa)
    }
    dst[4 * o] = tf;
    dst[4 * o + 1] = cr;
    dst[4 * o + 2] = lam;
    dst[4 * o + 3] = ys;
  }
}
__global__ void k_scale_ell(int64_t n, int w, double a, const double* val, const double* diag, double* oval,
                            double* odiag) {
  GS(i, n) {
    for (int k = 0; k < w; ++k) oval[(int64_t)k * n + i] = a * val[(int64_t)k * n + i];
    odiag[i] = a * diag[i];
  }
}
__global__ void k_copy_i(int64_t n, const int32_t* a, int32_t* b) {
  GS(i, n) b[i] = a[i];
}
__global__ void k_rhs_in(int64_t nact, const int32_t* act, const uint8_t* ppe, const int32_t* cell_in,
                         const double* rhs_in, double* rhs, double* x) {
  GS(r, nact) {
    const int32_t c = act[r];
    rhs[r] = ppe[c] ? -rhs_in[cell_in[c]] : 0.0;
    x[r] = 0.0;
  }
}
__global__ void k_p_out(int64_t Nc, const int32_t* map, const uint8_t* ppe, const int32_t* cell_in, const double* x,
                        double* out) {
  GS(c, Nc) {
    const int32_t r = map[c];
    out[cell_in[c]] = (r >= 0 && ppe[c]) ? x[r] : 0.0;
  }
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
fvs_status solver_alloc(fvs_solver s) {
  fvs_mesh m = s->mesh;
  const int64_t Nc = m->Nc, Nf = m->Nf, Nv = m->Nv;
  FVS_TRY(s->T.alloc(Nc)); FVS_TRY(s->Told.alloc(Nc)); FVS_TRY(s->Tnew.alloc(Nc));
  FVS_TRY(s->fs.alloc(Nc)); FVS_TRY(s->fsnew.alloc(Nc));
  FVS_TRY(s->u.alloc(3 * Nc)); FVS_TRY(s->uold.alloc(3 * Nc)); FVS_TRY(s->unew.alloc(3 * Nc));
  FVS_TRY(s->ustar.alloc(3 * Nc));
  FVS_TRY(s->F.alloc(Nf)); FVS_TRY(s->Fold.alloc(Nf)); FVS_TRY(s->Fnew.alloc(Nf));
  FVS_TRY(s->p.alloc(Nc)); FVS_TRY(s->tliq.alloc(Nc)); FVS_TRY(s->tsol.alloc(Nc));
  FVS_TRY(s->lm.alloc(Nc)); FVS_TRY(s->ppe.alloc(Nc)); FVS_TRY(s->flow.alloc(Nc)); FVS_TRY(s->fcase.alloc(Nf));
  FVS_TRY(s->flag.alloc(Nc + 1)); FVS_TRY(s->excl.alloc(Nc + 1)); FVS_TRY(s->map.alloc(Nc));
  FVS_TRY(s->act.alloc(Nc + 1)); FVS_TRY(s->nS.alloc(Nv));
  FVS_TRY(s->pv.alloc(Nv)); FVS_TRY(s->fSv.alloc(Nv)); FVS_TRY(s->gradf.alloc(3 * Nf));
  FVS_TRY(s->ebase.alloc(Nc)); FVS_TRY(s->erhs.alloc(Nc)); FVS_TRY(s->edx.alloc(Nc)); FVS_TRY(s->Tlin.alloc(Nc));
  FVS_TRY(s->lT.alloc(Nc));
  FVS_TRY(s->Tit.alloc(Nc)); FVS_TRY(s->fsit.alloc(Nc));
  FVS_TRY(s->cnt.alloc(8));
  FVS_TRY(s->red.init());
  FVS_TRY(s->ustar.zero(s->stream));
  FVS_TRY(s->fcase.zero(s->stream));
  s->aproj.amg = &s->amg;
  return FVS_OK;
}

static fvs_status apply_properties(fvs_solver s, const fvs_props* p);
static fvs_status conduction_operator(fvs_solver s);

fvs_status solver_set_properties(fvs_solver s, const fvs_props* p) {
  s->has_mold = false;   // new properties: every cell metal until fvs_set_mold
  return apply_properties(s, p);
}

fvs_status solver_set_mold(fvs_solver s, double rho, double cp, double k, double h, double T_init) {
  if (!s->have_props) {
    set_error("fvs_set_properties must come first");
    return FVS_ERR_STATE;
  }
  if (!(rho > 0 && cp > 0 && k > 0 && h > 0)) {
    set_error("invalid mold data (rho, cp, k and h must be positive)");
    return FVS_ERR_ARG;
  }
  s->has_mold = true;
  s->mold_rho = rho;
  s->mold_cp = cp;
  s->mold_k = k;
  s->mold_h = h;
  s->mold_T = T_init;
  std::vector<fvs_patch_bc> bc = s->bc;
  const std::vector<double> kT(s->k_T, s->k_T + s->n_k), kv(s->k_val, s->k_val + s->n_k);
  fvs_props p = s->props;
  p.bc = bc.data();
  p.n_patches = (int32_t)bc.size();
  p.n_k = s->n_k;
  p.k_T = kT.data();
  p.k_val = kv.data();
  return apply_properties(s, &p);
}

fvs_status solver_set_grain(fvs_solver s, double kp, double D_s, double r0) {
  if (!s->have_props) {
    set_error("fvs_set_properties must come first");
    return FVS_ERR_STATE;
  }
  if (!(kp > 0.0 && kp < 1.0 && D_s >= 0.0 && r0 >= 0.0)) {
    set_error("invalid grain-growth data (0 < kp < 1, D_s >= 0, r0 >= 0)");
    return FVS_ERR_ARG;
  }
  s->grain_on = D_s > 0.0;
  s->grain_kp = kp;
  s->grain_Ds = D_s;
  s->grain_r0 = r0;
  const int64_t Nc = s->mesh->Nc;
  FVS_TRY(s->r2.alloc(Nc));
  k_grain_init<<<stride_grid(Nc, 256), 256, 0, s->stream>>>(Nc, s->metal, r0, s->r2); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  FVS_CUDA(cudaStreamSynchronize(s->stream));
  return FVS_OK;
}

static fvs_status apply_properties(fvs_solver s, const fvs_props* p) {
  fvs_mesh m = s->mesh;
  if (p->n_patches < m->npatch || (p->n_patches > 0 && !p->bc)) {
    set_error("props give %d wall patches, the mesh uses %d", p->n_patches, m->npatch);
    return FVS_ERR_ARG;
  }
  const fvs_material& mt = p->mat;
  if (!(mt.rho > 0 && mt.k > 0 && mt.cp > 0 && mt.T_liq > mt.T_sol && mt.mu >= 0 && mt.latent >= 0)) {
    set_error("invalid material data");
    return FVS_ERR_ARG;
  }
  if (!fs_law_valid(mt, mt.T_liq)) {
    set_error("invalid solid-fraction law (model %d; Scheil needs 0 < kp < 1, T_eps > 0, "
              "T_sol + T_eps < T_liq < T_f)", (int)mt.fs_model);
    return FVS_ERR_ARG;
  }
  for (int i = 0; i < p->n_patches; ++i) {
    const int t = p->bc[i].type;
    if (t != FVS_BC_ADIABATIC && t != FVS_BC_DIRICHLET && t != FVS_BC_CONVECTIVE) {
      set_error("patch %d: unknown wall type %d", i, t);
      return FVS_ERR_ARG;
    }
    if (t == FVS_BC_CONVECTIVE && !(p->bc[i].h > 0)) {
      set_error("patch %d: a convective wall needs h > 0", i);
      return FVS_ERR_ARG;
    }
  }
  if (p->n_k < 0 || p->n_k > 16 || (p->n_k > 0 && (!p->k_T || !p->k_val))) {
    set_error("k(T) table: 0..16 points with both arrays given");
    return FVS_ERR_ARG;
  }
  for (int i = 0; i < p->n_k; ++i) {
    if (!(p->k_val[i] > 0) || (i > 0 && !(p->k_T[i] > p->k_T[i - 1]))) {
      set_error("k(T) table: temperatures must increase and conductivities be positive");
      return FVS_ERR_ARG;
    }
  }
  s->props = *p;
  s->bc.assign(p->bc, p->bc + p->n_patches);
  s->props.bc = nullptr;
  s->n_k = p->n_k;
  for (int i = 0; i < p->n_k; ++i) {
    s->k_T[i] = p->k_T[i];
    s->k_val[i] = p->k_val[i];
  }
  s->props.k_T = nullptr;
  s->props.k_val = nullptr;
  if (s->props.max_krylov_iters <= 0) s->props.max_krylov_iters = 500;
  if (s->props.max_e_iters <= 0) s->props.max_e_iters = 40;
  if (!(s->props.p_rtol > 0)) s->props.p_rtol = 1e-8;
  if (!(s->props.mom_rtol > 0)) s->props.mom_rtol = 1e-10;
  if (!(s->props.e_rtol > 0)) s->props.e_rtol = 1e-10;
  if (!(s->props.e_tol_T > 0)) s->props.e_tol_T = 1e-8;
  const int np = std::max(1, p->n_patches);
  std::vector<int32_t> ht(np, 0);
  std::vector<double> hT(np, 0.0), hh(np, 0.0);
  for (int i = 0; i < p->n_patches; ++i) {
    ht[i] = p->bc[i].type;
    hT[i] = p->bc[i].T;
    hh[i] = p->bc[i].h;
  }
  FVS_TRY(s->bc_type.alloc(np));
  FVS_TRY(s->bc_T.alloc(np));
  FVS_TRY(s->bc_h.alloc(np));
  FVS_CUDA(cudaMemcpyAsync(s->bc_type.p, ht.data(), np * sizeof(int32_t), cudaMemcpyHostToDevice, s->stream));
  FVS_CUDA(cudaMemcpyAsync(s->bc_T.p, hT.data(), np * sizeof(double), cudaMemcpyHostToDevice, s->stream));
  FVS_CUDA(cudaMemcpyAsync(s->bc_h.p, hh.data(), np * sizeof(double), cudaMemcpyHostToDevice, s->stream));
  // the host vectors must outlive the copies
  FVS_CUDA(cudaStreamSynchronize(s->stream));
  // materials per cell (zones count only with a mold material) and the
  // conductive operator: k_f times the face gradient, the series flux on
  // metal-mold faces
  FVS_TRY(s->metal.alloc(m->Nc)); FVS_TRY(s->rcp.alloc(m->Nc)); FVS_TRY(s->rL.alloc(m->Nc));
  FVS_TRY(s->kface.alloc(m->Nf)); FVS_TRY(s->gint.alloc(m->Nf));
  const MoldMat mm{s->has_mold ? 1 : 0, mt.rho, mt.cp, mt.k, mt.rho * mt.latent, s->mold_rho, s->mold_cp, s->mold_k,
                   s->mold_h};
  k_cell_materials<<<stride_grid(m->Nc, 256), 256, 0, s->stream>>>(m->Nc, m->zone, mm, s->metal, s->rcp, s->rL);
  FVS_COUNT_LAUNCH();
  s->have_props = true;
  FVS_TRY(solver_set_state(s, nullptr, nullptr, 0));
  return conduction_operator(s);
}

// conductive operator L (face conductivities inside; with k(T) those of the
// current T) and Ke = -1/2 L with the same pattern
static fvs_status conduction_operator(fvs_solver s) {
  fvs_mesh m = s->mesh;
  const fvs_material& mt = s->props.mat;
  const MoldMat mm{s->has_mold ? 1 : 0, mt.rho, mt.cp, mt.k, mt.rho * mt.latent, s->mold_rho, s->mold_cp, s->mold_k,
                   s->mold_h};
  KTable kt;
  kt.n = s->n_k;
  for (int i = 0; i < s->n_k; ++i) {
    kt.T[i] = s->k_T[i];
    kt.k[i] = s->k_val[i];
  }
  k_face_conductance<<<stride_grid(m->Nf, 256), 256, 0, s->stream>>>(
      m->Nf, m->own, m->nei, m->patch, s->bc_type, s->bc_T, s->bc_h, s->metal, m->A, m->dof, m->dnf, mm, kt,
      s->n_k > 0 ? s->T.p : nullptr, s->kface, s->gint);
  FVS_COUNT_LAUNCH();
  FVS_TRY(assemble_temperature_operator(m, s->bc_type, s->bc_T, s->LT, s->lT, s->stream, s->kface, s->gint));
  FVS_TRY(s->Ke.alloc(m->Nc, m->W));
  k_copy_i<<<stride_grid((int64_t)m->Nc * m->W, 256), 256, 0, s->stream>>>((int64_t)m->Nc * m->W, s->LT.col,
                                                                            s->Ke.col); FVS_COUNT_LAUNCH();
  k_scale_ell<<<stride_grid(m->Nc, 256), 256, 0, s->stream>>>(m->Nc, m->W, -0.5, s->LT.val, s->LT.diag,
                                                             s->Ke.val, s->Ke.diag); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

fvs_status solver_set_state(fvs_solver s, const double* T, const double* u, int on_device) {
  if (!s->have_props) {
    set_error("fvs_set_properties must come first");
    return FVS_ERR_STATE;
  }
  fvs_mesh m = s->mesh;
  const int64_t Nc = m->Nc;
  cudaStream_t st = s->stream;
  DBuf<double> dT, du;
  const double* pT = T;
  const double* pu = u;
  if (T && !on_device) {
    FVS_TRY(dT.alloc(Nc));
    FVS_CUDA(cudaMemcpyAsync(dT.p, T, Nc * sizeof(double), cudaMemcpyHostToDevice, st));
    pT = dT.p;
  }
  if (u && !on_device) {
    FVS_TRY(du.alloc(3 * Nc));
    FVS_CUDA(cudaMemcpyAsync(du.p, u, 3 * Nc * sizeof(double), cudaMemcpyHostToDevice, st));
    pu = du.p;
  }
  const Mat mt = mat_of(s->props);
  k_init_state<<<stride_grid(Nc, 256), 256, 0, st>>>(Nc, m->cell_in, pT, s->props.T_init, pu, mt, s->T, s->Told,
                                                     s->fs, s->u, s->uold, s->p, s->tliq, s->tsol, s->metal,
                                                     s->mold_T);
  FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  FVS_TRY(s->F.zero(st)); FVS_TRY(s->Fold.zero(st)); FVS_TRY(s->Fnew.zero(st));
  FVS_TRY(s->ustar.zero(st));
  FVS_TRY(s->r2.alloc(Nc));
  k_grain_init<<<stride_grid(Nc, 256), 256, 0, st>>>(Nc, s->metal, s->grain_r0, s->r2); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  FVS_CUDA(cudaStreamSynchronize(st));
  s->time = 0.0;
  s->nstep = 0;
  s->have_step = false;
  s->k_valid = false;
  s->numbered = false;
  s->force_full = false;
  s->amg_ok = false;
  return FVS_OK;
}

// tags, compaction and face cases for the current temperature
// a new system numbering: the LM cells in mesh order
static fvs_status renumber_lm(fvs_solver s) {
  fvs_mesh m = s->mesh;
  cudaStream_t st = s->stream;
  const int64_t Nc = m->Nc;
  const char* mg = getenv("FVS_MARGIN");
  if (!(mg && *mg == '0')) {
    k_margin<<<stride_grid(Nc, 256), 256, 0, st>>>(Nc, m->cf, m->own, m->nei, s->lm, s->metal, s->flag);
    FVS_COUNT_LAUNCH();
  }
  FVS_TRY(exclusive_scan(st, s->sw, Nc + 1, s->flag, s->excl));
  k_compact<<<stride_grid(Nc, 256), 256, 0, st>>>(Nc, s->flag, s->excl, s->map, s->act); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  int32_t na = 0;
  FVS_CUDA(cudaMemcpyAsync(&na, s->excl.p + Nc, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  FVS_CUDA(cudaStreamSynchronize(st));
  s->nact = na;
  s->nmargin = std::max<int64_t>(0, (int64_t)na - s->nlm);
  s->numbered = true;
  s->renumbered = true;
  s->k_valid = false;
  return FVS_OK;
}

static fvs_status classify(fvs_solver s) {
  fvs_mesh m = s->mesh;
  cudaStream_t st = s->stream;
  const int64_t Nc = m->Nc, Nf = m->Nf, Nv = m->Nv;
  const Mat mt = mat_of(s->props);
  FVS_TRY(s->flag.zero(st));
  FVS_TRY(s->cnt.zero(st));
  k_tag<<<stride_grid(Nc, 256), 256, 0, st>>>(Nc, s->T, mt.Ts, s->lm, s->flag, s->u, s->uold, s->cnt.p,
                                               s->map, s->numbered ? 1 : 0, s->metal);
  FVS_COUNT_LAUNCH();
  int tc[5];
  FVS_CUDA(cudaMemcpyAsync(tc, s->cnt.p, 5 * sizeof(int), cudaMemcpyDeviceToHost, st));
  FVS_CUDA(cudaStreamSynchronize(st));
  s->nlm = tc[4];
  // The system numbering (LM cells when it was made, and the solid metal
  // cells across a face from them) is kept while cells freeze or the cells
  // of that margin melt, and the frozen share stays small: rows of cells
  // without pressure are identity rows, so the AMG hierarchy built for that
  // numbering keeps serving as the preconditioner (refreshed).  A cell that
  // melts outside the numbering, a larger frozen share, or the rebuild
  // policy renumbers.
  const char* rf = getenv("FVS_REFRESH_FRACTION");   // frozen share kept on one numbering
  const double frac = (rf && *rf) ? atof(rf) : 0.01;
  const int64_t dead_cap = std::max<int64_t>(64, (int64_t)(frac * (double)s->nact)) + s->nmargin;
  const bool renumber = !s->numbered || tc[2] > 0 || tc[3] > dead_cap || s->force_full;
  s->renumbered = false;
  if (renumber) FVS_TRY(renumber_lm(s));
  if (tc[1] != 0) s->k_valid = false;
  FVS_TRY(s->cnt.zero(st));
  FVS_TRY(s->flow.zero(st));
  k_faces_open<<<stride_grid(Nf, 256), 256, 0, st>>>(Nf, m->own, m->nei, s->lm, s->F, s->Fold, s->flow); FVS_COUNT_LAUNCH();
  k_ppe_cells<<<stride_grid(Nc, 256), 256, 0, st>>>(Nc, s->lm, s->flow, s->ppe); FVS_COUNT_LAUNCH();
  k_vertex_nonppe<<<stride_grid(Nv, 256), 256, 0, st>>>(Nv, m->vc_ptr, m->vc_idx, s->ppe, s->nS); FVS_COUNT_LAUNCH();
  k_face_case<<<stride_grid(Nf, 256), 256, 0, st>>>(Nf, m->own, m->nei, m->fv, s->lm, s->nS, s->fcase); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  k_count_u8<<<stride_grid(Nc, 256), 256, 0, st>>>(Nc, s->ppe, s->cnt); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  int hc[2];
  FVS_CUDA(cudaMemcpyAsync(hc, s->cnt.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  FVS_CUDA(cudaStreamSynchronize(st));
  s->nppe = hc[0];
  return FVS_OK;
}

static PpeCtx ppe_ctx(fvs_solver s) {
  fvs_mesh m = s->mesh;
  PpeCtx x;
  x.Nc = m->Nc; x.Nf = m->Nf; x.nact = s->nact; x.W = m->W; x.WF = m->WF;
  x.act = s->act; x.map = s->map; x.cf = m->cf; x.own = m->own; x.nei = m->nei; x.fv = m->fv;
  x.vc_ptr = m->vc_ptr; x.vc_idx = m->vc_idx; x.nb = m->nb; x.nnb = m->nnb; x.fnb = m->fnb; x.nfnb = m->nfnb;
  x.nS = s->nS; x.cfs = m->cfs; x.ppe = s->ppe; x.fcase = s->fcase;
  x.cd = m->cd; x.ce = m->ce; x.cz = m->cz; x.Pbval = m->Pb.val; x.Pbcol = m->Pb.col;
  x.rho = s->props.mat.rho;
  return x;
}

static fvs_status assemble_pressure(fvs_solver s) {
  fvs_mesh m = s->mesh;
  cudaStream_t st = s->stream;
  // phase times for FVS_DEBUG (waits for the stream at each mark)
  const bool dbg = getenv("FVS_DEBUG") != nullptr;
  if (dbg) cudaStreamSynchronize(st);
  auto t_mark = std::chrono::steady_clock::now();
  auto lap = [&]() {
    cudaStreamSynchronize(st);
    const auto now = std::chrono::steady_clock::now();
    const double ms = std::chrono::duration<double, std::milli>(now - t_mark).count();
    t_mark = now;
    return ms;
  };
  FVS_TRY(s->K.alloc(s->nact, m->W));
  DBuf<int> err;
  FVS_TRY(err.alloc(1));
  FVS_TRY(err.zero(st));
  if (s->nact > 0) {
    // one thread per row: the re-assembled rows next to solid cells are
    // latency-bound searches, so as many as possible run at once
    k_ppe_matrix<<<(unsigned)((s->nact + 127) / 128), 128, 0, st>>>(ppe_ctx(s), s->K.col, s->K.val, s->K.diag, err);
    FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
  }
  int h = 0;
  FVS_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  FVS_CUDA(cudaStreamSynchronize(st));
  if (h) {
    set_error("pressure assembly referenced a deleted column (flags 0x%x)", h);
    return FVS_ERR_STATE;
  }
  // AMG hierarchy for the new active set (Section 2.5); on failure the
  // solve falls back to single-grid Jacobi BiCGStab
  // Same numbering and a usable hierarchy: refresh its fine level only
  // (new diagonal, rows of frozen cells left out of the null-space
  // projection); otherwise build the hierarchy anew.
  const double t_matrix = dbg ? lap() : 0.0;
  // the preconditioner's operator: K itself, or its face-coupling part
  // (decided at each full setup; a refresh keeps the choice)
  auto fill_compact = [&]() -> fvs_status {
    FVS_TRY(s->Kp.alloc(s->nact, 7));
    k_ppe_compact<<<stride_grid(s->nact, 256), 256, 0, st>>>(s->nact, m->Nc, m->W, s->act, s->map, s->ppe, m->cf,
                                                              m->own, m->nei, s->K.col, s->K.val, s->Kp.col,
                                                              s->Kp.val, s->Kp.diag);
    FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    return FVS_OK;
  };
  if (!s->renumbered && s->amg_ok && !s->force_full && s->nact > 0) {
    if (s->pc_compact) FVS_TRY(fill_compact());
    const fvs_status r = s->amg.refresh(st, s->act, s->ppe);
    if (r == FVS_OK) {
      s->amg_full = false;
      if (dbg) fprintf(stderr, "[fvs step] pressure matrix %.2f ms, hierarchy refresh %.2f ms\n", t_matrix, lap());
      return FVS_OK;
    }
    if (r != FVS_ERR_NOT_CONVERGED) return r;
    if (dbg) fprintf(stderr, "[fvs step] refresh refused: %s\n", fvs_last_error());
    // the kept aggregation no longer fits: number the LM cells anew
    FVS_TRY(renumber_lm(s));
    return assemble_pressure(s);
  }
  if (!s->renumbered && s->nact > 0 && s->props.p_solver == FVS_PSOLVER_AMG) {
    // a full setup always starts from a numbering without frozen rows
    FVS_TRY(renumber_lm(s));
    return assemble_pressure(s);
  }
  s->amg_ok = false;
  s->amg_full = true;
  s->force_full = false;
  s->steps_since_setup = 0;
  if (s->props.p_solver == FVS_PSOLVER_AMG && s->nact > 0) {
    s->amg.opt.fp32 = s->props.precision == FVS_PREC_MIXED;
    // stop coarsening below a thousand rows: the dense inverse of that level
    // is one matrix-vector product per V-cycle, cheaper than the several
    // latency-bound launches per level that the small levels below it cost
    s->amg.opt.coarsest = SOLVER_COARSEST;
    // BiCGStab (non-orthogonal meshes) takes a V(1,2) cycle: the second
    // post-sweep saves more iterations than it costs (128^3 jittered cavity,
    // 20 steps: 429 -> 352 iterations, 49.4 -> 48.8 ms a step); CG keeps the
    // symmetric V(1,1)
    s->amg.opt.npost = m->orthogonal ? 1 : 2;
    // the vertex-interpolation couplings are small next to the face
    // couplings; leaving them out of the hierarchy cuts the bytes of every
    // V-cycle sweep (7 instead of 27 entries a fine row, narrower Galerkin
    // rows below) while the Krylov method keeps the full K
    const char* pc = getenv("FVS_PC_COMPACT");
    s->pc_compact = m->W > 7 && !(pc && *pc == '0');
    if (s->pc_compact) FVS_TRY(fill_compact());
    fvs_status r = s->amg.setup(st, s->pc_compact ? s->Kp : s->K);
    if (r == FVS_OK) {
      s->amg_ok = true;
      s->amg_levels = s->amg.levels();
      // liquid pockets: the singular parts (identity rows of cells without
      // pressure are parts of their own when the whole system is one level)
      s->ncomp = 0;
      for (uint8_t g : s->amg.sing_host) s->ncomp += g ? 1 : 0;
    } else if (r != FVS_ERR_NOT_CONVERGED) {
      return r;
    }
  }
  return FVS_OK;
}

// ---------------------------------------------------------------------------
// connected parts of the pressure system (single-grid solve)
// ---------------------------------------------------------------------------
// par[i] <= i always holds (roots hook onto smaller roots), so a walk up the
// parents ends at a root; the walk is bounded all the same
__device__ __forceinline__ int32_t cc_root(const int32_t* par, int32_t i) {
  for (int k = 0; k < (1 << 24); ++k) {
    const int32_t q = par[i];
    if (q == i || q < 0) return i;
    i = q;
  }
  return i;
}
__global__ void k_cc_init(int64_t n, const int32_t* act, const uint8_t* ppe, int32_t* par) {
  GS(i, n) par[i] = ppe[act[i]] ? (int32_t)i : -1;
}
// every stored coupling between two rows of the system joins their parts
__global__ void k_cc_hook(int64_t n, int w, const int32_t* col, const double* val, int32_t* par, int* changed) {
  GS(i, n) {
    if (par[i] < 0) continue;
    for (int k = 0; k < w; ++k) {
      const int32_t j = col[(int64_t)k * n + i];
      if (j == (int32_t)i || val[(int64_t)k * n + i] == 0.0 || par[j] < 0) continue;
      const int32_t a = cc_root(par, (int32_t)i), b = cc_root(par, j);
      if (a == b) continue;
      atomicMin(&par[a > b ? a : b], a > b ? b : a);
      *changed = 1;
    }
  }
}
__global__ void k_cc_compress(int64_t n, int32_t* par, int32_t* is_root) {
  GS(i, n) {
    const int32_t r = par[i] < 0 ? -1 : cc_root(par, (int32_t)i);
    if (r >= 0) par[i] = r;
    is_root[i] = (r == (int32_t)i) ? 1 : 0;
  }
}
__global__ void k_cc_label(int64_t n, const int32_t* par, const int32_t* rid, int32_t* lab, double* cnt) {
  GS(i, n) {
    const int32_t r = par[i];
    const int32_t c = r < 0 ? -1 : rid[r];
    lab[i] = c;
    if (c >= 0) atomicAdd(&cnt[c], 1.0);
  }
}
__global__ void k_part_sum(int64_t n, const int32_t* lab, const double* v, double* sum) {
  GS(i, n) if (lab[i] >= 0) atomicAdd(&sum[lab[i]], v[i]);
}
__global__ void k_part_sub(int64_t n, const int32_t* lab, const double* sum, const double* cnt, double* v) {
  GS(i, n) {
    const int32_t c = lab[i];
    if (c >= 0) v[i] -= sum[c] / cnt[c];
  }
}

fvs_status PartProjector::setup(cudaStream_t s, const Ell& K, const int32_t* act, const uint8_t* ppe,
                                ScanWork& sw) {
  const int64_t n = K.n;
  ncomp = 0;
  if (n == 0) return FVS_OK;
  FVS_TRY(par.alloc(n + 1)); FVS_TRY(root_flag.alloc(n + 1)); FVS_TRY(root_id.alloc(n + 1));
  FVS_TRY(lab.alloc(n + 1)); FVS_TRY(changed.alloc(1));
  const int g = stride_grid(n, 256);
  k_cc_init<<<g, 256, 0, s>>>(n, act, ppe, par); FVS_COUNT_LAUNCH();
  int done = 0;
  for (int it = 0; it < 200; ++it) {
    FVS_TRY(changed.zero(s));
    k_cc_hook<<<g, 256, 0, s>>>(n, K.w, K.col, K.val, par, changed); FVS_COUNT_LAUNCH();
    k_cc_compress<<<g, 256, 0, s>>>(n, par, root_flag); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    int h = 1;
    FVS_CUDA(cudaMemcpyAsync(&h, changed.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    FVS_CUDA(cudaStreamSynchronize(s));
    if (!h) {
      done = 1;
      break;
    }
  }
  if (!done) {
    set_error("pressure system parts: labels did not settle");
    return FVS_ERR_NOT_CONVERGED;
  }
  FVS_TRY(exclusive_scan(s, sw, n, root_flag, root_id));
  FVS_CUDA(cudaMemcpyAsync(&ncomp, sw.total.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  FVS_CUDA(cudaStreamSynchronize(s));
  FVS_TRY(cnt.alloc(ncomp + 1)); FVS_TRY(sum.alloc(ncomp + 1));
  FVS_TRY(cnt.zero(s));
  k_cc_label<<<g, 256, 0, s>>>(n, par, root_id, lab, cnt); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

fvs_status PartProjector::apply(cudaStream_t s, double* v) {
  const int64_t n = lab.n ? (int64_t)lab.n - 1 : 0;
  if (ncomp == 0 || n == 0) return FVS_OK;
  FVS_TRY(sum.zero(s));
  k_part_sum<<<stride_grid(n, 256), 256, 0, s>>>(n, lab, v, sum); FVS_COUNT_LAUNCH();
  k_part_sub<<<stride_grid(n, 256), 256, 0, s>>>(n, lab, sum, cnt, v); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

// solve K x = rhs (compact) with the configured method; fills stats
static fvs_status solve_pressure(fvs_solver s, double rtol, SolveResult& res, int& fallback) {
  cudaStream_t st = s->stream;
  fallback = 0;
  const int maxit = s->props.max_krylov_iters;
  // on a refreshed hierarchy a slow solve means it has gone stale (e.g. a
  // liquid pocket split by freezing cells): stop early and let the caller
  // rebuild it rather than fall back to single-grid Jacobi
  const bool refreshed = s->amg_ok && !s->amg_full && s->p_its_ref > 0;
  if (refreshed) {
    const int cap = std::min(maxit, std::max(s->p_its_ref * 2, s->p_its_ref + 12));
    if (s->mesh->orthogonal)
      FVS_TRY(pcg(st, s->red, s->kw, s->K, s->amg, s->prhs, s->px, rtol, cap, &s->aproj, res, &s->g_p));
    else
      FVS_TRY(bicgstab(st, s->red, s->kw, s->K, nullptr, s->amg, s->prhs, s->px, rtol, cap, &s->aproj, res, 0.0,
                       &s->g_p));
    if (res.converged) FVS_TRY(s->amg.project(st, s->px));
    return FVS_OK;
  }
  if (s->amg_ok) {
    if (s->mesh->orthogonal)
      FVS_TRY(pcg(st, s->red, s->kw, s->K, s->amg, s->prhs, s->px, rtol, maxit, &s->aproj, res, &s->g_p));
    else
      FVS_TRY(bicgstab(st, s->red, s->kw, s->K, nullptr, s->amg, s->prhs, s->px, rtol, maxit, &s->aproj, res, 0.0,
                       &s->g_p));
    if (res.converged) {
      FVS_TRY(s->amg.project(st, s->px));
      return FVS_OK;
    }
  }
  // single-grid Jacobi BiCGStab: the configured solver, or the fallback of
  // a failed AMG solve (Section 2.5); the null space of every connected
  // part (liquid pocket) is projected out with labels of its own
  fallback = s->props.p_solver == FVS_PSOLVER_AMG ? 1 : 0;
  JacobiPrecond J;
  J.A = &s->K;
  FVS_TRY(s->pparts.setup(st, s->K, s->act, s->ppe, s->sw));
  FVS_TRY(bicgstab(st, s->red, s->kw, s->K, nullptr, J, s->prhs, s->px, rtol, fallback ? maxit * 4 : maxit,
                   &s->pparts, res));
  FVS_TRY(s->pparts.apply(st, s->px));
  return FVS_OK;
}

fvs_status solver_step(fvs_solver s, double dt, fvs_step_stats* stats) {
  if (!s->have_props) {
    set_error("fvs_set_properties must come first");
    return FVS_ERR_STATE;
  }
  if (!(dt > 0)) {
    set_error("dt must be positive");
    return FVS_ERR_ARG;
  }
  fvs_mesh m = s->mesh;
  cudaStream_t st = s->stream;
  const int64_t Nc = m->Nc, Nf = m->Nf, Nv = m->Nv;
  const Mat mt = mat_of(s->props);
  fvs_step_stats S{};
  fvs_status status = FVS_OK;

  // 1. tags, compaction, face cases
  FVS_TRY(classify(s));
  int64_t na = s->nact;
  S.n_active = s->nlm;

  // natural convection off: velocity, fluxes and pressure stay zero (they
  // were zeroed with the state), only the energy equation runs
  const bool flow_on = !s->props.no_flow;
  if (!flow_on) {
    na = 0;
    FVS_TRY(s->u.zero(st));       // a velocity given to fvs_set_state does not move anything
    FVS_TRY(s->uold.zero(st));
  }

  // 2. momentum predictor
  FVS_TRY(s->M.alloc(na, m->W));
  FVS_TRY(s->mrhs.alloc(3 * na + 1));
  FVS_TRY(s->mx.alloc(3 * na + 1));
  if (na > 0) {
    k_mom_matrix<<<stride_grid(na, 256), 256, 0, st>>>(na, Nc, m->W, s->act, s->map, s->lm, m->Lu.col, m->Lu.val,
                                                       m->V, s->fs, mt, dt, s->M.col, s->M.val, s->M.diag);
    FVS_COUNT_LAUNCH();
    k_mom_rhs<<<stride_grid(na, 256), 256, 0, st>>>(na, Nc, m->W, s->act, s->lm, m->cf, m->cfs, m->own, m->nei, s->F,
                                                    s->Fold, s->u, s->uold, m->Lu.col, m->Lu.val, m->V, s->T, mt, dt,
                                                    s->mrhs, s->mx); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    FVS_TRY(s->jinv_m.alloc(na));
    k_inverse<<<stride_grid(na, 256), 256, 0, st>>>(na, s->M.diag, s->jinv_m); FVS_COUNT_LAUNCH();
    JacobiPrecond J;
    J.A = &s->M;
    J.dinv = s->jinv_m;
    // the three components are judged against the largest right side (a
    // component with a near-zero right side would otherwise chase roundoff)
    double bmax = 0.0;
    for (int d = 0; d < 3; ++d) {
      FVS_TRY(s->red.dot(st, na, s->mrhs.p + d * na, s->mrhs.p + d * na, S_TMP0 + (d == 2 ? 0 : d)));
      FVS_TRY(s->red.fetch(st));
      bmax = std::max(bmax, sqrt(s->red.host[S_TMP0 + (d == 2 ? 0 : d)]));
    }
    for (int d = 0; d < 3; ++d) {
      SolveResult r;
      FVS_TRY(bicgstab(st, s->red, s->kw, s->M, nullptr, J, s->mrhs.p + d * na, s->mx.p + d * na,
                       s->props.mom_rtol, s->props.max_krylov_iters, nullptr, r, bmax, &s->g_m[d]));
      S.mom_its += r.iters;
      if (!r.converged) {
        status = FVS_ERR_NOT_CONVERGED;
        set_error("momentum component %d: relative residual %.3e after %d iterations", d, r.relres, r.iters);
      }
    }
  }
  if (flow_on) {
  k_scatter3<<<stride_grid(Nc, 256), 256, 0, st>>>(Nc, na, s->map, s->lm, s->mx, s->ustar); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();

  // 3. pressure system
  if (!s->k_valid) {
    const auto t0 = std::chrono::steady_clock::now();
    FVS_TRY(assemble_pressure(s));
    FVS_CUDA(cudaStreamSynchronize(st));
    S.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    s->k_valid = true;
    S.p_rebuilt = s->amg_full ? 1 : 2;
    na = s->nact;   // a failed refresh renumbers
  }
  FVS_TRY(s->prhs.alloc(na + 1));
  FVS_TRY(s->px.alloc(na + 1));
  if (na > 0) {
    k_ppe_rhs<<<stride_grid(na, 256), 256, 0, st>>>(na, Nc, Nf, s->act, s->ppe, m->cf, m->cfs, s->fcase, m->own,
                                                    m->nei, m->A, m->nrm, s->ustar, dt, s->p, s->prhs, s->px); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    SolveResult r;
    int fb = 0;
    FVS_TRY(solve_pressure(s, s->props.p_rtol, r, fb));
    // a refreshed hierarchy that has gone stale: rebuild it for the next step
    // when the solve was slow, at once (and solve again) when it failed
    if (!s->amg_full && s->amg_ok && r.converged &&
        r.iters > std::max(s->p_its_ref * 3 / 2, s->p_its_ref + 6))
      s->force_full = true;
    if (getenv("FVS_DEBUG") && !s->amg_full && s->amg_ok && (!r.converged || s->force_full))
      fprintf(stderr, "[fvs step] refreshed solve %s: %d iterations (reference %d)\n",
              r.converged ? "slow" : "stalled", r.iters, s->p_its_ref);
    if (!s->amg_full && s->amg_ok && !r.converged) {
      const auto t0 = std::chrono::steady_clock::now();
      FVS_TRY(renumber_lm(s));
      s->force_full = true;
      FVS_TRY(assemble_pressure(s));
      FVS_CUDA(cudaStreamSynchronize(st));
      S.setup_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      S.p_rebuilt = 1;
      const int64_t nb = s->nact;
      FVS_TRY(s->prhs.alloc(nb + 1));
      FVS_TRY(s->px.alloc(nb + 1));
      k_ppe_rhs<<<stride_grid(nb, 256), 256, 0, st>>>(nb, Nc, Nf, s->act, s->ppe, m->cf, m->cfs, s->fcase, m->own,
                                                      m->nei, m->A, m->nrm, s->ustar, dt, s->p, s->prhs, s->px);
      FVS_COUNT_LAUNCH();
      FVS_LAUNCH_CHECK();
      const int first_its = r.iters;
      FVS_TRY(solve_pressure(s, s->props.p_rtol, r, fb));
      if (s->amg_full) s->p_its_ref = r.iters;
      r.iters += first_its;
    } else if (s->amg_full) {
      s->p_its_ref = r.iters;
    }
    // periodic renumbering and rebuild after a run of refreshes
    if (S.p_rebuilt == 2 && ++s->steps_since_setup >= 25) s->force_full = true;
    S.p_its = r.iters;
    S.p_relres = r.relres;
    S.fallback = fb;
    if (!r.converged) {
      status = FVS_ERR_NOT_CONVERGED;
      set_error("pressure: relative residual %.3e after %d iterations (fallback %d)", r.relres, r.iters, fb);
    }
  }
  k_scatter1<<<stride_grid(Nc, 256), 256, 0, st>>>(Nc, s->map, s->ppe, s->px, s->p); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();

  // 4. correction
  k_vertex_p<<<stride_grid(Nv, 256), 256, 0, st>>>(Nv, m->vc_ptr, m->vc_idx, s->ppe, s->p, s->nS, s->pv, s->fSv); FVS_COUNT_LAUNCH();
  k_face_correct<<<stride_grid(Nf, 256), 256, 0, st>>>(Nf, Nc, m->own, m->nei, m->fv, s->fcase, m->fnb, m->nfnb,
                                                       s->ppe, s->p, s->pv, s->fSv, m->A, m->nrm, m->cd, m->ce,
                                                       m->cz, m->Jinv, s->ustar, dt, mt.rho, s->Fnew, s->gradf); FVS_COUNT_LAUNCH();
  k_cell_correct<<<stride_grid(Nc, 256), 256, 0, st>>>(Nc, Nf, s->lm, m->cf, s->fcase, s->gradf, s->ustar, dt,
                                                       mt.rho, s->unew); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  }   // flow_on

  // conductivities of T^n when k depends on T (both Crank-Nicolson halves)
  if (s->n_k > 0) FVS_TRY(conduction_operator(s));

  // 5. energy: linearised latent heat, inner solve, enthalpy inversion
  k_energy_base<<<stride_grid(Nc, 256), 256, 0, st>>>(Nc, m->W, m->cf, m->cfs, m->own, m->nei, s->F, s->Fold, s->T,
                                                      s->Told, s->LT.col, s->LT.val, s->lT, m->V, s->rcp, dt, s->ebase); FVS_COUNT_LAUNCH();
  k_energy_guess<<<stride_grid(Nc, 256), 256, 0, st>>>(Nc, s->T, s->Told, mt.law, s->Tnew, s->fsnew, s->metal);
  FVS_COUNT_LAUNCH();
  {
    FVS_TRY(s->jinv_e.alloc(Nc));
    JacobiPrecond J;
    J.A = &s->Ke;
    J.dextra = s->edx;
    J.dinv = s->jinv_e;
    const char* el = getenv("FVS_ENERGY_LINES");
    const bool lines = el && *el == '1';
    if (lines && (!s->eline.ready || s->eline.built_from != s->Ke.col.p || s->eline.n != s->Ke.n ||
                  s->eline.w != s->Ke.w))
      FVS_TRY(s->eline.build(st, s->Ke));
    s->eline.dextra = s->edx;
    Precond& PE = lines ? static_cast<Precond&>(s->eline) : static_cast<Precond&>(J);
    // Tnew / fsnew hold the iterate m; Tlin the linear solution
    DBuf<double>& Tm = s->Tnew;
    DBuf<double>& fsm = s->fsnew;
    int it = 0;
    bool conv = false;
    double dT_prev = 1e300;
    for (it = 1; it <= s->props.max_e_iters; ++it) {
      // inexact inner solves: early passes only need to resolve a fraction
      // of the nonlinear change; the last passes reach e_rtol
      const double rtol_m = std::max(s->props.e_rtol, std::min(1e-4, 1e-5 * dT_prev));
      k_energy_lin<<<stride_grid(Nc, 256), 256, 0, st>>>(Nc, m->V, mt, dt, Tm, fsm, s->fs, s->ebase, s->edx,
                                                          s->erhs, s->Tlin, s->rcp, s->rL, s->metal, s->Ke.diag,
                                                          s->jinv_e);
      FVS_COUNT_LAUNCH();
      FVS_LAUNCH_CHECK();
      if (lines) FVS_TRY(s->eline.factor(st));
      SolveResult r;
      FVS_TRY(bicgstab(st, s->red, s->kw, s->Ke, s->edx, PE, s->erhs, s->Tlin, rtol_m,
                       s->props.max_krylov_iters, nullptr, r, 0.0, &s->g_e));
      S.e_lin_its += r.iters;
      if (!r.converged) {
        status = FVS_ERR_NOT_CONVERGED;
        set_error("energy pass %d: relative residual %.3e after %d iterations", it, r.relres, r.iters);
      }
      // next iterate, then its change against the current one
      k_energy_update<<<stride_grid(Nc, 256), 256, 0, st>>>(Nc, mt, s->Tlin, Tm, fsm, s->Tit, s->fsit, s->metal);
      FVS_COUNT_LAUNCH();
      FVS_LAUNCH_CHECK();
      FVS_TRY(s->red.max_abs_diff2(st, Nc, s->Tit, Tm, s->fsit, fsm, S_TMP0, S_TMP1));
      dswap(s->Tit, Tm);
      dswap(s->fsit, fsm);
      FVS_TRY(s->red.fetch(st));
      if (s->red.host[S_TMP0] <= s->props.e_tol_T && s->red.host[S_TMP1] <= 1e-12 && rtol_m <= s->props.e_rtol) {
        conv = true;
        break;
      }
      dT_prev = s->red.host[S_TMP0];
    }
    S.e_its = std::min(it, s->props.max_e_iters);
    if (!conv) {
      status = FVS_ERR_NOT_CONVERGED;
      set_error("latent-heat loop: max|dT| %.3e after %d passes", s->red.host[S_TMP0], S.e_its);
    }
  }

  // 6. crossing times, then rotate the time levels
  k_crossings<<<stride_grid(Nc, 256), 256, 0, st>>>(Nc, s->T, s->Tnew, mt.Ts, mt.Tl, s->time, dt, s->tliq, s->tsol,
                                                    s->metal);
  FVS_COUNT_LAUNCH();
  if (s->grain_on) {
    k_grain<<<stride_grid(Nc, 256), 256, 0, st>>>(Nc, s->fs, s->fsnew, s->metal, s->grain_kp, s->grain_Ds, dt,
                                                  s->r2);
    FVS_COUNT_LAUNCH();
  }
  FVS_LAUNCH_CHECK();
  dswap(s->Told, s->T);     // Told <- T^n
  dswap(s->T, s->Tnew);     // T <- T^{n+1}
  dswap(s->fs, s->fsnew);
  if (flow_on) {
    dswap(s->uold, s->u);     // uold <- u^n
    dswap(s->u, s->unew);     // u <- u^{n+1}
    dswap(s->Fold, s->F);     // Fold <- F^n
    dswap(s->F, s->Fnew);     // F <- F^{n+1}
  }
  FVS_CUDA(cudaStreamSynchronize(st));
  s->time += dt;
  s->nstep += 1;
  s->have_step = true;

  S.n_ppe = s->nppe;
  S.n_components = s->amg_ok ? s->ncomp : (s->pparts.ncomp > 0 ? s->pparts.ncomp : -1);
  S.amg_levels = s->amg_ok ? s->amg_levels : 0;
  S.status = status;
  s->last = S;
  if (stats) *stats = S;
  return status;
}

fvs_status solver_pressure_solve(fvs_solver s, const double* rhs, double* p_out, double rtol, int* iters,
                                 double* relres) {
  if (!s->have_step) {
    set_error("fvs_pressure_solve needs the active set of a completed step");
    return FVS_ERR_STATE;
  }
  fvs_mesh m = s->mesh;
  cudaStream_t st = s->stream;
  FVS_TRY(s->prhs.alloc(s->nact + 1));
  FVS_TRY(s->px.alloc(s->nact + 1));
  if (s->nact > 0) {
    k_rhs_in<<<stride_grid(s->nact, 256), 256, 0, st>>>(s->nact, s->act, s->ppe, m->cell_in, rhs, s->prhs, s->px); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    // a NaN or infinity in the right side is the caller's error: refuse it
    // before any iteration runs
    FVS_TRY(s->red.dot(st, s->nact, s->prhs, s->prhs, S_TMP0));
    FVS_TRY(s->red.fetch(st));
    const double bb = s->red.host[S_TMP0];
    if (!(bb == bb) || bb > 1.7e308) {
      set_error("fvs_pressure_solve: the right side holds a non-finite value");
      return FVS_ERR_ARG;
    }
  }
  SolveResult r;
  int fb = 0;
  FVS_TRY(solve_pressure(s, rtol, r, fb));
  k_p_out<<<stride_grid(m->Nc, 256), 256, 0, st>>>(m->Nc, s->map, s->ppe, m->cell_in, s->px, p_out); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  FVS_CUDA(cudaStreamSynchronize(st));
  if (iters) *iters = r.iters;
  if (relres) *relres = r.relres;
  return r.converged ? FVS_OK : FVS_ERR_NOT_CONVERGED;
}

fvs_status solver_query(fvs_solver s, fvs_field f, double* dst, int64_t len, int on_device) {
  fvs_mesh m = s->mesh;
  cudaStream_t st = s->stream;
  const int64_t Nc = m->Nc, Nf = m->Nf;
  int64_t need = 0;
  switch (f) {
    case FVS_T: case FVS_FS: case FVS_P: case FVS_TAG: case FVS_GRAIN: need = Nc; break;
    case FVS_U: case FVS_USTAR: need = 3 * Nc; break;
    case FVS_QOI: need = 4 * Nc; break;
    case FVS_CROSS: need = 2 * Nc; break;
    case FVS_FLUX: case FVS_FACE_CASE: need = Nf; break;
    default: set_error("unknown field %d", (int)f); return FVS_ERR_ARG;
  }
  if (len < need) {
    set_error("destination holds %lld values, field needs %lld", (long long)len, (long long)need);
    return FVS_ERR_ARG;
  }
  DBuf<double> tmp;
  double* out = dst;
  if (!on_device) {
    FVS_TRY(tmp.alloc(need));
    out = tmp.p;
  }
  const int gc = stride_grid(Nc, 256), gf = stride_grid(Nf, 256);
  const Mat mt = mat_of(s->props);
  switch (f) {
    case FVS_T: k_gather_out<<<gc, 256, 0, st>>>(Nc, 1, m->cell_in, s->T, out); break;
    case FVS_FS: k_gather_out<<<gc, 256, 0, st>>>(Nc, 1, m->cell_in, s->fs, out); break;
    case FVS_P: k_gather_out<<<gc, 256, 0, st>>>(Nc, 1, m->cell_in, s->p, out); break;
    case FVS_U: k_gather_out<<<gc, 256, 0, st>>>(Nc, 3, m->cell_in, s->u, out); break;
    case FVS_USTAR: k_gather_out<<<gc, 256, 0, st>>>(Nc, 3, m->cell_in, s->ustar, out); break;
    case FVS_FLUX: k_gather_out<<<gf, 256, 0, st>>>(Nf, 1, m->face_in, s->F, out); break;
    case FVS_TAG: k_gather_u8<<<gc, 256, 0, st>>>(Nc, m->cell_in, s->lm, out); break;
    case FVS_FACE_CASE: k_gather_u8<<<gf, 256, 0, st>>>(Nf, m->face_in, s->fcase, out); break;
    case FVS_QOI: k_qoi<<<gc, 256, 0, st>>>(Nc, m->cell_in, s->tliq, s->tsol, mt.Ts, mt.Tl, out); break;
    case FVS_GRAIN: k_sqrt_out<<<gc, 256, 0, st>>>(Nc, m->cell_in, s->r2, out); break;
    case FVS_CROSS: {
      DBuf<double> both;
      FVS_TRY(both.alloc(2 * Nc));
      FVS_CUDA(cudaMemcpyAsync(both.p, s->tliq.p, Nc * sizeof(double), cudaMemcpyDeviceToDevice, st));
      FVS_CUDA(cudaMemcpyAsync(both.p + Nc, s->tsol.p, Nc * sizeof(double), cudaMemcpyDeviceToDevice, st));
      k_gather_out<<<gc, 256, 0, st>>>(Nc, 2, m->cell_in, both, out); FVS_COUNT_LAUNCH();
      FVS_LAUNCH_CHECK();
      FVS_CUDA(cudaStreamSynchronize(st));
      break;
    }
    default: break;
  }
  if (f != FVS_CROSS) FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  if (!on_device) FVS_CUDA(cudaMemcpyAsync(dst, out, need * sizeof(double), cudaMemcpyDeviceToHost, st));
  FVS_CUDA(cudaStreamSynchronize(st));
  return FVS_OK;
}

}  // namespace fvs
