// Mesh ingest, renumbering, connectivity, geometry and base operators
// (Section 2.3: collocated finite volumes on unstructured hexahedra; Eq. 11
// splits the face normal derivative into direct and cross terms, Eq. 12
// gives the face gradient from the local frame C1C2 / V1V3 / V2V4 with
// vertex values averaged from the surrounding cells).
#include <cub/cub.cuh>

#include "mesh.cuh"
#include "scan.cuh"

namespace fvs {

#define GS(i, n) for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

enum { MERR_RANGE = 1, MERR_FACECOUNT = 2, MERR_VALENCE = 4, MERR_NB = 8, MERR_GEOM = 16, MERR_OWNER = 32 };

// ---------------------------------------------------------------------------
// validation and renumbering
// ---------------------------------------------------------------------------
__global__ void k_validate(int64_t Nv, int64_t Nc, int64_t Nf, const int32_t* cells, const int32_t* faces,
                           const int32_t* fcells, const int32_t* patch, int* err) {
  GS(i, Nc) {
    for (int k = 0; k < 8; ++k) {
      const int32_t v = cells[i * 8 + k];
      if (v < 0 || v >= Nv) atomicOr(err, MERR_RANGE);
    }
  }
  GS(f, Nf) {
    for (int k = 0; k < 4; ++k) {
      const int32_t v = faces[f * 4 + k];
      if (v < 0 || v >= Nv) atomicOr(err, MERR_RANGE);
    }
    const int32_t o = fcells[2 * f], q = fcells[2 * f + 1];
    if (o < 0 || o >= Nc || q >= Nc || q < -1) atomicOr(err, MERR_RANGE);
    if (o == q) atomicOr(err, MERR_OWNER);
    if (q < 0 && (patch[f] < 0 || patch[f] > 63)) atomicOr(err, MERR_RANGE);
  }
}

__global__ void k_bbox_part(int64_t Nv, const double* X, double* part) {
  __shared__ double sh[32];
  double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
  GS(i, Nv) {
    for (int d = 0; d < 3; ++d) {
      mn[d] = fmin(mn[d], X[3 * i + d]);
      mx[d] = fmax(mx[d], X[3 * i + d]);
    }
  }
  for (int d = 0; d < 3; ++d) {
    const double a = -block_max(-mn[d], sh);
    const double b = block_max(mx[d], sh);
    if (threadIdx.x == 0) {
      part[6 * blockIdx.x + d] = a;
      part[6 * blockIdx.x + 3 + d] = b;
    }
  }
}

__global__ void k_bbox_final(int nb, double* part) {
  if (threadIdx.x == 0) {
    for (int b = 1; b < nb; ++b)
      for (int d = 0; d < 3; ++d) {
        part[d] = fmin(part[d], part[6 * b + d]);
        part[3 + d] = fmax(part[3 + d], part[6 * b + 3 + d]);
      }
  }
}

__device__ __forceinline__ uint64_t spread21(uint64_t x) {
  x &= 0x1fffffULL;
  x = (x | (x << 32)) & 0x1f00000000ffffULL;
  x = (x | (x << 16)) & 0x1f0000ff0000ffULL;
  x = (x | (x << 8)) & 0x100f00f00f00f00fULL;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ULL;
  x = (x | (x << 2)) & 0x1249249249249249ULL;
  return x;
}
__device__ __forceinline__ uint64_t morton(const double* bb, double x, double y, double z) {
  const double s = 2097151.0;
  double p[3] = {x, y, z};
  uint64_t q[3];
  for (int d = 0; d < 3; ++d) {
    const double ext = bb[3 + d] - bb[d];
    double t = ext > 0 ? (p[d] - bb[d]) / ext : 0.0;
    t = fmin(fmax(t, 0.0), 1.0);
    q[d] = (uint64_t)(t * s);
  }
  return spread21(q[0]) | (spread21(q[1]) << 1) | (spread21(q[2]) << 2);
}

__global__ void k_cell_keys(int64_t Nc, const double* X, const int32_t* cells, const double* bb, int reorder,
                            uint64_t* key, int32_t* val) {
  GS(c, Nc) {
    double x = 0, y = 0, z = 0;
    for (int k = 0; k < 8; ++k) {
      const int32_t v = cells[c * 8 + k];
      x += X[3 * v]; y += X[3 * v + 1]; z += X[3 * v + 2];
    }
    key[c] = reorder ? morton(bb, x / 8, y / 8, z / 8) : (uint64_t)c;
    val[c] = (int32_t)c;
  }
}
__global__ void k_node_keys(int64_t Nv, const double* X, const double* bb, int reorder, uint64_t* key, int32_t* val) {
  GS(v, Nv) {
    key[v] = reorder ? morton(bb, X[3 * v], X[3 * v + 1], X[3 * v + 2]) : (uint64_t)v;
    val[v] = (int32_t)v;
  }
}
__global__ void k_invert(int64_t n, const int32_t* fwd, int32_t* inv) {
  GS(i, n) inv[fwd[i]] = (int32_t)i;
}
__global__ void k_face_keys(int64_t Nf, const int32_t* fcells, const int32_t* cell_new, int reorder,
                            uint64_t* key, int32_t* val) {
  GS(f, Nf) {
    key[f] = reorder ? (((uint64_t)cell_new[fcells[2 * f]]) << 32) | (uint64_t)f : (uint64_t)f;
    val[f] = (int32_t)f;
  }
}

// gather into new numbering
__global__ void k_gather_nodes(int64_t Nv, const double* X, const int32_t* node_in, double* Xn) {
  GS(v, Nv) {
    const int32_t o = node_in[v];
    Xn[v] = X[3 * o];
    Xn[Nv + v] = X[3 * o + 1];
    Xn[2 * Nv + v] = X[3 * o + 2];
  }
}
__global__ void k_gather_cells(int64_t Nc, const int32_t* cells, const int32_t* cell_in, const int32_t* node_new,
                               int32_t* cn) {
  GS(c, Nc) {
    const int32_t o = cell_in[c];
    for (int k = 0; k < 8; ++k) cn[k * Nc + c] = node_new[cells[o * 8 + k]];
  }
}
__global__ void k_gather_faces(int64_t Nf, const int32_t* faces, const int32_t* fcells, const int32_t* patch,
                               const int32_t* face_in, const int32_t* node_new, const int32_t* cell_new,
                               int32_t* fv, int32_t* own, int32_t* nei, int32_t* pat) {
  GS(f, Nf) {
    const int32_t o = face_in[f];
    for (int k = 0; k < 4; ++k) fv[k * Nf + f] = node_new[faces[o * 4 + k]];
    own[f] = cell_new[fcells[2 * o]];
    const int32_t q = fcells[2 * o + 1];
    nei[f] = q >= 0 ? cell_new[q] : -1;
    pat[f] = q >= 0 ? -1 : patch[o];
  }
}

// ---------------------------------------------------------------------------
// connectivity
// ---------------------------------------------------------------------------
__global__ void k_cell_faces(int64_t Nf, int64_t Nc, const int32_t* own, const int32_t* nei, int32_t* cnt,
                             int32_t* cf, int8_t* cfs, int* err) {
  GS(f, Nf) {
    const int32_t o = own[f];
    int s = atomicAdd(&cnt[o], 1);
    if (s < 6) { cf[s * Nc + o] = (int32_t)f; cfs[s * Nc + o] = 1; } else atomicOr(err, MERR_FACECOUNT);
    const int32_t q = nei[f];
    if (q >= 0) {
      s = atomicAdd(&cnt[q], 1);
      if (s < 6) { cf[s * Nc + q] = (int32_t)f; cfs[s * Nc + q] = -1; } else atomicOr(err, MERR_FACECOUNT);
    }
  }
}
__global__ void k_cell_faces_sort(int64_t Nc, const int32_t* cnt, int32_t* cf, int8_t* cfs, int* err) {
  GS(c, Nc) {
    if (cnt[c] != 6) { atomicOr(err, MERR_FACECOUNT); continue; }
    int32_t a[6]; int8_t b[6];
    for (int k = 0; k < 6; ++k) { a[k] = cf[k * Nc + c]; b[k] = cfs[k * Nc + c]; }
    for (int i = 1; i < 6; ++i)
      for (int j = i; j > 0 && a[j - 1] > a[j]; --j) {
        int32_t t = a[j]; a[j] = a[j - 1]; a[j - 1] = t;
        int8_t u = b[j]; b[j] = b[j - 1]; b[j - 1] = u;
      }
    for (int k = 0; k < 6; ++k) { cf[k * Nc + c] = a[k]; cfs[k * Nc + c] = b[k]; }
  }
}

__global__ void k_vertex_count(int64_t Nc, const int32_t* cn, int32_t* cnt) {
  GS(c, Nc) for (int k = 0; k < 8; ++k) atomicAdd(&cnt[cn[k * Nc + c]], 1);
}
__global__ void k_vertex_fill(int64_t Nc, const int32_t* cn, const int32_t* ptr, int32_t* cur, int32_t* idx) {
  GS(c, Nc) for (int k = 0; k < 8; ++k) {
    const int32_t v = cn[k * Nc + c];
    const int32_t s = atomicAdd(&cur[v], 1);
    idx[ptr[v] + s] = (int32_t)c;
  }
}
__global__ void k_vertex_sort(int64_t Nv, const int32_t* ptr, int32_t* idx, int* err) {
  GS(v, Nv) {
    const int32_t lo = ptr[v], hi = ptr[v + 1];
    if (hi - lo > FVS_MAX_VCELLS || hi - lo < 1) atomicOr(err, MERR_VALENCE);
    for (int32_t i = lo + 1; i < hi; ++i)
      for (int32_t j = i; j > lo && idx[j - 1] > idx[j]; --j) {
        const int32_t t = idx[j]; idx[j] = idx[j - 1]; idx[j - 1] = t;
      }
  }
}
__global__ void k_vertex_boundary(int64_t Nf, const int32_t* fv, const int32_t* nei, uint8_t* vb) {
  GS(f, Nf) if (nei[f] < 0) for (int k = 0; k < 4; ++k) vb[fv[k * Nf + f]] = 1;
}

// sorted unique union of the cell lists of nvert vertices; returns the count
// (or -1 if it would exceed cap).  buf must hold nvert*FVS_MAX_VCELLS.
__device__ int union_cells(const int32_t* verts, int nvert, const int32_t* ptr, const int32_t* idx,
                           int32_t* buf, int cap) {
  int n = 0;
  for (int a = 0; a < nvert; ++a) {
    const int32_t v = verts[a];
    for (int32_t e = ptr[v]; e < ptr[v + 1]; ++e) {
      const int32_t c = idx[e];
      // insert keeping buf sorted and unique
      int pos = n;
      while (pos > 0 && buf[pos - 1] > c) --pos;
      if (pos > 0 && buf[pos - 1] == c) continue;
      if (n >= cap) return -1;
      for (int j = n; j > pos; --j) buf[j] = buf[j - 1];
      buf[pos] = c;
      ++n;
    }
  }
  return n;
}

__global__ void k_cell_nb(int64_t Nc, const int32_t* cn, const int32_t* ptr, const int32_t* idx, int W,
                          int32_t* nb, int32_t* nnb, int* err) {
  int32_t buf[FVS_MAX_NB];
  GS(c, Nc) {
    int32_t vs[8];
    for (int k = 0; k < 8; ++k) vs[k] = cn[k * Nc + c];
    const int n = union_cells(vs, 8, ptr, idx, buf, FVS_MAX_NB);
    if (n < 0) { atomicOr(err, MERR_NB); nnb[c] = 0; continue; }
    nnb[c] = n;
    if (nb) for (int k = 0; k < W; ++k) nb[k * Nc + c] = k < n ? buf[k] : buf[0];
  }
}
// face-neighbour stencil of an orthogonal mesh: the cell and the cells across
// its faces, sorted (every cross-diffusion weight is zero there, so no
// coefficient reaches a cell that shares only an edge or a vertex)
__global__ void k_cell_nb_faces(int64_t Nc, const int32_t* cf, const int32_t* own, const int32_t* nei, int W,
                                int32_t* nb, int32_t* nnb) {
  GS(c, Nc) {
    int32_t buf[7];
    int n = 1;
    buf[0] = (int32_t)c;
    for (int s = 0; s < 6; ++s) {
      const int32_t f = cf[s * Nc + c];
      const int32_t o = own[f], q = nei[f];
      const int32_t j = o == (int32_t)c ? q : o;
      if (j < 0) continue;
      bool dup = false;
      for (int k = 0; k < n; ++k) dup |= buf[k] == j;
      if (!dup) buf[n++] = j;
    }
    for (int a = 1; a < n; ++a)
      for (int b = a; b > 0 && buf[b - 1] > buf[b]; --b) {
        const int32_t t = buf[b]; buf[b] = buf[b - 1]; buf[b - 1] = t;
      }
    nnb[c] = n;
    if (nb) for (int k = 0; k < W; ++k) nb[k * Nc + c] = k < n ? buf[k] : buf[0];
  }
}
__global__ void k_face_nb(int64_t Nf, const int32_t* fv, const int32_t* ptr, const int32_t* idx, int WF,
                          int32_t* fnb, int32_t* nfnb, int* err) {
  int32_t buf[FVS_MAX_FNB];
  GS(f, Nf) {
    int32_t vs[4];
    for (int k = 0; k < 4; ++k) vs[k] = fv[k * Nf + f];
    const int n = union_cells(vs, 4, ptr, idx, buf, FVS_MAX_FNB);
    if (n < 0) { atomicOr(err, MERR_NB); nfnb[f] = 0; continue; }
    nfnb[f] = n;
    if (fnb) for (int k = 0; k < WF; ++k) fnb[k * Nf + f] = k < n ? buf[k] : buf[0];
  }
}
__global__ void k_max_i32(int64_t n, const int32_t* a, int* out) {
  int m = 0;
  GS(i, n) m = max(m, (int)a[i]);
  m = max(m, __shfl_down_sync(0xffffffffu, m, 16));
  m = max(m, __shfl_down_sync(0xffffffffu, m, 8));
  m = max(m, __shfl_down_sync(0xffffffffu, m, 4));
  m = max(m, __shfl_down_sync(0xffffffffu, m, 2));
  m = max(m, __shfl_down_sync(0xffffffffu, m, 1));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// ---------------------------------------------------------------------------
// geometry (Section 2.3, Eq. 11-12)
// ---------------------------------------------------------------------------
__global__ void k_cell_centres(int64_t Nc, int64_t Nv, const double* Xn, const int32_t* cn, double* xc) {
  GS(c, Nc) {
    double s[3] = {0, 0, 0};
    for (int k = 0; k < 8; ++k) {
      const int32_t v = cn[k * Nc + c];
      for (int d = 0; d < 3; ++d) s[d] += Xn[d * Nv + v];
    }
    for (int d = 0; d < 3; ++d) xc[d * Nc + c] = s[d] / 8.0;
  }
}

__global__ void k_face_geometry(int64_t Nf, int64_t Nv, int64_t Nc, const double* Xn, const double* xc,
                                const int32_t* fv, const int32_t* own, const int32_t* nei, double* A,
                                double* nrm, double* cd, double* ce, double* cz, double* Jinv, double* xs,
                                double* skew, double* dof, double* dnf, int* err) {
  GS(f, Nf) {
    double P[4][3];
    for (int k = 0; k < 4; ++k) {
      const int32_t v = fv[k * Nf + f];
      for (int d = 0; d < 3; ++d) P[k][d] = Xn[d * Nv + v];
    }
    double e1[3], e2[3], S[3], xf[3];
    for (int d = 0; d < 3; ++d) {
      e1[d] = P[2][d] - P[0][d];   // V1 -> V3 (eta)
      e2[d] = P[3][d] - P[1][d];   // V2 -> V4 (zeta)
      xf[d] = 0.25 * (P[0][d] + P[1][d] + P[2][d] + P[3][d]);
    }
    S[0] = 0.5 * (e1[1] * e2[2] - e1[2] * e2[1]);
    S[1] = 0.5 * (e1[2] * e2[0] - e1[0] * e2[2]);
    S[2] = 0.5 * (e1[0] * e2[1] - e1[1] * e2[0]);
    const double a = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
    const double n[3] = {S[0] / a, S[1] / a, S[2] / a};
    const int32_t o = own[f], q = nei[f];
    double dv[3];
    for (int d = 0; d < 3; ++d) dv[d] = (q >= 0 ? xc[d * Nc + q] : xf[d]) - xc[d * Nc + o];
    const double nd = n[0] * dv[0] + n[1] * dv[1] + n[2] * dv[2];
    const double J[9] = {dv[0], dv[1], dv[2], e1[0], e1[1], e1[2], e2[0], e2[1], e2[2]};
    double Ji[9];
    const double det = inv3(J, Ji);
    if (!(a > 0.0) || !(nd > 0.0) || det == 0.0) atomicOr(err, MERR_GEOM);
    // t = n - d/(n.d); w = J^-T t so that t . (J^-1 delta) = w . delta
    const double t[3] = {n[0] - dv[0] / nd, n[1] - dv[1] / nd, n[2] - dv[2] / nd};
    double w[3];
    for (int j = 0; j < 3; ++j) w[j] = Ji[0 * 3 + j] * t[0] + Ji[1 * 3 + j] * t[1] + Ji[2 * 3 + j] * t[2];
    A[f] = a;
    for (int d = 0; d < 3; ++d) nrm[d * Nf + f] = n[d];
    cd[f] = a * (1.0 / nd + w[0]);
    ce[f] = a * w[1];
    cz[f] = a * w[2];
    for (int k = 0; k < 9; ++k) Jinv[k * Nf + f] = Ji[k];
    xs[f] = (xf[0] * S[0] + xf[1] * S[1] + xf[2] * S[2]) / 3.0;
    // distances from the owner / neighbour centre to the face centre
    double a2 = 0.0, b2 = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double ea = xf[d] - xc[d * Nc + o];
      a2 += ea * ea;
      if (q >= 0) {
        const double eb = xf[d] - xc[d * Nc + q];
        b2 += eb * eb;
      }
    }
    dof[f] = sqrt(a2);
    dnf[f] = sqrt(b2);
    const double l1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    const double l2 = sqrt(e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]);
    skew[f] = fmax(fabs(w[0]) * nd, fmax(fabs(w[1]) * l1, fabs(w[2]) * l2));
  }
}

__global__ void k_volumes(int64_t Nc, const int32_t* cf, const int8_t* cfs, const double* xs, double* V, int* err) {
  GS(c, Nc) {
    double v = 0.0;
    for (int k = 0; k < 6; ++k) v += (double)cfs[k * Nc + c] * xs[cf[k * Nc + c]];
    V[c] = v;
    if (!(v > 0.0)) atomicOr(err, MERR_GEOM);
  }
}

// ---------------------------------------------------------------------------
// base operator rows (Eq. 10-12): sum over the faces of c of
//   sigma * [cd (phi_C2 - phi_C1) + ce (phi_V3 - phi_V1) + cz (phi_V4 - phi_V2)]
// kind 0: velocity (walls and wall vertices carry 0)
// kind 1: pressure with every cell flowing (walls carry no flux)
// kind 2: temperature (fixed-temperature walls and their vertices carry the
//         wall value; adiabatic walls carry no flux; faces with gint > 0 carry
//         the orthogonal series flux only: metal-mold interfaces, and
//         convective walls, whose gint includes the film coefficient)
// ---------------------------------------------------------------------------
struct RowCtx {
  int64_t Nc, Nf;
  const int32_t *cf, *fv, *own, *nei, *patch, *vc_ptr, *vc_idx, *nb, *nnb;
  const int8_t* cfs;
  const uint8_t* vbnd;
  const double *cd, *ce, *cz;
  const int32_t* bc_type;
  const double* bc_T;
  const double* vfix;     // temperature: fixed vertex value or NaN if free
  const double* kf;       // temperature: per-face conductivity factor (null: 1)
  const double* gint;     // temperature: series conductance (> 0 on metal-mold faces and convective walls)
};

__device__ __forceinline__ void add_vertex(const RowCtx& x, int kind, int64_t c, int nn, int32_t v, double coef,
                                           double* acc, double& cst) {
  if (kind == 0 && x.vbnd[v]) return;                 // wall vertex: u = 0
  if (kind == 2) {
    const double fixed = x.vfix[v];
    if (fixed == fixed) { cst += coef * fixed; return; }
  }
  const int32_t lo = x.vc_ptr[v], hi = x.vc_ptr[v + 1];
  const double share = coef / (double)(hi - lo);
  for (int32_t e = lo; e < hi; ++e) {
    const int p = find_sorted(x.nb + c, x.Nc, nn, x.vc_idx[e]);
    if (p >= 0) acc[p] += share;
  }
}

__device__ void assemble_base_row(const RowCtx& x, int kind, int64_t c, double* acc, double& cst) {
  const int nn = x.nnb[c];
  for (int k = 0; k < FVS_MAX_NB; ++k) acc[k] = 0.0;
  cst = 0.0;
  const int pc = find_sorted(x.nb + c, x.Nc, nn, (int32_t)c);
  for (int s = 0; s < 6; ++s) {
    const int32_t f = x.cf[s * x.Nc + c];
    double sg = (double)x.cfs[s * x.Nc + c];
    const int32_t q = x.nei[f];
    if (kind == 2 && x.gint && x.gint[f] > 0.0) {
      if (q < 0) {
        // convective wall: gint (T_amb - T_c), c the owner, no cross terms
        if (pc >= 0) acc[pc] -= sg * x.gint[f];
        cst += sg * x.gint[f] * x.bc_T[x.patch[f]];
        continue;
      }
      // metal-mold interface: orthogonal flux through the series resistance
      const int p2 = find_sorted(x.nb + c, x.Nc, nn, q);
      const int p1 = find_sorted(x.nb + c, x.Nc, nn, x.own[f]);
      if (p2 >= 0) acc[p2] += sg * x.gint[f];
      if (p1 >= 0) acc[p1] -= sg * x.gint[f];
      continue;
    }
    if (kind == 2 && x.kf) sg *= x.kf[f];   // conductive flux: k_f times the face gradient
    double phib = 0.0;
    if (q < 0) {
      if (kind == 1) continue;
      if (kind == 2) {
        if (x.bc_type[x.patch[f]] != FVS_BC_DIRICHLET) continue;
        phib = x.bc_T[x.patch[f]];
      }
      // flux = cd (phi_b - phi_c): c is the owner of a wall face
      if (pc >= 0) acc[pc] -= sg * x.cd[f];
      cst += sg * x.cd[f] * phib;
    } else {
      const int p2 = find_sorted(x.nb + c, x.Nc, nn, q);
      const int p1 = find_sorted(x.nb + c, x.Nc, nn, x.own[f]);
      if (p2 >= 0) acc[p2] += sg * x.cd[f];
      if (p1 >= 0) acc[p1] -= sg * x.cd[f];
    }
    const int32_t v1 = x.fv[f], v2 = x.fv[x.Nf + f], v3 = x.fv[2 * x.Nf + f], v4 = x.fv[3 * x.Nf + f];
    add_vertex(x, kind, c, nn, v3, sg * x.ce[f], acc, cst);
    add_vertex(x, kind, c, nn, v1, -sg * x.ce[f], acc, cst);
    add_vertex(x, kind, c, nn, v4, sg * x.cz[f], acc, cst);
    add_vertex(x, kind, c, nn, v2, -sg * x.cz[f], acc, cst);
  }
}

__global__ void k_assemble_base(RowCtx x, int kind, int W, int32_t* col, double* val, double* diag, double* cvec) {
  double acc[FVS_MAX_NB];
  GS(c, x.Nc) {
    double cst;
    assemble_base_row(x, kind, c, acc, cst);
    const int nn = x.nnb[c];
    double dg = 0.0;
    for (int k = 0; k < W; ++k) {
      const int32_t j = x.nb[k * x.Nc + c];
      const bool used = k < nn;
      col[k * x.Nc + c] = used ? j : (int32_t)c;
      val[k * x.Nc + c] = used ? acc[k] : 0.0;
      if (used && j == (int32_t)c) dg = acc[k];
    }
    diag[c] = dg;
    if (cvec) cvec[c] = cst;
  }
}

__global__ void k_dirichlet_vertices(int64_t Nf, const int32_t* fv, const int32_t* nei, const int32_t* patch,
                                     const int32_t* bc_type, const double* bc_T, double* vsum, int32_t* vcnt) {
  GS(f, Nf) {
    if (nei[f] >= 0) continue;
    const int32_t p = patch[f];
    if (bc_type[p] != FVS_BC_DIRICHLET) continue;
    for (int k = 0; k < 4; ++k) {
      const int32_t v = fv[k * Nf + f];
      atomicAdd(&vsum[v], bc_T[p]);
      atomicAdd(&vcnt[v], 1);
    }
  }
}
__global__ void k_vfix(int64_t Nv, const double* vsum, const int32_t* vcnt, double* vfix) {
  GS(v, Nv) vfix[v] = vcnt[v] > 0 ? vsum[v] / (double)vcnt[v] : __longlong_as_double(0x7ff8000000000000LL);
}

static RowCtx row_ctx(fvs_mesh m) {
  RowCtx x;
  x.Nc = m->Nc; x.Nf = m->Nf;
  x.cf = m->cf; x.fv = m->fv; x.own = m->own; x.nei = m->nei; x.patch = m->patch;
  x.vc_ptr = m->vc_ptr; x.vc_idx = m->vc_idx; x.nb = m->nb; x.nnb = m->nnb;
  x.cfs = m->cfs; x.vbnd = m->vbnd;
  x.cd = m->cd; x.ce = m->ce; x.cz = m->cz;
  x.bc_type = nullptr; x.bc_T = nullptr; x.vfix = nullptr;
  x.kf = nullptr; x.gint = nullptr;
  return x;
}

fvs_status assemble_temperature_operator(fvs_mesh m, const int32_t* d_bc_type, const double* d_bc_T, Ell& LT,
                                         double* lT, cudaStream_t s, const double* kf, const double* gint) {
  DBuf<double> vsum, vfix;
  DBuf<int32_t> vcnt;
  FVS_TRY(vsum.alloc(m->Nv)); FVS_TRY(vfix.alloc(m->Nv)); FVS_TRY(vcnt.alloc(m->Nv));
  FVS_TRY(vsum.zero(s)); FVS_TRY(vcnt.zero(s));
  k_dirichlet_vertices<<<stride_grid(m->Nf, 256), 256, 0, s>>>(m->Nf, m->fv, m->nei, m->patch, d_bc_type, d_bc_T,
                                                              vsum, vcnt); FVS_COUNT_LAUNCH();
  k_vfix<<<stride_grid(m->Nv, 256), 256, 0, s>>>(m->Nv, vsum, vcnt, vfix); FVS_COUNT_LAUNCH();
  FVS_TRY(LT.alloc(m->Nc, m->W));
  RowCtx x = row_ctx(m);
  x.bc_type = d_bc_type; x.bc_T = d_bc_T; x.vfix = vfix;
  x.kf = kf; x.gint = gint;
  k_assemble_base<<<stride_grid(m->Nc, 128, 4), 128, 0, s>>>(x, 2, m->W, LT.col, LT.val, LT.diag, lT); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  FVS_CUDA(cudaStreamSynchronize(s));
  return FVS_OK;
}

// zones in the mesh numbering from the caller's cell order; values other
// than 0 (metal) and 1 (mold) are flagged
__global__ void k_zone_in(int64_t Nc, const int32_t* cell_in, const int32_t* zin, uint8_t* zone, int* err) {
  GS(c, Nc) {
    const int32_t z = zin[cell_in[c]];
    if (z != 0 && z != 1) atomicOr(err, 1);
    zone[c] = z == 1 ? 1 : 0;
  }
}

fvs_status mesh_set_zones(fvs_mesh m, const int32_t* zone_host) {
  cudaStream_t s = m->stream;
  const int64_t Nc = m->Nc;
  DBuf<int32_t> zin;
  DBuf<int> err;
  FVS_TRY(zin.alloc(Nc + 1));
  FVS_TRY(err.alloc(1));
  FVS_TRY(err.zero(s));
  FVS_CUDA(cudaMemcpyAsync(zin.p, zone_host, Nc * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  k_zone_in<<<stride_grid(Nc, 256), 256, 0, s>>>(Nc, m->cell_in, zin, m->zone, err); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  int h = 0;
  FVS_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  FVS_CUDA(cudaStreamSynchronize(s));
  if (h) {
    set_error("cell zones must be 0 (metal) or 1 (mold)");
    return FVS_ERR_ARG;
  }
  return FVS_OK;
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
static fvs_status check_err(DBuf<int>& err, cudaStream_t s, const char* stage) {
  int h = 0;
  FVS_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  FVS_CUDA(cudaStreamSynchronize(s));
  if (h) {
    set_error("mesh validation failed at %s (flags 0x%x: %s%s%s%s%s%s)", stage, h,
              (h & MERR_RANGE) ? "id out of range; " : "", (h & MERR_FACECOUNT) ? "cell without 6 faces; " : "",
              (h & MERR_VALENCE) ? "vertex valence; " : "", (h & MERR_NB) ? "neighbour list too long; " : "",
              (h & MERR_GEOM) ? "non-positive area/volume or degenerate face frame; " : "",
              (h & MERR_OWNER) ? "face with identical owners; " : "");
    return FVS_ERR_MESH;
  }
  return FVS_OK;
}

template <typename T>
static fvs_status upload(DBuf<T>& d, const T* h, size_t n, cudaStream_t s) {
  FVS_TRY(d.alloc(n));
  FVS_CUDA(cudaMemcpyAsync(d.p, h, n * sizeof(T), cudaMemcpyHostToDevice, s));
  return FVS_OK;
}

static fvs_status sort_pairs(cudaStream_t s, int64_t n, DBuf<uint64_t>& key, DBuf<int32_t>& val,
                             DBuf<int32_t>& out) {
  DBuf<uint64_t> key2;
  FVS_TRY(key2.alloc(n));
  FVS_TRY(out.alloc(n));
  size_t bytes = 0;
  FVS_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, bytes, key.p, key2.p, val.p, out.p, (int)n, 0, 64, s));
  DBuf<uint8_t> tmp;
  FVS_TRY(tmp.alloc(bytes + 16));
  FVS_CUDA(cub::DeviceRadixSort::SortPairs(tmp.p, bytes, key.p, key2.p, val.p, out.p, (int)n, 0, 64, s));
  FVS_CUDA(cudaStreamSynchronize(s));
  return FVS_OK;
}

fvs_status mesh_build(fvs_mesh m, const double* nodes, int64_t Nv, const int32_t* cells, int64_t Nc,
                      const int32_t* faces, int64_t Nf, const int32_t* fcells, const int32_t* patch, int reorder) {
  cudaStream_t s = m->stream;
  m->Nc = Nc; m->Nf = Nf; m->Nv = Nv;
  DBuf<int> err;
  FVS_TRY(err.alloc(1));
  FVS_TRY(err.zero(s));

  DBuf<double> X;
  DBuf<int32_t> C, F, FC, P;
  FVS_TRY(upload(X, nodes, (size_t)Nv * 3, s));
  FVS_TRY(upload(C, cells, (size_t)Nc * 8, s));
  FVS_TRY(upload(F, faces, (size_t)Nf * 4, s));
  FVS_TRY(upload(FC, fcells, (size_t)Nf * 2, s));
  FVS_TRY(upload(P, patch, (size_t)Nf, s));
  k_validate<<<stride_grid(std::max(Nc, Nf), 256), 256, 0, s>>>(Nv, Nc, Nf, C, F, FC, P, err); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  FVS_TRY(check_err(err, s, "ids"));

  // bounding box and renumbering
  const int bbn = 64;
  DBuf<double> bb;
  FVS_TRY(bb.alloc(6 * bbn));
  k_bbox_part<<<bbn, 256, 0, s>>>(Nv, X, bb); FVS_COUNT_LAUNCH();
  k_bbox_final<<<1, 32, 0, s>>>(bbn, bb); FVS_COUNT_LAUNCH();
  DBuf<uint64_t> key;
  DBuf<int32_t> val, node_in, node_new;
  FVS_TRY(key.alloc(std::max(std::max(Nc, Nf), Nv)));
  FVS_TRY(val.alloc(std::max(std::max(Nc, Nf), Nv)));
  k_cell_keys<<<stride_grid(Nc, 256), 256, 0, s>>>(Nc, X, C, bb, reorder, key, val); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  FVS_TRY(sort_pairs(s, Nc, key, val, m->cell_in));
  FVS_TRY(m->cell_new.alloc(Nc));
  k_invert<<<stride_grid(Nc, 256), 256, 0, s>>>(Nc, m->cell_in, m->cell_new); FVS_COUNT_LAUNCH();
  k_node_keys<<<stride_grid(Nv, 256), 256, 0, s>>>(Nv, X, bb, reorder, key, val); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  FVS_TRY(sort_pairs(s, Nv, key, val, node_in));
  FVS_TRY(node_new.alloc(Nv));
  k_invert<<<stride_grid(Nv, 256), 256, 0, s>>>(Nv, node_in, node_new); FVS_COUNT_LAUNCH();
  k_face_keys<<<stride_grid(Nf, 256), 256, 0, s>>>(Nf, FC, m->cell_new, reorder, key, val); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  FVS_TRY(sort_pairs(s, Nf, key, val, m->face_in));
  FVS_TRY(m->face_new.alloc(Nf));
  k_invert<<<stride_grid(Nf, 256), 256, 0, s>>>(Nf, m->face_in, m->face_new); FVS_COUNT_LAUNCH();

  DBuf<double> Xn;
  DBuf<int32_t> cn;
  FVS_TRY(Xn.alloc(3 * Nv));
  FVS_TRY(cn.alloc(8 * Nc));
  FVS_TRY(m->fv.alloc(4 * Nf)); FVS_TRY(m->own.alloc(Nf)); FVS_TRY(m->nei.alloc(Nf)); FVS_TRY(m->patch.alloc(Nf));
  k_gather_nodes<<<stride_grid(Nv, 256), 256, 0, s>>>(Nv, X, node_in, Xn); FVS_COUNT_LAUNCH();
  k_gather_cells<<<stride_grid(Nc, 256), 256, 0, s>>>(Nc, C, m->cell_in, node_new, cn); FVS_COUNT_LAUNCH();
  k_gather_faces<<<stride_grid(Nf, 256), 256, 0, s>>>(Nf, F, FC, P, m->face_in, node_new, m->cell_new, m->fv,
                                                      m->own, m->nei, m->patch); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();

  // cell -> faces
  DBuf<int32_t> cnt;
  FVS_TRY(cnt.alloc(std::max(Nc, Nv) + 1));
  FVS_TRY(cnt.zero(s));
  FVS_TRY(m->cf.alloc(6 * Nc)); FVS_TRY(m->cfs.alloc(6 * Nc));
  k_cell_faces<<<stride_grid(Nf, 256), 256, 0, s>>>(Nf, Nc, m->own, m->nei, cnt, m->cf, m->cfs, err); FVS_COUNT_LAUNCH();
  k_cell_faces_sort<<<stride_grid(Nc, 256), 256, 0, s>>>(Nc, cnt, m->cf, m->cfs, err); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  FVS_TRY(check_err(err, s, "cell faces"));

  // vertex -> cells
  FVS_TRY(cnt.zero(s));
  FVS_TRY(m->vc_ptr.alloc(Nv + 1));
  k_vertex_count<<<stride_grid(Nc, 256), 256, 0, s>>>(Nc, cn, cnt); FVS_COUNT_LAUNCH();
  ScanWork sw;
  FVS_TRY(exclusive_scan(s, sw, Nv + 1, cnt, m->vc_ptr));
  FVS_TRY(m->vc_idx.alloc(8 * Nc));
  FVS_TRY(cnt.zero(s));
  k_vertex_fill<<<stride_grid(Nc, 256), 256, 0, s>>>(Nc, cn, m->vc_ptr, cnt, m->vc_idx); FVS_COUNT_LAUNCH();
  k_vertex_sort<<<stride_grid(Nv, 256), 256, 0, s>>>(Nv, m->vc_ptr, m->vc_idx, err); FVS_COUNT_LAUNCH();
  FVS_TRY(m->vbnd.alloc(Nv));
  FVS_TRY(m->vbnd.zero(s));
  k_vertex_boundary<<<stride_grid(Nf, 256), 256, 0, s>>>(Nf, m->fv, m->nei, m->vbnd); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  FVS_TRY(check_err(err, s, "vertex cells"));

  // neighbour lists: count pass, width, fill pass
  DBuf<int> mx;
  FVS_TRY(mx.alloc(2));
  FVS_TRY(mx.zero(s));
  FVS_TRY(m->nnb.alloc(Nc)); FVS_TRY(m->nfnb.alloc(Nf));
  k_cell_nb<<<stride_grid(Nc, 128, 4), 128, 0, s>>>(Nc, cn, m->vc_ptr, m->vc_idx, 0, nullptr, m->nnb, err); FVS_COUNT_LAUNCH();
  k_face_nb<<<stride_grid(Nf, 128, 4), 128, 0, s>>>(Nf, m->fv, m->vc_ptr, m->vc_idx, 0, nullptr, m->nfnb, err); FVS_COUNT_LAUNCH();
  k_max_i32<<<stride_grid(Nc, 256), 256, 0, s>>>(Nc, m->nnb, mx.p); FVS_COUNT_LAUNCH();
  k_max_i32<<<stride_grid(Nf, 256), 256, 0, s>>>(Nf, m->nfnb, mx.p + 1); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  FVS_TRY(check_err(err, s, "neighbour lists"));
  int hmx[2];
  FVS_CUDA(cudaMemcpyAsync(hmx, mx.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  FVS_CUDA(cudaStreamSynchronize(s));
  m->W = hmx[0];
  m->WF = hmx[1];
  FVS_TRY(m->nb.alloc((size_t)m->W * Nc)); FVS_TRY(m->fnb.alloc((size_t)m->WF * Nf));
  k_cell_nb<<<stride_grid(Nc, 128, 4), 128, 0, s>>>(Nc, cn, m->vc_ptr, m->vc_idx, m->W, m->nb, m->nnb, err); FVS_COUNT_LAUNCH();
  k_face_nb<<<stride_grid(Nf, 128, 4), 128, 0, s>>>(Nf, m->fv, m->vc_ptr, m->vc_idx, m->WF, m->fnb, m->nfnb, err); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();

  // geometry
  DBuf<double> xc, xs, skew;
  FVS_TRY(xc.alloc(3 * Nc)); FVS_TRY(xs.alloc(Nf)); FVS_TRY(skew.alloc(Nf));
  FVS_TRY(m->A.alloc(Nf)); FVS_TRY(m->nrm.alloc(3 * Nf)); FVS_TRY(m->cd.alloc(Nf)); FVS_TRY(m->ce.alloc(Nf));
  FVS_TRY(m->cz.alloc(Nf)); FVS_TRY(m->Jinv.alloc(9 * Nf)); FVS_TRY(m->V.alloc(Nc));
  k_cell_centres<<<stride_grid(Nc, 256), 256, 0, s>>>(Nc, Nv, Xn, cn, xc); FVS_COUNT_LAUNCH();
  FVS_TRY(m->dof.alloc(Nf)); FVS_TRY(m->dnf.alloc(Nf));
  FVS_TRY(m->zone.alloc(Nc));
  FVS_TRY(m->zone.zero(s));   // every cell metal until fvs_mesh_set_zones says otherwise
  k_face_geometry<<<stride_grid(Nf, 128), 128, 0, s>>>(Nf, Nv, Nc, Xn, xc, m->fv, m->own, m->nei, m->A, m->nrm,
                                                      m->cd, m->ce, m->cz, m->Jinv, xs, skew, m->dof, m->dnf, err);
  FVS_COUNT_LAUNCH();
  k_volumes<<<stride_grid(Nc, 256), 256, 0, s>>>(Nc, m->cf, m->cfs, xs, m->V, err); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  FVS_TRY(check_err(err, s, "geometry"));
  {
    // total volume and the largest dimensionless cross-diffusion weight
    Reducer red;
    FVS_TRY(red.init());
    DBuf<double> ones, zero;
    FVS_TRY(ones.alloc(Nc));
    FVS_TRY(zero.alloc(Nf));
    FVS_TRY(zero.zero(s));
    FVS_TRY(vfill(s, Nc, 1.0, ones));
    FVS_TRY(red.dot(s, Nc, m->V, ones, S_TMP0));
    FVS_TRY(red.max_abs_diff2(s, Nf, skew, zero, nullptr, nullptr, S_TMP1, -1));
    FVS_TRY(red.fetch(s));
    m->total_volume = red.host[S_TMP0];
    m->orthogonal = red.host[S_TMP1] < 1e-10 ? 1 : 0;
  }
  const char* full_st = getenv("FVS_FULL_STENCIL");   // keep the vertex-neighbour stencil
  if (m->orthogonal && !(full_st && *full_st && *full_st != '0')) {
    // orthogonal mesh: the cross-diffusion weights vanish, so every operator
    // couples a cell to the cells across its faces only.  The stencil drops
    // to those (7 slots instead of 27: a quarter of the bytes and FMAs of
    // every operator row) and the weights are set to exact zeros.
    FVS_TRY(m->ce.zero(s));
    FVS_TRY(m->cz.zero(s));
    FVS_TRY(mx.zero(s));
    k_cell_nb_faces<<<stride_grid(Nc, 256), 256, 0, s>>>(Nc, m->cf, m->own, m->nei, 0, nullptr, m->nnb);
    FVS_COUNT_LAUNCH();
    k_max_i32<<<stride_grid(Nc, 256), 256, 0, s>>>(Nc, m->nnb, mx.p); FVS_COUNT_LAUNCH();
    int w = 0;
    FVS_CUDA(cudaMemcpyAsync(&w, mx.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    FVS_CUDA(cudaStreamSynchronize(s));
    m->W = w;
    m->nb.release();
    FVS_TRY(m->nb.alloc((size_t)m->W * Nc));
    k_cell_nb_faces<<<stride_grid(Nc, 256), 256, 0, s>>>(Nc, m->cf, m->own, m->nei, m->W, m->nb, m->nnb);
    FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
  }
  // counts
  {
    std::vector<int32_t> hn(Nf);
    FVS_CUDA(cudaMemcpyAsync(hn.data(), m->nei.p, Nf * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    std::vector<int32_t> hp(Nf);
    FVS_CUDA(cudaMemcpyAsync(hp.data(), m->patch.p, Nf * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    FVS_CUDA(cudaStreamSynchronize(s));
    int64_t nfi = 0;
    int pmax = -1;
    for (int64_t f = 0; f < Nf; ++f) {
      if (hn[f] >= 0) ++nfi; else pmax = std::max(pmax, (int)hp[f]);
    }
    m->Nfi = nfi;
    m->npatch = pmax + 1;
  }

  // base operators
  RowCtx x = row_ctx(m);
  FVS_TRY(m->Lu.alloc(Nc, m->W));
  FVS_TRY(m->Pb.alloc(Nc, m->W));
  k_assemble_base<<<stride_grid(Nc, 128, 4), 128, 0, s>>>(x, 0, m->W, m->Lu.col, m->Lu.val, m->Lu.diag, nullptr); FVS_COUNT_LAUNCH();
  k_assemble_base<<<stride_grid(Nc, 128, 4), 128, 0, s>>>(x, 1, m->W, m->Pb.col, m->Pb.val, m->Pb.diag, nullptr); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  FVS_CUDA(cudaStreamSynchronize(s));
  return FVS_OK;
}

}  // namespace fvs
