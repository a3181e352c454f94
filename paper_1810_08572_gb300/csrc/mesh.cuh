// Device-resident unstructured hexahedral mesh (Section 2.3, Fig. 1) after
// renumbering, with its geometry and the fixed parts of the operators.
#pragma once

#include "la.cuh"

// Largest vertex-neighbour stencil of a cell and neighbour set of a face.
#define FVS_MAX_NB 64
#define FVS_MAX_FNB 48
#define FVS_MAX_VCELLS 24

struct fvs_mesh_s {
  cudaStream_t stream = nullptr;
  int device = 0;
  int64_t Nc = 0, Nf = 0, Nv = 0, Nfi = 0;
  int W = 0;    // width of the cell neighbour lists nb(c) (vertex neighbours incl. c)
  int WF = 0;   // width of the face neighbour lists N(f)
  int npatch = 0;
  int orthogonal = 0;
  double total_volume = 0.0;

  // numbering: *_in maps new -> input id, *_new maps input -> new id
  fvs::DBuf<int32_t> cell_in, cell_new, face_in, face_new;

  // connectivity in new numbering (all slot-major / SoA)
  fvs::DBuf<int32_t> fv;     // [4*Nf]  face corners V1..V4
  fvs::DBuf<int32_t> own, nei, patch;   // [Nf]
  fvs::DBuf<int32_t> cf;     // [6*Nc]  faces of each cell
  fvs::DBuf<int8_t> cfs;     // [6*Nc]  +1 if the cell owns the face, -1 if neighbour
  fvs::DBuf<int32_t> vc_ptr, vc_idx;   // vertex -> cells (CSR, sorted)
  fvs::DBuf<uint8_t> vbnd;   // 1 if the vertex lies on a wall
  fvs::DBuf<int32_t> nb, nnb;    // [W*Nc] sorted vertex neighbours of each cell (incl. itself)
  fvs::DBuf<int32_t> fnb, nfnb;  // [WF*Nf] sorted N(f): cells sharing a vertex with f

  // geometry
  fvs::DBuf<double> V;       // [Nc]
  fvs::DBuf<double> A;       // [Nf] face area
  fvs::DBuf<double> nrm;     // [3*Nf] unit normal (owner -> neighbour)
  fvs::DBuf<double> cd, ce, cz;   // [Nf] A (1/(n.d) + w0), A w1, A w2 (Eq. 11-12)
  fvs::DBuf<double> Jinv;    // [9*Nf] inverse local Jacobian, row-major per face (slot-major)
  fvs::DBuf<double> dof, dnf; // [Nf] owner / neighbour centre to face centre distances (0 on walls)
  fvs::DBuf<uint8_t> zone;   // [Nc] 0 metal, 1 mold (all 0 unless set)

  // base operators over nb(c), unit coefficient (Eq. 10-12):
  // Lu: velocity diffusion, no-slip walls; Pb: pressure, all cells flowing
  fvs::Ell Lu, Pb;
};

namespace fvs {
fvs_status mesh_build(fvs_mesh m, const double* nodes, int64_t Nv, const int32_t* cells, int64_t Nc,
                      const int32_t* faces, int64_t Nf, const int32_t* fcells, const int32_t* patch,
                      int reorder);

// Cell zones (caller's cell order): 0 metal, 1 mold.
fvs_status mesh_set_zones(fvs_mesh m, const int32_t* zone_host);

// Assemble the unit temperature operator with wall data: L (same pattern as
// Lu) and constant l (Dirichlet walls).  bc_type/bc_T indexed by patch.
// With kf (per face) each face's flux is scaled by it (the conductive
// operator); faces with gint > 0 (metal-mold interface) carry only
// gint (T_C2 - T_C1).
fvs_status assemble_temperature_operator(fvs_mesh m, const int32_t* d_bc_type, const double* d_bc_T,
                                         Ell& LT, double* lT, cudaStream_t s, const double* kf = nullptr,
                                         const double* gint = nullptr);
}  // namespace fvs
