// Lockstep batch of plain solves on one mesh (the sampling of Section 2.7:
// every sample is a deterministic solve with its own melt temperature, wall
// temperature and liquidus).  All samples advance together: every field
// carries a sample index and lives [row][sample] with the sample fastest, the
// sample count rounded up to a multiple of 32 (Sp), so one launch per phase
// advances every sample and a warp reads 32 samples of one row at once.
//
// Shared across samples: the mesh, the velocity and temperature operators
// (matrix bytes read once per row for all samples), the pressure base
// operator, and the AMG aggregation formed on it.  Per sample: masks (liquid /
// mushy, pressure cells, face cases), the pressure rows next to solid cells
// (re-assembled per sample, Section 2.4.2), the Galerkin values of every
// coarse level and the coarsest inverse.  Rows of solid (momentum) or
// non-flowing (pressure) cells are identity rows; the Krylov vectors stay zero
// there, so the shared operators need no column masks.
#pragma once

#include "amg.cuh"
#include "mesh.cuh"

namespace fvs {

constexpr int BATCH_NCM = 8;   // liquid pockets per sample handled by the null-space projection

// per-sample scalar slots of the batched Krylov drivers: sc[slot * Sp + s]
enum BSlot {
  B_RHO = 0, B_RHO_OLD, B_ALPHA, B_OMEGA, B_RV, B_TS, B_TT, B_RR, B_BB, B_RZ, B_RZ_OLD, B_PQ, B_TOL2,
  B_FIRST, B_T0, B_T1, B_T2, B_NSLOT
};

// Staging of x for a batched operator: the rows are cut into blocks of R
// consecutive rows; block b lists the distinct columns its rows reference
// (ucol[uptr[b] .. uptr[b+1])), and every stored entry q = k*n + i carries
// its column's position in that list (li[q] < 256).  A kernel block loads
// x of those columns for its 32 samples into shared memory once (all loads
// independent) and gathers from there, instead of one dependent global
// gather per entry.
struct XStage {
  int R = 0;                      // rows per block; 0: not built
  int64_t nblk = 0;
  int umax = 0;                   // largest column list of a block
  DBuf<int32_t> uptr, ucol;
  DBuf<uint8_t> li;
};

// launch shape of a batched operator kernel: blocks of 32 samples x rows,
// at most per_sm blocks per SM, or the staged kernel over stage->R rows per
// block (chosen by the autotuner)
struct BShape {
  int rows = 8;
  int per_sm = 16;
  const XStage* stage = nullptr;
};

// one level of the batched AMG hierarchy
struct BLevel {
  int64_t n = 0;
  int w = 0;
  const int32_t* col = nullptr;   // shared pattern [k*n + i] (level 0: the pressure base operator's)
  const int32_t* rlen = nullptr;  // levels >= 1: stored entries per row
  DBuf<double> val;               // levels >= 1: per-sample values [(k*n + i)*Sp + s]
  DBuf<int32_t> dslot;            // levels >= 1: slot of the diagonal in each row (-1 none)
  DBuf<double> dinv;              // [i*Sp + s]
  const int32_t* agg = nullptr;   // row -> aggregate of the next level (shared)
  const int32_t* mptr = nullptr;  // members of the next level's rows (shared CSR)
  const int32_t* midx = nullptr;
  DBuf<int32_t> gptr, gidx;       // Galerkin map: coarse entry q = r*nc + I <- this level's entries k*n + i
  DBuf<double> b, x, r, y;        // V-cycle work [n*Sp]
  DBuf<float> valf, dinvf;        // FP32 copies (mixed precision)
  DBuf<float> bf, xf, rf, yf;
  DBuf<int32_t> lab;              // null-space labels [i*Sp + s] (levels used for label pull-down)
  BShape shape;                   // tuned launch shape of this level's operator
  XStage stage;                   // levels >= 1: x staging of this level's pattern
};

// a device-driven Krylov loop captured as a graph (conditional while-node)
struct BatchGraph {
  cudaGraphExec_t exec = nullptr;
  uint64_t key = 0;
  int maxit = 0;
  unsigned long long kernels = 0;   // launches per iteration (launch counter)
  bool disabled = false;
  ~BatchGraph() { reset(); }
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    key = 0;
  }
};

struct BatchWork {               // Krylov work vectors [n*Sp]
  DBuf<double> r, rh, p, ph, v, sv, sh, t, z, q;
  fvs_status ensure(size_t len);
};

struct Batch {
  fvs_mesh mesh = nullptr;
  cudaStream_t stream = nullptr;
  int64_t S = 0;                  // samples
  int Sp = 0;                     // samples rounded up to 32
  int tiles = 0;                  // Sp / 32
  fvs_props props{};
  double time = 0.0;

  // per-sample inputs
  DBuf<double> Tliq, Twall, Tmelt;   // [Sp]
  // grain growth (Eq. 24-26): r^2 [Nc*Sp] when D_s > 0
  double grain_kp = 0.0, grain_Ds = 0.0;
  DBuf<double> r2;
  DBuf<uint8_t> run;              // 1 while the sample is being advanced
  std::vector<int64_t> steps;     // steps taken per sample

  // state [Nc*Sp] (vectors [3][Nc][Sp]), face fluxes [Nf*Sp]
  DBuf<double> T, Told, Tnew, fs, fsnew, Tit, fsit, Tlin;
  DBuf<double> u, uold, unew, ustar;
  DBuf<double> F, Fold, Fnew, gradf;
  DBuf<double> p, tliq, tsol;
  DBuf<uint8_t> lm, flow, ppe, fcase;
  DBuf<int32_t> nS;
  DBuf<double> pv, fSv;

  // shared operators
  Ell LT;                         // unit temperature operator, every wall at T = 1
  DBuf<double> lT1;               // its constant part at T_wall = 1
  DBuf<double> kev, kevd;         // -k/2 LT values and diagonal
  DBuf<double> moff;              // -mu/2 Lu off-diagonal values (diagonal slots 0)
  Ell K0;                         // pressure base operator -Pb / rho (every cell flowing)
  DBuf<float> K0f, mvalf;         // FP32 copies of the base values and override rows

  // per-step per-sample systems
  DBuf<double> mdiag;             // momentum diagonal [Nc*Sp] (1 on solid rows)
  DBuf<double> mrhs, mx;          // [3][Nc][Sp]
  DBuf<double> edx, ebase, erhs;  // energy extra diagonal, explicit part, right side
  DBuf<double> jd;                // Jacobi inverse diagonals [Nc*Sp]
  DBuf<double> mfloor;            // momentum: per-sample right-side norm floor [Sp]
  DBuf<uint8_t> econv;            // latent-heat loop converged [Sp]
  DBuf<uint8_t> etake;            // sample iterates in this pass [Sp]
  DBuf<double> ertol;             // inner tolerance of the pass [Sp]
  DBuf<int> nlm;                  // liquid + mushy cells per sample [Sp]
  DBuf<int32_t> ovr;              // pressure row source per (c, s): -2 identity, -1 base, >= 0 override row
  DBuf<double> mval;              // override rows [o*W + k]
  DBuf<int> ocount;
  int64_t ocap = 0;
  DBuf<double> prhs, px;

  // AMG: the aggregation of the base operator, per-sample values
  Amg base;
  std::vector<std::unique_ptr<BLevel>> lv;
  int nc = 0;                     // coarsest rows
  DBuf<double> Ainv;              // [Sp][nc][nc]
  DBuf<int32_t> clab;             // [Sp][nc]
  DBuf<uint8_t> csing;            // [Sp][nc]
  DBuf<int> cncomp;               // [Sp]
  DBuf<int32_t> cid;              // compact projected part per (s, coarsest part) [Sp*nc]
  DBuf<double> ccnt, csum;        // [Sp*BATCH_NCM]
  DBuf<int> ccount;               // [Sp*nc] fine rows per coarsest part
  bool amg_ok = false;
  bool fp32 = false;              // FP32 V-cycle inside the FP64 Krylov method
  AmgOptions aopt;

  // reductions
  int nb = 0;                     // row blocks of the reduction kernels
  DBuf<double> part;              // [2 * Sp * nb] (and BATCH_NCM * Sp * nb for parts)
  DBuf<int> redcnt;               // [tiles] finished blocks of a reduction (the last one resets it)
  DBuf<double> sc;                // [B_NSLOT * Sp]
  DBuf<uint8_t> kact;             // Krylov: sample still iterating
  DBuf<uint8_t> krestart;         // Krylov: sample restarts (breakdown)
  DBuf<int> kcount;
  DBuf<int> err;
  double* host = nullptr;         // pinned [B_NSLOT * Sp + 64]
  double* phase_ms = nullptr;     // phase times (debug)
  uint64_t batch_version = 0;     // bumped when operator or hierarchy buffers move
  BatchGraph gmom[3], gp, ge;     // captured solve loops
  BShape shp_mom, shp_energy;     // tuned launch shapes of the shared operators
  XStage stage_p, stage_m, stage_e;   // x staging of the fine pressure, momentum and energy patterns
  BatchWork kw;

  ~Batch();
};

struct UqSpec;
fvs_status batch_run(fvs_mesh mesh, const fvs_props* base, int64_t n, const double* inputs, double dt,
                     int max_steps, const UqSpec& spec, double* qoi, int64_t* steps);

}  // namespace fvs
