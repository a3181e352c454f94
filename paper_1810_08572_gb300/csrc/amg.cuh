// Aggregation algebraic multigrid for the pressure system (Section 2.5: the
// paper preconditions its Krylov solver with BoomerAMG; this GPU-native
// replacement aggregates by a parallel maximal independent set on the strong
// connections, builds Galerkin coarse operators with piecewise-constant
// transfers, and solves the coarsest level densely with one pinned unknown
// per singular connected part -- the disjoint liquid pockets of Section 2.5).
#pragma once

#include <memory>
#include <vector>

#include "la.cuh"
#include "scan.cuh"

namespace fvs {

struct AmgLevel {
  Ell own;              // coarse operator (levels >= 1)
  const Ell* A = nullptr;
  DBuf<double> dinv;    // 1 / diagonal
  DBuf<float> dinvf;
  DBuf<float> valf;     // FP32 copy of the operator values (mixed precision)
  DBuf<int32_t> rlen;   // coarse levels: stored entries per row (the rest of the row is padding)
  DBuf<int32_t> agg;    // row -> aggregate (row of the next level)
  DBuf<int32_t> mptr, midx;   // members of each aggregate of the next level (CSR)
  DBuf<double> b, x, y, r, t;    // V-cycle work
  DBuf<float> bf, xf, yf, rf, tf; // FP32 V-cycle work
  DBuf<uint8_t> dirty;  // rows changed since the last setup or refresh
  int64_t n = 0;
  double stored = 0.0;  // operator entries the V-cycle reads (coarse levels: sum of rlen)
  double cheb_b = 0.0;  // Chebyshev smoother: Gershgorin bound of the spectrum of D^-1 A
};

struct AmgOptions {
  double theta = 0.08;     // strength threshold
  double omega = 0.85;     // Jacobi damping
  double coarse_scale = 1.5;  // over-correction of the piecewise-constant coarse correction
  int max_levels = 20;
  int coarsest = 160;      // stop coarsening at or below this size (shared-memory inverse)
  int npre = 1, npost = 1;
  double mis2_ratio = 0.85; // distance-2 aggregation where distance-1 sets keep more than this share of rows
  int mis2_from = 1 << 30;  // levels from this one on aggregate by distance-2 sets directly
  bool fp32 = false;       // V-cycle in single precision
  // smoother: 0 weighted Jacobi (omega), 1 Chebyshev polynomial in D^-1 A
  // on [b / cheb_ratio, b] with b each level's Gershgorin bound (degree npre
  // before and npost after the coarse correction; degree 1 is Jacobi with
  // the weight 2 / (b + b / cheb_ratio))
  int smoother = 0;
  double cheb_ratio = 4.0;
};

struct Amg : Precond {
  AmgOptions opt;
  std::vector<std::unique_ptr<AmgLevel>> lv;
  int nc = 0;                    // coarsest size
  DBuf<double> Ainv;             // [nc*nc] pinned inverse of the coarsest operator
  DBuf<uint64_t> rowhash;        // fingerprints of the fine rows the hierarchy was formed from
  DBuf<int32_t> clab;            // coarsest component labels
  DBuf<uint8_t> csing;           // per component: 1 if singular (row sums zero)
  DBuf<int32_t> fine_lab;        // labels of the fine rows
  int ncomp = 0;
  std::vector<uint8_t> sing_host;
  DBuf<double> csum, ccnt;       // per-component sums / counts (fine)
  DBuf<double> cpart;            // block partials for component sums
  ScanWork sw;
  bool ready = false;

  bool masked = false;            // the projection reads the fine labels (rows with label -1 take no part)
  int refreshes = 0;              // refreshes since the setup

  fvs_status setup(cudaStream_t s, const Ell& A);
  fvs_status count_stored(cudaStream_t s);   // AmgLevel::stored of every level
  // The operator's values changed on the same rows: rows of cells without
  // pressure (ppe[act[i]] == 0: frozen since the setup) leave their
  // aggregates and the null-space labels; rows that carry pressure without
  // an aggregate (cells melted again, or margin rows melted for the first
  // time) join the aggregate of their most strongly coupled neighbour and
  // take its label; the Galerkin rows of every aggregate whose member rows
  // changed (row fingerprints) are recomputed on the kept aggregation, level
  // by level.  The coarsest inverse of the setup is kept.
  // FVS_ERR_NOT_CONVERGED: the kept aggregation does not fit any more (a
  // coarse row outgrew its width, a row found no label, or two parts met),
  // so a new setup is needed.
  fvs_status refresh(cudaStream_t s, const int32_t* act, const uint8_t* ppe);
  fvs_status apply(cudaStream_t s, const double* r, double* z) override;
  uint64_t version = 0;          // bumped by every setup
  // coarsest inverse above the shared-memory size: one pivot and one
  // elimination launch per column, replayed as a captured graph (kept while
  // the level size and buffers stay the same)
  DBuf<double> gj_fac;
  DBuf<int32_t> gj_perm;
  DBuf<int> c_err, c_ncd;
  cudaGraphExec_t gj_exec = nullptr;
  uint64_t gj_key = 0;
  ~Amg() { if (gj_exec) cudaGraphExecDestroy(gj_exec); }
  uint64_t signature() const override {
    // Chebyshev weights are launch arguments: new bounds need a new graph
    return version * 2654435761ULL + (opt.fp32 ? 1 : 0) + (masked ? 2 : 0) +
           (opt.smoother == 1 ? bound_epoch * 4 : 0);
  }
  // subtract the component mean on every singular component (fine level)
  fvs_status project(cudaStream_t s, double* v);
  int levels() const { return (int)lv.size(); }

 private:
  // x0_ready: the level's first Jacobi iterate from zero is already in its x
  // (formed by the restriction from the level above)
  template <typename T>
  fvs_status vcycle_t(cudaStream_t s, int l, const T* b, T* y, bool x0_ready = false);
  fvs_status coarsest_setup(cudaStream_t s);
  fvs_status setup_fp32(cudaStream_t s);
  // Chebyshev smoother: Gershgorin bounds of every smoothed level (after a
  // setup or a refresh, when the operator values are final)
  fvs_status cheb_bounds(cudaStream_t s);
  double first_weight(const AmgLevel& L) const;   // weight of the first sweep
  DBuf<unsigned long long> gbound;
  uint64_t bound_epoch = 0;
};

struct AmgProjector : Projector {
  Amg* amg = nullptr;
  fvs_status apply(cudaStream_t s, double* v) override { return amg->project(s, v); }
};

// Pinned dense inverses of Sp coarsest systems at once (one block each):
// values of system s at val[(k*n + i)*Sp + s]; outputs Ainv[(i*n + j)*Sp + s],
// part labels lab[i*Sp + s], singular flags sing[c*Sp + s], part counts
// ncomp[s].  n must not exceed amg_smem_coarsest().
int amg_smem_coarsest();
fvs_status amg_coarsest_batched(cudaStream_t s, int n, int w, const int32_t* col, const double* val, int Sp,
                                double* Ainv, int32_t* lab, uint8_t* sing, int* ncomp, int* err);

}  // namespace fvs
