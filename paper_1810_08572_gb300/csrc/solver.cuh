// Solver state and the time step (Section 2.2, steps 1-5).
#pragma once

#include "amg.cuh"
#include "mesh.cuh"
#include "scan.cuh"

template <typename T>
inline void dswap(fvs::DBuf<T>& a, fvs::DBuf<T>& b) {
  T* p = a.p; size_t n = a.n;
  a.p = b.p; a.n = b.n;
  b.p = p; b.n = n;
}

namespace fvs {
// Connected parts of the pressure system found on the GPU from the pattern
// of its matrix, for the single-grid solve (Section 2.5: each liquid pocket
// is a separate singular block): the right side and the result are
// projected to zero mean on each part, as the AMG path does with the labels
// of its coarsest level.
struct PartProjector : Projector {
  DBuf<int32_t> par, root_flag, root_id, lab;
  DBuf<double> sum, cnt;
  DBuf<int> changed;
  int ncomp = 0;
  // labels of the rows i with ppe[act[i]] (the others are identity rows and
  // stay out of every part)
  fvs_status setup(cudaStream_t s, const Ell& K, const int32_t* act, const uint8_t* ppe, ScanWork& sw);
  fvs_status apply(cudaStream_t s, double* v) override;
};
}  // namespace fvs

struct fvs_solver_s {
  fvs_mesh mesh = nullptr;
  cudaStream_t stream = nullptr;
  bool have_props = false;
  bool have_step = false;     // tags / compact systems of a step exist
  bool k_valid = false;       // pressure system and AMG match the current tags
  bool numbered = false;      // map/act hold a system numbering
  bool renumbered = false;    // this step made a new numbering
  bool force_full = false;    // next step renumbers and rebuilds the hierarchy
  bool amg_full = false;      // the hierarchy was built (not refreshed) this step
  int steps_since_setup = 0;
  int p_its_ref = 0;          // pressure iterations right after the last full setup
  int64_t nlm = 0;            // liquid + mushy cells
  fvs_props props{};
  std::vector<fvs_patch_bc> bc;
  // mold zone (conduction only) and the metal-mold interface coefficient
  bool has_mold = false;
  double mold_rho = 0.0, mold_cp = 0.0, mold_k = 0.0, mold_h = 0.0, mold_T = 0.0;
  // grain growth (Eq. 24-26): r^2 per cell
  bool grain_on = false;
  double grain_kp = 0.0, grain_Ds = 0.0, grain_r0 = 0.0;
  fvs::DBuf<double> r2;
  // inverse Jacobi diagonals of the energy system (per latent-heat pass) and
  // of the momentum system (per step)
  fvs::DBuf<double> jinv_e, jinv_m;
  // line preconditioner of the energy system (FVS_ENERGY_LINES=1 instead of
  // Jacobi): chains found once from the energy operator, factors per pass
  fvs::LinePrecond eline;
  double time = 0.0;
  int64_t nstep = 0;

  // state (mesh numbering); vectors of 3 are stored component-major [3*Nc]
  fvs::DBuf<double> T, Told, Tnew, fs, fsnew;
  fvs::DBuf<double> u, uold, unew, ustar;
  fvs::DBuf<double> F, Fold, Fnew;
  fvs::DBuf<double> p, tliq, tsol;

  // wall data and the energy operator (-k/2 times the unit operator)
  fvs::DBuf<int32_t> bc_type;
  fvs::DBuf<double> bc_T, bc_h;
  // k(T) of the metal: piecewise linear table (n_k = 0: constant mat.k)
  int n_k = 0;
  double k_T[16] = {0}, k_val[16] = {0};
  fvs::DBuf<uint8_t> metal;        // [Nc] 1 metal, 0 mold
  fvs::DBuf<double> rcp, rL;       // [Nc] rho cp and rho L (0 in the mold)
  fvs::DBuf<double> kface, gint;   // [Nf] face conductivity, interface conductance
  fvs::Ell LT;            // unit temperature operator
  fvs::DBuf<double> lT;   // its constant part from fixed-temperature walls
  fvs::Ell Ke;            // -k/2 LT

  // active set
  fvs::DBuf<uint8_t> lm, ppe, flow, fcase;
  fvs::DBuf<int32_t> flag, excl, map, act, nS;
  int64_t nact = 0, nppe = 0;
  int64_t nmargin = 0;    // rows of the numbering beyond the LM cells when it was made
  fvs::ScanWork sw;

  // compact systems
  fvs::Ell M;             // momentum predictor on LM cells
  fvs::Ell K;             // pressure: K = -A on LM cells (identity rows for non-flowing)
  fvs::Ell Kp;            // K's diagonal and face couplings, the rest lumped (AMG operator)
  bool pc_compact = false;        // the hierarchy was built on Kp
  fvs::DBuf<double> mrhs, mx;     // [3*nact]
  fvs::DBuf<double> prhs, px;     // [nact]
  fvs::DBuf<double> pv, fSv;      // vertex pressure sums / solid fractions [Nv]
  fvs::DBuf<double> gradf;        // [3*Nf]

  // energy work
  fvs::DBuf<double> ebase, erhs, edx, Tlin, Tit, fsit;
  fvs::DBuf<int> cnt;

  fvs::Reducer red;
  fvs::KrylovWork kw;
  fvs::Amg amg;
  fvs::AmgProjector aproj;
  fvs::PartProjector pparts;      // parts of the system for the single-grid solve
  bool amg_ok = false;
  int amg_levels = 0;
  int ncomp = 0;
  fvs_step_stats last{};
  fvs::Prof prof;
  fvs::IterGraph g_p, g_e, g_m[3];   // captured Krylov iterations
};

namespace fvs {
fvs_status solver_alloc(fvs_solver s);
// places the staging array of fvs_query_fields_noalloc on the current device
fvs_status noalloc_reserve();
fvs_status solver_set_properties(fvs_solver s, const fvs_props* p);
fvs_status solver_set_mold(fvs_solver s, double rho, double cp, double k, double h, double T_init);
fvs_status solver_set_grain(fvs_solver s, double kp, double D_s, double r0);
fvs_status solver_set_state(fvs_solver s, const double* T, const double* u, int on_device);
fvs_status solver_step(fvs_solver s, double dt, fvs_step_stats* st);
fvs_status solver_pressure_solve(fvs_solver s, const double* rhs, double* p_out, double rtol, int* iters,
                                 double* relres);
fvs_status solver_query(fvs_solver s, fvs_field f, double* dst, int64_t len, int on_device);
// What a plain UQ run computes besides the solves: the samples' liquidus
// temperatures, which outputs, grain growth, and the optional final fields
struct UqSpec {
  std::vector<double> T_liq;            // per sample
  int qoi_kind = FVS_QOI_MEANS;
  double grain_kp = 0.0, grain_Ds = 0.0, grain_r0 = 0.0;
  double* T_out = nullptr;              // host [n*Nc], input numbering (nullable)
  double* u_out = nullptr;              // host [n*Nc*3]
  double* p_out = nullptr;              // host [n*Nc]
};
fvs_status uq_batch(fvs_mesh mesh, const fvs_props* base, int64_t n, const double* inputs, double dt,
                    int max_steps, int n_streams, const UqSpec& spec, double* qoi, int64_t* steps);
fvs_status surrogate_dims(fvs_surrogate s, int* nin, int* nout);
// FVS_UQ_SURROGATE: the ensemble answers the samples it can, plain solves
// (lockstep or streams per opt->plain_mode) the rest
fvs_status uq_surrogate(fvs_mesh mesh, const fvs_props* base, int64_t n, const double* inputs, double dt,
                        int max_steps, const fvs_uq_options& opt, const UqSpec& spec, double* qoi, int64_t* steps);
}  // namespace fvs
