/*
 * fvs.h - C ABI of the GB300 finite-volume solidification solver.
 *
 * The library advances the fractional-step method of Shahane et al.,
 * "Finite Volume Simulation Framework for Die Casting with Uncertainty
 * Quantification" (arXiv:1810.08572), on unstructured hexahedral meshes:
 * momentum predictor with Boussinesq buoyancy and Darcy drag (Section 2.2,
 * Eq. 6), pressure Poisson equation on the liquid/mushy cells with the
 * coefficient smearing of Section 2.4.2 (Eq. 9, Eq. 15-16), consistent face
 * flux and velocity correction (Eq. 8, Eq. 17), and the energy equation with
 * latent heat by source linearisation (Eq. 4, Eq. 18-20, Section 2.4.4).
 *
 * Conventions for every entry point:
 *  - Every function returns an fvs_status; FVS_OK (0) on success.  No entry
 *    point aborts, traps or exits; fvs_last_error() gives a message for the
 *    last failure on the calling thread.
 *  - "host" pointers are plain CPU memory, "device" pointers are CUDA device
 *    memory of the GPU that was current when the object was created.
 *  - Inputs are copied; the caller keeps ownership of every buffer it
 *    passes.  The library owns (and frees in the destroy calls) all device
 *    memory it allocates.
 *  - A stream argument is a cudaStream_t passed as void* (NULL = legacy
 *    default stream).  All work of an object runs in order on its stream.
 *  - Field arrays exchanged with the caller are in the caller's (input)
 *    numbering of cells and faces, whatever reordering the mesh applied.
 *  - There is no CPU fallback: without a usable GPU the calls fail with
 *    FVS_ERR_CUDA.
 */
#ifndef FVS_H
#define FVS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FVS_OK = 0,
  FVS_ERR_ARG = 1,           /* bad argument (NULL, size, range)                 */
  FVS_ERR_MESH = 2,          /* mesh failed validation                          */
  FVS_ERR_CUDA = 3,          /* CUDA runtime error                              */
  FVS_ERR_NOMEM = 4,         /* device allocation failed                        */
  FVS_ERR_NOT_CONVERGED = 5, /* a solve stopped at its iteration limit; fields
                                are left consistent and the residual reported   */
  FVS_ERR_TIMEOUT = 6,       /* a bounded device wait ran out                   */
  FVS_ERR_STATE = 7          /* call out of order (e.g. step before properties) */
} fvs_status;

typedef struct fvs_mesh_s* fvs_mesh;
typedef struct fvs_solver_s* fvs_solver;
typedef struct fvs_surrogate_s* fvs_surrogate;   /* learned surrogate, see below */

/* Message for the last non-OK status returned on this thread (never NULL). */
const char* fvs_last_error(void);

/* Library version string, e.g. "fvs 0.1 sm_103a". */
const char* fvs_version(void);

/* Number of CUDA kernels this library has launched in the process so far
 * (all objects, all threads). */
int64_t fvs_launch_count(void);

/* ------------------------------------------------------------------------
 * Mesh (Section 2.3, Fig. 1).
 *   nodes_xyz      host  double [n_nodes*3]
 *   cell_nodes     host  int32  [n_cells*8]  hexahedron corners (VTK order)
 *   face_nodes     host  int32  [n_faces*4]  corners V1..V4 in cyclic order
 *                  with the right-hand normal 1/2 (V3-V1) x (V4-V2) pointing
 *                  from the owner C1 to the neighbour C2 (outward on walls);
 *                  V1V3 and V2V4 are the local eta and zeta axes of Eq. 12
 *   face_cells     host  int32  [n_faces*2]  (owner, neighbour), neighbour -1
 *                  on the boundary
 *   boundary_patch host  int32  [n_faces]    -1 interior, else wall patch id
 *                  0..63 (wall data are given per patch in fvs_props)
 *   reorder        1: renumber cells (Morton order of centres), vertices
 *                  and faces (by owner) for coalesced access; 0: keep input
 *                  order
 * Fails with FVS_ERR_MESH unless every cell has exactly six faces, every
 * interior face has two distinct owners, all ids are in range, and all
 * volumes and face areas are positive.
 * ------------------------------------------------------------------------ */
fvs_status fvs_mesh_create(const double* nodes_xyz, int64_t n_nodes,
                           const int32_t* cell_nodes, int64_t n_cells,
                           const int32_t* face_nodes, int64_t n_faces,
                           const int32_t* face_cells, const int32_t* boundary_patch,
                           int reorder, void* stream, fvs_mesh* out);
fvs_status fvs_mesh_destroy(fvs_mesh mesh);

/* Cell zones for castings in a mold (Section 2.4.4: the energy equation runs
 * on every cell; flow only in the metal).
 *   zone   host int32 [n_cells] in the caller's cell order: 0 metal, 1 mold
 * The zones take effect in solvers that are given a mold material
 * (fvs_set_mold); otherwise every cell is metal.  Call before
 * fvs_set_properties / fvs_set_mold of the solvers that use them.
 * FVS_ERR_ARG for values other than 0 and 1. */
fvs_status fvs_mesh_set_zones(fvs_mesh mesh, const int32_t* zone);

typedef struct {
  int64_t n_cells, n_faces, n_nodes, n_interior_faces;
  int32_t max_cell_neighbours; /* stencil width: cells sharing a vertex (27), or a face (7) on orthogonal meshes */
  int32_t max_face_neighbours; /* largest neighbour set N(f) of a face        */
  int32_t n_patches;           /* 1 + largest patch id                        */
  int32_t orthogonal;          /* 1 if no face carries cross diffusion        */
  double total_volume;
} fvs_mesh_info;
fvs_status fvs_mesh_get_info(fvs_mesh mesh, fvs_mesh_info* info);

/* Geometry in input numbering, for checking: which = 0 cell volumes [n_cells],
 * 1 face areas [n_faces]; dst is host memory of dst_len doubles. */
fvs_status fvs_mesh_geometry(fvs_mesh mesh, int which, double* dst, int64_t dst_len);

/* ------------------------------------------------------------------------
 * Material and run settings.
 *  Darcy drag D = darcy_C fs^2 / ((1 - fs)^3 + darcy_eps) (Eq. 3 with the
 *  dendrite spacing folded into darcy_C); buoyancy -rho beta (T - T_ref) g.
 *  Solid fraction (fs_model): FVS_FS_LINEAR, linear between T_sol and T_liq
 *  (Eq. 5 in its linear form; kp, T_f, T_eps unused), or FVS_FS_SCHEIL, the
 *  Gulliver-Scheil law fs = 1 - ((T - T_f)/(T_liq - T_f))^(1/(kp - 1)) of
 *  Eq. 5 smeared linearly across [T_sol - T_eps, T_sol + T_eps] (Eq. 21),
 *  which needs 0 < kp < 1, T_eps > 0 and T_sol + T_eps < T_liq < T_f.  Cells
 *  are liquid/mushy (flowing) while T > T_sol in both laws.  A zeroed
 *  struct tail selects the linear law.
 * ------------------------------------------------------------------------ */
enum { FVS_FS_LINEAR = 0, FVS_FS_SCHEIL = 1 };
typedef struct {
  double rho, k, cp, latent, T_sol, T_liq, mu, beta, T_ref;
  double g[3];
  double darcy_C, darcy_eps;
  int32_t fs_model;   /* FVS_FS_LINEAR or FVS_FS_SCHEIL                        */
  double kp;          /* partition coefficient (Scheil)                        */
  double T_f;         /* freezing temperature of the solvent, K (Scheil)       */
  double T_eps;       /* half-width of the smear band, K (Scheil)              */
} fvs_material;

/* Wall conditions of the energy equation (every wall is no-slip).
 *  FVS_BC_ADIABATIC   no heat flux
 *  FVS_BC_DIRICHLET   fixed wall temperature T; the wall's vertices take T
 *                     in the cross-diffusion terms (Eq. 11-12)
 *  FVS_BC_CONVECTIVE  heat-transfer coefficient h (W/m2 K) to an ambient
 *                     temperature T: the face carries the orthogonal flux
 *                     A (T - T_c)/(d/k_c + 1/h), d the distance from the cell
 *                     centre to the face centre and k_c the cell's
 *                     conductivity; the wall's vertices stay free (cell
 *                     means), as on adiabatic walls.  The paper fixes the
 *                     wall temperature (Section 4-5); this is the usual
 *                     film condition of a cooled die. */
enum { FVS_BC_ADIABATIC = 0, FVS_BC_DIRICHLET = 1, FVS_BC_CONVECTIVE = 2 };
typedef struct {
  int32_t type; /* FVS_BC_ADIABATIC, FVS_BC_DIRICHLET or FVS_BC_CONVECTIVE     */
  double T;     /* wall temperature, or the ambient temperature (K)            */
  double h;     /* FVS_BC_CONVECTIVE: heat-transfer coefficient (> 0)          */
} fvs_patch_bc;

enum { FVS_PREC_FP64 = 0, FVS_PREC_MIXED = 1 };
enum { FVS_PSOLVER_AMG = 0, FVS_PSOLVER_JACOBI = 1 };

typedef struct {
  fvs_material mat;
  int32_t n_patches;            /* entries in bc (>= the mesh's n_patches)      */
  const fvs_patch_bc* bc;       /* host, indexed by patch id                    */
  double T_init;                /* uniform initial temperature; fluid at rest   */
  double p_rtol;                /* pressure: ||b - A p||_2 / ||b||_2 target     */
  double mom_rtol;              /* momentum predictor relative residual target  */
  double e_rtol;                /* energy inner solve relative residual target  */
  double e_tol_T;               /* latent-heat loop: max |dT| stop rule (K)     */
  int32_t max_e_iters;          /* latent-heat loop limit                       */
  int32_t max_krylov_iters;     /* per linear solve                             */
  int32_t precision;            /* FVS_PREC_FP64 or FVS_PREC_MIXED              */
  int32_t p_solver;             /* FVS_PSOLVER_AMG (AMG-preconditioned Krylov,
                                   falling back to Jacobi BiCGStab on failure as
                                   in Section 2.5) or FVS_PSOLVER_JACOBI         */
  int32_t no_flow;              /* 1: natural convection off (Section 4 runs its
                                   castings without it): no momentum, pressure
                                   or correction step; u, fluxes and p stay 0
                                   and the energy equation is conduction with
                                   latent heat.  0: the full method            */
  int32_t n_k;                  /* points of a piecewise-linear conductivity
                                   k(T) of the metal (Section 3 uses a table;
                                   0: the constant mat.k), at most 16          */
  const double* k_T;            /* host [n_k] increasing temperatures (K)       */
  const double* k_val;          /* host [n_k] conductivities (W/m K), held
                                   constant outside the table.  Each step
                                   evaluates k per face at T^n: at the mean of
                                   the two cells, of the cell and a fixed wall
                                   value, or at the metal cell on convective
                                   walls and metal-mold faces; both
                                   Crank-Nicolson halves use it                */
} fvs_props;

fvs_status fvs_solver_create(fvs_mesh mesh, void* stream, fvs_solver* out);
fvs_status fvs_solver_destroy(fvs_solver solver);

/* Copies the settings and resets the state to the initial condition
 * (uniform T_init, u = 0, zero fluxes, time 0). */
fvs_status fvs_set_properties(fvs_solver solver, const fvs_props* props);

/* Mold material (zone-1 cells of fvs_mesh_set_zones): conduction only —
 * never liquid/mushy, no latent heat, no flow — with density rho (kg/m3),
 * heat capacity cp (J/kg K) and conductivity k (W/m K).  A face between a
 * metal and a mold cell carries the orthogonal conductive flux
 * A (T_2 - T_1) / (d_1/k_1 + 1/h + d_2/k_2), d_i the distance from cell
 * centre i to the face centre and h (W/m2 K) the interface heat-transfer
 * coefficient; faces inside a zone use that zone's k.  Resets the state as
 * fvs_set_properties does, with the mold cells at T_init (K).  A later
 * fvs_set_properties removes the mold again.  FVS_ERR_STATE before
 * fvs_set_properties; FVS_ERR_ARG for non-positive rho, cp, k or h. */
fvs_status fvs_set_mold(fvs_solver solver, double rho, double cp, double k, double h, double T_init);

/* Grain growth (Eq. 24-26): while a metal cell is mushy (0 < fs < 1) its
 * grain radius r grows by d(r^2)/dt = lambda_s^2 D_s, integrated by the
 * trapezoidal rule between the solid fractions at both ends of each step.
 * lambda_s = -S/(2 sqrt(pi)) + sqrt(S^2/(4 pi) - S) with the supersaturation
 * S = 2 (C_l - C_0)/(C_s - C_l) of the Scheil interface contents
 * C_l = C_0 (1 - fs)^(kp - 1), C_s = kp C_l (C_0 cancels; the sign is the one
 * that keeps lambda_s real).  kp: partition coefficient (0 < kp < 1), D_s:
 * solute diffusion coefficient in the liquid (m2/s, >= 0; 0 switches growth
 * off), r0: initial radius (m, >= 0).  Resets every metal cell to r0 now and
 * whenever the state is reset; stays set across fvs_set_properties.
 * FVS_ERR_STATE before fvs_set_properties; FVS_ERR_ARG otherwise. */
fvs_status fvs_set_grain_growth(fvs_solver solver, double kp, double D_s, double r0);

/* Overwrite the state with a given temperature field (and velocity, or NULL
 * for rest): T^n = T^{n-1} = T, fs = fs(T), u^n = u^{n-1} = u (zero in solid
 * cells), fluxes and pressure zero, time 0, crossing times reset.
 * T [n_cells], u [n_cells*3] (x,y,z per cell); on_device selects the memory
 * space of both. */
fvs_status fvs_set_state(fvs_solver solver, const double* T, const double* u, int on_device);

typedef struct {
  int64_t n_active;   /* liquid + mushy cells (rows of momentum)            */
  int64_t n_ppe;      /* cells in the pressure system                        */
  int32_t mom_its;    /* Krylov iterations, sum of the three components      */
  int32_t p_its;      /* pressure Krylov iterations                          */
  int32_t e_its;      /* latent-heat loop passes                             */
  int32_t e_lin_its;  /* energy Krylov iterations, summed over passes        */
  double p_relres;    /* final pressure relative residual                    */
  int32_t fallback;   /* 1 if the pressure solve fell back to Jacobi BiCGStab */
  int32_t n_components; /* connected parts of the pressure system            */
  int32_t amg_levels;
  int32_t status;     /* fvs_status of the step                              */
  int32_t p_rebuilt;  /* pressure system of this step: 0 reused unchanged
                         (no cell changed phase), 1 renumbered with the AMG
                         hierarchy built anew, 2 reassembled on the kept
                         numbering with the hierarchy refreshed on its fine
                         level (cells only froze)                             */
  double setup_ms;    /* host wall time of that rebuild (0 if reused)        */
} fvs_step_stats;

/* Advance n_steps time steps of size dt (Section 2.2, steps 1-5 plus the
 * crossing-time bookkeeping for Eq. 22-23).  'last' (nullable, host) gets the
 * statistics of the final step.  Returns FVS_ERR_NOT_CONVERGED if a solve hit
 * its iteration limit (the step is still completed). */
fvs_status fvs_step(fvs_solver solver, double dt, int32_t n_steps, fvs_step_stats* last);

/* Solve the pressure system of the current state's active set (tags of the
 * last step, Section 2.4.2) for a given right side.
 *   rhs    device double [n_cells], input numbering; entries of cells outside
 *          the pressure system are ignored
 *   p_out  device double [n_cells]; zero outside the pressure system, zero
 *          mean on each connected part
 * The right side is projected to zero sum on each connected part.  The
 * system is A p = rhs with A p = sum over flowing faces of
 * (A_f / rho) (n . grad p)_f (Eq. 9 left side). */
fvs_status fvs_pressure_solve(fvs_solver solver, const double* rhs, double* p_out,
                              double rtol, int32_t* iters, double* relres);

typedef enum {
  FVS_T = 0,       /* temperature [n_cells]                                   */
  FVS_FS = 1,      /* solid fraction [n_cells]                                */
  FVS_U = 2,       /* velocity [n_cells*3]                                    */
  FVS_P = 3,       /* pressure [n_cells]                                      */
  FVS_FLUX = 4,    /* face volume flux owner->neighbour [n_faces]             */
  FVS_TAG = 5,     /* 1 liquid/mushy, 0 solid, as double [n_cells]            */
  FVS_QOI = 6,     /* per cell: t_f, cooling rate, SDAS (um), yield (MPa)
                      [n_cells*4]; NaN where the cell has not solidified      */
  FVS_USTAR = 7,   /* predictor velocity u* of the last step [n_cells*3]      */
  FVS_CROSS = 8,   /* liquidus / solidus crossing times [n_cells*2], -1 unset */
  FVS_FACE_CASE = 9, /* pressure face case 0 wall,1,2,3 as double [n_faces]  */
  FVS_GRAIN = 10   /* grain radius in m [n_cells] (fvs_set_grain_growth), 0 in
                      the mold                                                */
} fvs_field;

/* Copy a field (double values, input numbering) into dst (dst_len doubles,
 * host or device per dst_on_device). */
fvs_status fvs_query_fields(fvs_solver solver, fvs_field field, double* dst,
                            int64_t dst_len, int dst_on_device);

/* ------------------------------------------------------------------------
 * Batched uncertainty quantification (Section 2.7: non-intrusive sampling of
 * the stochastic inputs, one plain solve per sample; Section 5: melt
 * temperature, wall temperature and solute content as the inputs).
 *   base      host: material and solver settings shared by all samples
 *             (its bc and T_init are replaced per sample: every wall patch
 *             is held at the sample's wall temperature)
 *   inputs    host double [n_samples*3], per sample: melt temperature (K),
 *             wall temperature (K), solute concentration C0 (wt%)
 *   dt        time step (s); each sample starts at rest at its melt
 *             temperature and runs until a step starts with every cell solid,
 *             or for max_steps steps
 *   opt       host, nullable (NULL: the zero-initialised options)
 *   qoi_out   host double [n_samples*4], per opt->qoi_kind:
 *             FVS_QOI_MEANS: means over the solidified cells of the local
 *               solidification time t_f (s), cooling rate (K/s), SDAS (um)
 *               and yield strength (MPa) (Eq. 22-23); NaN if no cell
 *               solidified
 *             FVS_QOI_EXTREMES: the four outputs of Section 5, taken over
 *               the whole domain: total solidification time (the latest
 *               solidus crossing, s; NaN while a cell is still above the
 *               solidus), maximum SDAS (um), minimum yield strength (MPa)
 *               and maximum grain radius (m; 0 without grain growth)
 *   steps_out host int64 [n_samples] steps taken, 0 for samples the surrogate
 *             answered (nullable)
 * Options:
 *   mode      FVS_UQ_LOCKSTEP (0): all samples advance together, every
 *             field stored [row][sample], one launch per phase for all
 *             samples, shared operators and AMG aggregation, per-sample
 *             pressure rows and coarse values (needs a coarsest AMG level of
 *             at most 160 rows on the all-liquid pressure operator, else
 *             FVS_ERR_NOT_CONVERGED; a k(T) table needs FVS_UQ_STREAMS);
 *             FVS_UQ_STREAMS (1): independent solves, each on its own CUDA
 *             stream and solver;
 *             FVS_UQ_SURROGATE (2): the trained models answer every sample
 *             inside the box [box_lo, box_hi] whose ensemble agrees (the
 *             spread of the models' predictions, standard deviation over
 *             models divided by the magnitude of their mean, at most
 *             max_spread for every output; max_spread <= 0 skips the test);
 *             the other samples fall back to plain solves in plain_mode.
 *             The models must have been trained on this qoi_kind.
 *   n_streams FVS_UQ_STREAMS: concurrent samples (0 = 8)
 *   liquidus_T0, liquidus_slope
 *             the sample's liquidus T_liq = liquidus_T0 + liquidus_slope C0
 *             (a straight liquidus line; Section 5 reads it off the Al-Si
 *             phase diagram, with liquidus_T0 the solvent's freezing point);
 *             both 0: every sample keeps base->mat.T_liq.  FVS_ERR_ARG if a
 *             sample's liquidus does not suit the solid-fraction law
 *   grain_kp, grain_Ds, grain_r0
 *             grain growth in every sample as fvs_set_grain_growth
 *             (grain_Ds = 0: off)
 *   models, n_models, box_lo, box_hi [3], max_spread, plain_mode
 *             FVS_UQ_SURROGATE only (plain_mode LOCKSTEP or STREAMS)
 *   used_plain host int32 [n_samples] out (nullable): 1 where the sample
 *             was solved plainly
 *   T_out, p_out [n_samples*n_cells], u_out [n_samples*n_cells*3]
 *             host, nullable: each plainly solved sample's final
 *             temperature, pressure and velocity (x,y,z per cell) in the
 *             caller's cell order (rows of surrogate samples are untouched)
 * Blocks until all samples are done.
 * ------------------------------------------------------------------------ */
enum { FVS_UQ_LOCKSTEP = 0, FVS_UQ_STREAMS = 1, FVS_UQ_SURROGATE = 2 };
enum { FVS_QOI_MEANS = 0, FVS_QOI_EXTREMES = 1 };
typedef struct {
  int32_t mode;
  int32_t n_streams;
  int32_t qoi_kind;
  double liquidus_T0;
  double liquidus_slope;
  double grain_kp, grain_Ds, grain_r0;
  int32_t n_models;
  const fvs_surrogate* models;
  const double* box_lo;
  const double* box_hi;
  double max_spread;
  int32_t plain_mode;
  int32_t* used_plain;
  double* T_out;
  double* u_out;
  double* p_out;
} fvs_uq_options;
fvs_status fvs_uq_batch(fvs_mesh mesh, const fvs_props* base, int64_t n_samples, const double* inputs,
                        double dt, int32_t max_steps, const fvs_uq_options* opt, double* qoi_out,
                        int64_t* steps_out);

/* ------------------------------------------------------------------------
 * Learned surrogate of the UQ map (the role the polynomial-chaos expansion
 * of Section 2.7, Eq. 27-28, plays in the paper): a multilayer perceptron
 * from the stochastic process inputs to the microstructure outputs of
 * Section 2.6 (Eq. 22-23).  Hidden layers GELU(W h + b), linear output,
 * mean-squared-error loss on standardised inputs and outputs.  BF16 weights
 * and activations with FP32 accumulation on the tensor cores; FP32 master
 * weights and Adam.  Parameters are exchanged as one flat host array of
 * doubles: for each layer its weight matrix [n_out x n_in] row-major, then
 * its bias [n_out].
 * ------------------------------------------------------------------------ */
/* n_in, n_hidden, n_out in 1..128, 1..16 hidden layers; weights drawn
 * uniform(-sqrt(6/fan_in), +sqrt(6/fan_in)) from a counter-based generator
 * keyed by seed, biases zero; scaling is the identity until set. */
fvs_status fvs_surrogate_create(int32_t n_in, int32_t n_hidden, int32_t n_hidden_layers, int32_t n_out,
                                uint64_t seed, void* stream, fvs_surrogate* out);
fvs_status fvs_surrogate_destroy(fvs_surrogate s);
/* Standardisation: x' = (x - mu_in)/sd_in, y = y' sd_out + mu_out (host arrays
 * of n_in and n_out doubles; scales must be positive). */
fvs_status fvs_surrogate_set_scaling(fvs_surrogate s, const double* mu_in, const double* sd_in,
                                     const double* mu_out, const double* sd_out);
/* Number of parameters in the flat layout, or -1 for a NULL handle. */
int64_t fvs_surrogate_num_params(fvs_surrogate s);
/* set = 1: load the flat host array into the model; set = 0: read it out. */
fvs_status fvs_surrogate_params(fvs_surrogate s, double* inout, int64_t len, int set);
/* Loss (mean over samples and outputs of the squared standardised error) and
 * its gradient with respect to the flat parameters at the current weights.
 * X host [n x n_in], T host [n x n_out], grad host [len]. */
fvs_status fvs_surrogate_gradients(fvs_surrogate s, const double* X, const double* T, int64_t n, double* grad,
                                   int64_t grad_len, double* loss);
/* Full-batch Adam (beta 0.9 / 0.999, eps 1e-8) for the given epochs;
 * final_loss (nullable) gets the loss after training. */
fvs_status fvs_surrogate_train(fvs_surrogate s, const double* X, const double* T, int64_t n, int32_t epochs,
                               double lr, double* final_loss);
/* Y [n x n_out] = model(X [n x n_in]); both host or both device memory. */
fvs_status fvs_surrogate_predict(fvs_surrogate s, const double* X, double* Y, int64_t n, int on_device);

/* ------------------------------------------------------------------------
 * Polynomial chaos surrogate (the paper's own: Section 2.7, Eq. 27-28, and
 * the total Sobol indices of Section 5).  An output is expanded in products
 * of orthonormal polynomials of the standardised inputs, truncated at a
 * total degree: probabilists' Hermite He_n/sqrt(n!) of (x - mean)/sd for a
 * normal input (the paper's inputs), Legendre sqrt(2n+1) P_n of
 * (2x - lo - hi)/(hi - lo) for a uniform one.  Terms are ordered by total
 * degree, then by their multi-indices with the last input varying fastest.
 * The coefficients solve the Vandermonde system of Eq. 28 in the least-
 * squares sense (normal equations, Cholesky, two refinement steps on the
 * Vandermonde residual), on the GPU.
 * ------------------------------------------------------------------------ */
enum { FVS_PCE_NORMAL = 0, FVS_PCE_UNIFORM = 1 };
typedef struct fvs_pce_s* fvs_pce;
/* n_in inputs (1..8) with family[j] and parameters (p1, p2)[j] = (mean, sd)
 * or (lo, hi), host arrays; total degree 0..24; n_out outputs (1..8). */
fvs_status fvs_pce_create(int32_t n_in, const int32_t* family, const double* p1, const double* p2,
                          int32_t degree, int32_t n_out, void* stream, fvs_pce* out);
fvs_status fvs_pce_destroy(fvs_pce p);
/* Number of expansion terms, or -1 for a NULL handle. */
int64_t fvs_pce_num_terms(fvs_pce p);
/* Multi-indices, host int32 [num_terms*n_in] (degree of input j in term k at
 * k*n_in + j). */
fvs_status fvs_pce_multi_indices(fvs_pce p, int32_t* alpha, int64_t len);
/* Collocation points in the inputs' units (Section 2.7: roots of the basis
 * polynomials): sparse = 0, the tensor product of level-point rules
 * (level^n_in points; Section 5 uses levels 3 and 6, 27 and 216 points);
 * sparse = 1, Smolyak's combination of the level-i rules with i points over
 * max(n_in, level) <= |i| <= level + n_in - 1.  X (host [cap*n_in]) may be
 * NULL to count the points into *n. */
fvs_status fvs_pce_nodes(fvs_pce p, int32_t level, int32_t sparse, double* X, int64_t cap, int64_t* n);
/* Fit to m runs: X host [m*n_in], Y host [m*n_out]; m >= num_terms.
 * rms_resid (nullable) gets the root-mean-square residual of the fit.
 * FVS_ERR_ARG when the points do not determine the coefficients. */
fvs_status fvs_pce_fit(fvs_pce p, const double* X, const double* Y, int64_t m, double* rms_resid);
/* Y [n*n_out] = expansion at X [n*n_in]; both host or both device. */
fvs_status fvs_pce_eval(fvs_pce p, const double* X, double* Y, int64_t n, int on_device);
/* Coefficients, host [num_terms*n_out] (term k, output q at k*n_out + q). */
fvs_status fvs_pce_coefficients(fvs_pce p, double* c, int64_t len);
/* From the coefficients: mean and variance per output (host [n_out]) and
 * the total and first-order Sobol indices (host [n_out*n_in]); any pointer
 * may be NULL. */
fvs_status fvs_pce_sensitivity(fvs_pce p, double* mean, double* var, double* total, double* first);

/* ------------------------------------------------------------------------
 * Kernel timing (not part of the method; for roofline measurement).
 * While enabled, every launch of the SpMV, residual and Jacobi kernels on the
 * fine pressure, energy and momentum matrices inside fvs_step is bracketed by
 * CUDA events on the solver's stream and credited with its algorithmic bytes
 * (matrix values and column ids once, each vector entry once).
 * fvs_profile_enable clears the records.  fvs_profile_read waits for the
 * stream, then writes up to max_records aggregates (host memory) and sets
 * *n_records to the number of kernel classes seen.
 * ------------------------------------------------------------------------ */
typedef struct {
  char name[48];      /* kernel@matrix, e.g. "spmv@pressure"               */
  int64_t launches;
  double total_ms;    /* summed event time of the launches                 */
  double bytes;       /* summed algorithmic bytes of the launches          */
} fvs_kernel_time;
fvs_status fvs_profile_enable(fvs_solver solver, int on);
fvs_status fvs_profile_read(fvs_solver solver, fvs_kernel_time* out, int32_t max_records, int32_t* n_records);

/* Same values and argument meaning as fvs_query_fields with a host
 * destination, for callers that must not allocate GPU memory (the paper has
 * no counterpart: this is a service of the library).  fvs_query_fields
 * stages the reordered field in a temporary device buffer; a caller that
 * samples a running simulation from a thread that must not block on or fail
 * in the allocator, or that runs with its device memory already fully
 * committed, cannot afford that.  This entry point stages the field in a
 * fixed device array built into the library instead, and calls no
 * allocating routine.
 *   dst  host memory of dst_len doubles
 * Limit: fields of at most 1,048,576 values; larger fields fail with
 * FVS_ERR_ARG (use fvs_query_fields).  The staging array (8 MiB) is placed on
 * a GPU, and its device address looked up, by the first fvs_solver_create on
 * that GPU (create solvers before any CUDA stream capture); it stays there
 * until the process exits, so this call itself allocates nothing.  All calls
 * share the array: each call overwrites every value it returns, and calls
 * whose GPU work overlaps (other streams, other threads) race on it. */
fvs_status fvs_query_fields_noalloc(fvs_solver solver, fvs_field field, double* dst, int64_t dst_len);

/* Measured FP64 fused-multiply-add rate of the current GPU (GFLOP/s, two
 * flops per FMA): eight independent FMA chains per thread, 8 blocks of 256
 * threads per SM, iters FMAs per chain, timed with CUDA events.  Not part
 * of the method: the roof that FP64 sparse kernels meet next to the copy
 * bandwidth. */
fvs_status fvs_measure_fp64_fma(int64_t iters, double* gflops);

/* Current simulated time and step count. */
fvs_status fvs_get_time(fvs_solver solver, double* time, int64_t* steps);

#ifdef __cplusplus
}
#endif
#endif /* FVS_H */
