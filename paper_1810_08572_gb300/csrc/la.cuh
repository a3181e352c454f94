// Sparse linear algebra of the solver: ELL matrices, SpMV, deterministic
// reductions, Jacobi, and the Krylov drivers (BiCGStab, CG).
#pragma once

#include "common.cuh"

namespace fvs {

// ELL matrix stored slot-major: entry k of row i at [k*n + i], so that one
// thread per row reads consecutive addresses across a warp.  Unused slots
// hold col = i and val = 0.
struct Ell {
  int64_t n = 0;
  int w = 0;
  DBuf<int32_t> col;
  DBuf<double> val;
  DBuf<double> diag;   // diagonal (Jacobi)
  DBuf<float> valf;    // FP32 copies for the mixed-precision V-cycle
  DBuf<float> diagf;
  fvs_status alloc(int64_t rows, int width) {
    n = rows;
    w = width;
    FVS_TRY(col.alloc((size_t)rows * width + 1));
    FVS_TRY(val.alloc((size_t)rows * width + 1));
    FVS_TRY(diag.alloc((size_t)rows + 1));
    return FVS_OK;
  }
};

// Scalar slots of the Krylov drivers (device memory).
enum Slot {
  S_RHO = 0, S_RHO_OLD, S_ALPHA, S_OMEGA, S_RV, S_TS, S_TT, S_RR, S_BB, S_RZ, S_RZ_OLD, S_PQ,
  S_TMP0, S_TMP1, S_TOL2, S_ITER, S_FIRST, S_NSLOT
};

// Reduction scratch owned by a solver: block partials + scalar slots +
// pinned host mirror.
struct Reducer {
  int blocks = 0;
  DBuf<double> part;   // [2*blocks]
  DBuf<double> sc;     // [S_NSLOT]
  DBuf<unsigned int> ticket;   // last-block counter of the fused reductions
  DBuf<int> iter;              // iteration counter of device-driven solve loops
  double* host = nullptr;  // pinned [S_NSLOT]
  fvs_status init();
  ~Reducer() { if (host) cudaFreeHost(host); }
  // out[slot] = x . y  (deterministic: fixed blocks, fixed order)
  fvs_status dot(cudaStream_t s, int64_t n, const double* x, const double* y, int slot);
  // two dots in one pass: sc[s0] = a.b, sc[s1] = c.d
  fvs_status dot2(cudaStream_t s, int64_t n, const double* a, const double* b,
                  const double* c, const double* d, int s0, int s1);
  fvs_status max_abs_diff2(cudaStream_t s, int64_t n, const double* a, const double* b,
                           const double* c, const double* d, int s0, int s1);
  fvs_status fetch(cudaStream_t s);   // copies sc -> host and waits
};

// y = A x (+ dextra .* x if dextra)
fvs_status spmv(cudaStream_t s, const Ell& A, const double* x, double* y, const double* dextra = nullptr);
// r = b - A x (- dextra .* x)
fvs_status residual(cudaStream_t s, const Ell& A, const double* x, const double* b, double* r,
                    const double* dextra = nullptr);

// Preconditioner interface: z = M^-1 r.
struct Precond {
  virtual ~Precond() {}
  virtual fvs_status apply(cudaStream_t s, const double* r, double* z) = 0;
  // identifies the state the launches depend on (a captured iteration is
  // replayed only while it is unchanged)
  virtual uint64_t signature() const = 0;
};

// One Krylov iteration captured as a CUDA graph and replayed while the
// operator, vectors and preconditioner stay the same.
struct IterGraph {
  cudaGraphExec_t exec = nullptr;
  uint64_t key = 0;
  unsigned long long kernels = 0;   // launches per replay (for the launch counter)
  bool disabled = false;
  // whole-solve loop: a conditional while-node whose body is one iteration
  cudaGraphExec_t loop = nullptr;
  uint64_t loop_key = 0;
  unsigned long long loop_kernels = 0;
  bool loop_disabled = false;
  ~IterGraph() { reset(); }
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    key = 0;
    if (loop) cudaGraphExecDestroy(loop);
    loop = nullptr;
    loop_key = 0;
  }
};
bool graphs_enabled();

// Jacobi: z = r / (diag + dextra)
struct JacobiPrecond : Precond {
  const Ell* A = nullptr;
  const double* dextra = nullptr;
  const double* dinv = nullptr;   // optional 1 / (diag + dextra), kept by the caller: z = dinv r
  fvs_status apply(cudaStream_t s, const double* r, double* z) override;
  uint64_t signature() const override {
    return (uint64_t)(uintptr_t)A->diag.p * 31u + (uint64_t)(uintptr_t)dextra * 17u +
           (uint64_t)(uintptr_t)dinv * 13u + (uint64_t)A->n;
  }
};

// Line preconditioner: z = P^-1 r with P the diagonal (plus dextra) and the
// couplings along chains of cells, each cell joined to the neighbours it is
// most strongly coupled to where that choice is mutual (a row's two largest
// off-diagonal magnitudes).  Strongly anisotropic cells (thin in one
// direction) make those chains lines across the thin direction, where
// Jacobi converges slowly.  P restricted to one chain is tridiagonal and is
// solved exactly; cells on no chain take the Jacobi step.  The chains are
// found once from the operator (build) and stored 32 lines to a group,
// position-major within the group, so a warp's loads at one position are
// contiguous; factor() recomputes the tridiagonal factors from the current
// values, apply() does one forward and one backward substitution per line.
struct LinePrecond : Precond {
  const Ell* A = nullptr;
  const double* dextra = nullptr;   // extra diagonal at factor() time (or null)
  int64_t n = 0;
  int w = 0;
  const int32_t* built_from = nullptr;   // column array the chains were found in
  int64_t nlines = 0, ngroups = 0, padded = 0;
  int max_len = 0;
  DBuf<int64_t> goff;      // [ngroups] first entry of each group
  DBuf<int32_t> llen;      // [ngroups * 32] length of each line (0: no line)
  DBuf<int32_t> cell;      // [padded] cell at (group, position, lane)
  DBuf<int8_t> sprev, snext;   // slot of the previous / next cell of the line in the cell's row (-1: none)
  DBuf<double> lo, inv, cp;    // sub-diagonal, 1 / pivot, super-diagonal / pivot
  bool ready = false;
  fvs_status build(cudaStream_t s, const Ell& A);
  fvs_status factor(cudaStream_t s);
  fvs_status apply(cudaStream_t s, const double* r, double* z) override;
  uint64_t signature() const override { return (uint64_t)(uintptr_t)inv.p * 29u + (uint64_t)n; }
};

struct KrylovWork {
  DBuf<double> r, rh, p, ph, v, sv, sh, t, z, q;
  fvs_status ensure(int64_t n);
};

struct SolveResult {
  int iters = 0;
  double relres = 0.0;
  bool converged = false;
};

// Right-preconditioned BiCGStab on A x = b (x holds the initial guess).
// proj: optional projection applied to the right side and residual updates
// (null-space handling of the pressure system).
struct Projector {
  virtual ~Projector() {}
  virtual fvs_status apply(cudaStream_t s, double* v) = 0;
};

// The residual is measured against max(||b||, bnorm_floor).
fvs_status bicgstab(cudaStream_t s, Reducer& red, KrylovWork& w, const Ell& A, const double* dextra,
                    Precond& M, const double* b, double* x, double rtol, int maxit,
                    Projector* proj, SolveResult& res, double bnorm_floor = 0.0, IterGraph* graph = nullptr);
fvs_status pcg(cudaStream_t s, Reducer& red, KrylovWork& w, const Ell& A, Precond& M,
               const double* b, double* x, double rtol, int maxit, Projector* proj, SolveResult& res,
               IterGraph* graph = nullptr);

// small vector kernels
fvs_status vcopy(cudaStream_t s, int64_t n, const double* a, double* b);
fvs_status vfill(cudaStream_t s, int64_t n, double v, double* a);

}  // namespace fvs
