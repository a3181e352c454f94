// Batched uncertainty quantification (Section 2.7: the stochastic inputs are
// sampled and each sample is a plain deterministic solve; Section 2.6 gives
// the per-cell microstructure outputs, Eq. 22-23).
//
// Samples share one read-only device mesh.  Each worker owns a solver on
// its own CUDA stream and takes samples from a shared counter, so the
// latency-bound parts of one sample (Krylov convergence checks, small AMG
// levels, launch gaps) overlap with the bandwidth-bound parts of others.
// All allocations are stream-ordered, so workers never synchronise the
// device as a whole.
#include <atomic>
#include <cmath>
#include <thread>
#include <vector>

#include "solver.cuh"

namespace fvs {

#define GS(i, n) for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// sums over solidified cells of t_f, cooling rate, SDAS, yield and the count
__global__ void k_qoi_part(int64_t Nc, const double* tliq, const double* tsol, double Ts, double Tl, double* part) {
  __shared__ double sh[32];
  double a[5] = {0, 0, 0, 0, 0};
  GS(c, Nc) {
    if (tliq[c] >= 0.0 && tsol[c] >= 0.0) {
      const double tf = tsol[c] - tliq[c];
      const double cr = (Tl - Ts) / tf;
      const double lam = 39.4 * pow(cr, -0.317);      // Eq. 22
      a[0] += tf;
      a[1] += cr;
      a[2] += lam;
      a[3] += 59.0 / sqrt(lam) + 120.3;              // Eq. 23
      a[4] += 1.0;
    }
  }
  for (int k = 0; k < 5; ++k) {
    const double v = block_sum(a[k], sh);
    if (threadIdx.x == 0) part[k * gridDim.x + blockIdx.x] = v;
  }
}
__global__ void k_qoi_final(int nb, const double* part, double* out) {
  __shared__ double sh[32];
  for (int k = 0; k < 5; ++k) {
    double a = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) a += part[k * nb + b];
    a = block_sum(a, sh);
    if (threadIdx.x == 0) out[k] = a;
  }
}

struct UqShared {
  fvs_mesh mesh;
  const fvs_props* base;
  const double* inputs;
  int64_t n;
  double dt;
  int max_steps;
  double* qoi;
  int64_t* steps;
  std::atomic<int64_t> next{0};
  std::atomic<int> status{FVS_OK};
  char err[512] = {0};
};

static fvs_status run_sample(fvs_solver s, UqShared& U, int64_t i, DBuf<double>& part, DBuf<double>& out) {
  const double T_melt = U.inputs[3 * i], T_wall = U.inputs[3 * i + 1], C0 = U.inputs[3 * i + 2];
  fvs_props p = *U.base;
  std::vector<fvs_patch_bc> bc(std::max(1, U.mesh->npatch));
  for (auto& b : bc) { b.type = FVS_BC_DIRICHLET; b.T = T_wall; }
  p.n_patches = (int32_t)bc.size();
  p.bc = bc.data();
  p.T_init = T_melt;
  p.mat.T_liq = U.base->mat.T_liq - 5.0 * (C0 - 4.0);
  FVS_TRY(solver_set_properties(s, &p));
  int64_t k = 0;
  for (; k < U.max_steps; ++k) {
    fvs_step_stats st;
    fvs_status r = solver_step(s, U.dt, &st);
    if (r != FVS_OK && r != FVS_ERR_NOT_CONVERGED) return r;
    if (st.n_active == 0) {
      // the step started fully solid; stop once everything is below the solidus
      ++k;
      break;
    }
  }
  const int nb = 2 * sm_count();
  k_qoi_part<<<nb, 256, 0, s->stream>>>(s->mesh->Nc, s->tliq, s->tsol, p.mat.T_sol, p.mat.T_liq, part.p);
  FVS_COUNT_LAUNCH();
  k_qoi_final<<<1, 1024, 0, s->stream>>>(nb, part.p, out.p);
  FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  double h[5];
  FVS_CUDA(cudaMemcpyAsync(h, out.p, 5 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  FVS_CUDA(cudaStreamSynchronize(s->stream));
  const double nan = std::nan("");
  for (int q = 0; q < 4; ++q) U.qoi[4 * i + q] = h[4] > 0 ? h[q] / h[4] : nan;
  if (U.steps) U.steps[i] = k;
  return FVS_OK;
}

static void worker(UqShared* U, int device) {
  cudaSetDevice(device);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    U->status = FVS_ERR_CUDA;
    return;
  }
  {
    AllocStream as(st);
    fvs_solver_s* s = new fvs_solver_s();
    s->mesh = U->mesh;
    s->stream = st;
    fvs_status r = solver_alloc(s);
    DBuf<double> part, out;
    if (r == FVS_OK) r = part.alloc(5 * 2 * (size_t)sm_count());
    if (r == FVS_OK) r = out.alloc(5);
    while (r == FVS_OK && U->status.load() == FVS_OK) {
      const int64_t i = U->next.fetch_add(1);
      if (i >= U->n) break;
      r = run_sample(s, *U, i, part, out);
    }
    if (r != FVS_OK) {
      int expected = FVS_OK;
      if (U->status.compare_exchange_strong(expected, r)) snprintf(U->err, sizeof(U->err), "%s", fvs_last_error());
    }
    cudaStreamSynchronize(st);
    delete s;
    part.release();
    out.release();
    cudaStreamSynchronize(st);
  }
  cudaStreamDestroy(st);
}

fvs_status uq_batch(fvs_mesh mesh, const fvs_props* base, int64_t n, const double* inputs, double dt,
                    int max_steps, int n_streams, double* qoi, int64_t* steps) {
  UqShared U;
  U.mesh = mesh;
  U.base = base;
  U.inputs = inputs;
  U.n = n;
  U.dt = dt;
  U.max_steps = max_steps;
  U.qoi = qoi;
  U.steps = steps;
  int nw = n_streams > 0 ? n_streams : 8;
  if (nw > n) nw = (int)n;
  FVS_CUDA(cudaStreamSynchronize(mesh->stream));
  std::vector<std::thread> th;
  for (int w = 0; w < nw; ++w) th.emplace_back(worker, &U, mesh->device);
  for (auto& t : th) t.join();
  if (U.status.load() != FVS_OK) {
    set_error("uq batch: %s", U.err);
    return (fvs_status)U.status.load();
  }
  return FVS_OK;
}

}  // namespace fvs
