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
#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>
#include <vector>

#include "batch.cuh"
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
// the outputs of Section 5 over the whole domain: latest solidus crossing
// (total solidification time), largest SDAS, smallest yield strength,
// largest grain radius, and the count of metal cells still above the solidus
__global__ void k_qoi_ext_part(int64_t Nc, const double* tliq, const double* tsol, const uint8_t* metal,
                               const double* r2, double Ts, double Tl, double* part) {
  __shared__ double sh[32];
  double a[5] = {-1.0, -1.0, 1e300, 0.0, 0.0};
  GS(c, Nc) {
    if (!metal[c]) continue;
    if (tsol[c] < 0.0) {
      a[4] += 1.0;
    } else {
      a[0] = fmax(a[0], tsol[c]);
      if (tliq[c] >= 0.0) {
        const double lam = 39.4 * pow((Tl - Ts) / (tsol[c] - tliq[c]), -0.317);   // Eq. 22
        a[1] = fmax(a[1], lam);
        a[2] = fmin(a[2], 59.0 / sqrt(lam) + 120.3);                            // Eq. 23
      }
    }
    if (r2) a[3] = fmax(a[3], sqrt(r2[c]));
  }
  a[0] = block_max(a[0], sh);
  a[1] = block_max(a[1], sh);
  a[2] = -block_max(-a[2], sh);
  a[3] = block_max(a[3], sh);
  a[4] = block_sum(a[4], sh);
  if (threadIdx.x == 0)
    for (int k = 0; k < 5; ++k) part[k * gridDim.x + blockIdx.x] = a[k];
}
__global__ void k_qoi_ext_final(int nb, const double* part, double* out) {
  __shared__ double sh[32];
  double a[5] = {-1.0, -1.0, 1e300, 0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    a[0] = fmax(a[0], part[b]);
    a[1] = fmax(a[1], part[nb + b]);
    a[2] = fmin(a[2], part[2 * nb + b]);
    a[3] = fmax(a[3], part[3 * nb + b]);
    a[4] += part[4 * nb + b];
  }
  a[0] = block_max(a[0], sh);
  a[1] = block_max(a[1], sh);
  a[2] = -block_max(-a[2], sh);
  a[3] = block_max(a[3], sh);
  a[4] = block_sum(a[4], sh);
  if (threadIdx.x == 0)
    for (int k = 0; k < 5; ++k) out[k] = a[k];
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
  const UqSpec* spec;
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
  (void)C0;   // the liquidus comes from the sample's C0 (UqSpec)
  p.T_init = T_melt;
  p.mat.T_liq = U.spec->T_liq[i];
  FVS_TRY(solver_set_properties(s, &p));
  if (U.spec->grain_Ds > 0.0) FVS_TRY(solver_set_grain(s, U.spec->grain_kp, U.spec->grain_Ds, U.spec->grain_r0));
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
  const int64_t Nc = s->mesh->Nc;
  if (U.spec->qoi_kind == FVS_QOI_EXTREMES) {
    k_qoi_ext_part<<<nb, 256, 0, s->stream>>>(Nc, s->tliq, s->tsol, s->metal, s->grain_on ? s->r2.p : nullptr,
                                              p.mat.T_sol, p.mat.T_liq, part.p);
    FVS_COUNT_LAUNCH();
    k_qoi_ext_final<<<1, 1024, 0, s->stream>>>(nb, part.p, out.p);
  } else {
    k_qoi_part<<<nb, 256, 0, s->stream>>>(Nc, s->tliq, s->tsol, p.mat.T_sol, p.mat.T_liq, part.p);
    FVS_COUNT_LAUNCH();
    k_qoi_final<<<1, 1024, 0, s->stream>>>(nb, part.p, out.p);
  }
  FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  double h[5];
  FVS_CUDA(cudaMemcpyAsync(h, out.p, 5 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  FVS_CUDA(cudaStreamSynchronize(s->stream));
  const double nan = std::nan("");
  if (U.spec->qoi_kind == FVS_QOI_EXTREMES) {
    const bool all_solid = h[4] == 0.0;
    U.qoi[4 * i + 0] = all_solid && h[0] >= 0.0 ? h[0] : nan;
    U.qoi[4 * i + 1] = h[1] >= 0.0 ? h[1] : nan;
    U.qoi[4 * i + 2] = h[1] >= 0.0 ? h[2] : nan;
    U.qoi[4 * i + 3] = h[3];
  } else {
    for (int q = 0; q < 4; ++q) U.qoi[4 * i + q] = h[4] > 0 ? h[q] / h[4] : nan;
  }
  if (U.steps) U.steps[i] = k;
  // final fields of the sample, caller's cell order
  if (U.spec->T_out) FVS_TRY(solver_query(s, FVS_T, U.spec->T_out + i * Nc, Nc, 0));
  if (U.spec->p_out) FVS_TRY(solver_query(s, FVS_P, U.spec->p_out + i * Nc, Nc, 0));
  if (U.spec->u_out) FVS_TRY(solver_query(s, FVS_U, U.spec->u_out + i * 3 * Nc, 3 * Nc, 0));
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
                    int max_steps, int n_streams, const UqSpec& spec, double* qoi, int64_t* steps) {
  UqShared U;
  U.mesh = mesh;
  U.spec = &spec;
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

// ---------------------------------------------------------------------------
// surrogate mode: an ensemble of trained networks answers the samples inside
// its training box on which the models agree; the rest are solved plainly
// ---------------------------------------------------------------------------
// Y [K][n][no]: per sample the ensemble mean of every output, and whether
// the sample is accepted (inside [lo, hi] and, with max_spread > 0, every
// output's standard deviation over the models at most max_spread |mean|)
__global__ void k_uq_accept(int64_t n, int K, int ni, int no, const double* X, const double* Y, const double* lo,
                            const double* hi, double max_spread, double* mean, int32_t* accept) {
  GS(i, n) {
    bool ok = true;
    for (int d = 0; d < ni; ++d) {
      const double x = X[i * ni + d];
      ok = ok && x >= lo[d] && x <= hi[d];
    }
    for (int q = 0; q < no; ++q) {
      double m = 0.0;
      for (int k = 0; k < K; ++k) m += Y[((int64_t)k * n + i) * no + q];
      m /= (double)K;
      double v = 0.0;
      for (int k = 0; k < K; ++k) {
        const double e = Y[((int64_t)k * n + i) * no + q] - m;
        v += e * e;
      }
      const double sd = K > 1 ? sqrt(v / (double)(K - 1)) : 0.0;
      if (max_spread > 0.0 && !(sd <= max_spread * fabs(m))) ok = false;
      mean[i * no + q] = m;
    }
    accept[i] = ok ? 1 : 0;
  }
}

fvs_status uq_surrogate(fvs_mesh mesh, const fvs_props* base, int64_t n, const double* inputs, double dt,
                        int max_steps, const fvs_uq_options& opt, const UqSpec& spec, double* qoi, int64_t* steps) {
  if (opt.n_models <= 0 || !opt.models || !opt.box_lo || !opt.box_hi) {
    set_error("fvs_uq_batch: surrogate mode needs models and the box of their training inputs");
    return FVS_ERR_ARG;
  }
  if (opt.plain_mode != FVS_UQ_LOCKSTEP && opt.plain_mode != FVS_UQ_STREAMS) {
    set_error("fvs_uq_batch: plain_mode must be FVS_UQ_LOCKSTEP or FVS_UQ_STREAMS");
    return FVS_ERR_ARG;
  }
  for (int k = 0; k < opt.n_models; ++k) {
    int ni = 0, no = 0;
    FVS_TRY(surrogate_dims(opt.models[k], &ni, &no));
    if (ni != 3 || no != 4) {
      set_error("fvs_uq_batch: surrogate %d maps %d inputs to %d outputs; the UQ map is 3 -> 4", k, ni, no);
      return FVS_ERR_ARG;
    }
  }
  const int K = opt.n_models;
  std::vector<int32_t> acc(n);
  std::vector<double> mean((size_t)n * 4);
  cudaStream_t st = nullptr;
  FVS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  fvs_status r = [&]() -> fvs_status {
    AllocStream as(st);
    DBuf<double> X, Y, M, box;
    DBuf<int32_t> A;
    FVS_TRY(X.alloc((size_t)n * 3)); FVS_TRY(Y.alloc((size_t)K * n * 4)); FVS_TRY(M.alloc((size_t)n * 4));
    FVS_TRY(box.alloc(6)); FVS_TRY(A.alloc(n));
    const double hb[6] = {opt.box_lo[0], opt.box_lo[1], opt.box_lo[2], opt.box_hi[0], opt.box_hi[1], opt.box_hi[2]};
    FVS_CUDA(cudaMemcpyAsync(X.p, inputs, (size_t)n * 3 * sizeof(double), cudaMemcpyHostToDevice, st));
    FVS_CUDA(cudaMemcpyAsync(box.p, hb, sizeof hb, cudaMemcpyHostToDevice, st));
    FVS_CUDA(cudaStreamSynchronize(st));
    // each model runs on its own stream and returns when its outputs are in Y
    for (int k = 0; k < K; ++k) FVS_TRY(fvs_surrogate_predict(opt.models[k], X.p, Y.p + (size_t)k * n * 4, n, 1));
    k_uq_accept<<<stride_grid(n, 256), 256, 0, st>>>(n, K, 3, 4, X, Y, box.p, box.p + 3, opt.max_spread, M, A);
    FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    FVS_CUDA(cudaMemcpyAsync(acc.data(), A.p, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    FVS_CUDA(cudaMemcpyAsync(mean.data(), M.p, (size_t)n * 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
    FVS_CUDA(cudaStreamSynchronize(st));
    return FVS_OK;
  }();
  cudaStreamDestroy(st);
  FVS_TRY(r);
  // plain solves of the samples the ensemble did not accept
  std::vector<int64_t> rej;
  for (int64_t i = 0; i < n; ++i) {
    if (opt.used_plain) opt.used_plain[i] = acc[i] ? 0 : 1;
    if (acc[i]) {
      for (int q = 0; q < 4; ++q) qoi[4 * i + q] = mean[4 * i + q];
      if (steps) steps[i] = 0;
    } else {
      rej.push_back(i);
    }
  }
  if (rej.empty()) return FVS_OK;
  const int64_t m = (int64_t)rej.size(), Nc = mesh->Nc;
  std::vector<double> xin((size_t)m * 3), q((size_t)m * 4);
  std::vector<int64_t> stp(m);
  UqSpec sub;
  sub.qoi_kind = spec.qoi_kind;
  sub.grain_kp = spec.grain_kp;
  sub.grain_Ds = spec.grain_Ds;
  sub.grain_r0 = spec.grain_r0;
  sub.T_liq.resize(m);
  std::vector<double> fT, fu, fp;
  if (spec.T_out) { fT.resize((size_t)m * Nc); sub.T_out = fT.data(); }
  if (spec.u_out) { fu.resize((size_t)m * Nc * 3); sub.u_out = fu.data(); }
  if (spec.p_out) { fp.resize((size_t)m * Nc); sub.p_out = fp.data(); }
  for (int64_t j = 0; j < m; ++j) {
    for (int d = 0; d < 3; ++d) xin[3 * j + d] = inputs[3 * rej[j] + d];
    sub.T_liq[j] = spec.T_liq[rej[j]];
  }
  const fvs_status ps = opt.plain_mode == FVS_UQ_LOCKSTEP
                            ? batch_run(mesh, base, m, xin.data(), dt, max_steps, sub, q.data(), stp.data())
                            : uq_batch(mesh, base, m, xin.data(), dt, max_steps, opt.n_streams, sub, q.data(),
                                       stp.data());
  if (ps != FVS_OK && ps != FVS_ERR_NOT_CONVERGED) return ps;
  for (int64_t j = 0; j < m; ++j) {
    const int64_t i = rej[j];
    for (int c = 0; c < 4; ++c) qoi[4 * i + c] = q[4 * j + c];
    if (steps) steps[i] = stp[j];
    if (spec.T_out) std::copy(fT.begin() + j * Nc, fT.begin() + (j + 1) * Nc, spec.T_out + i * Nc);
    if (spec.p_out) std::copy(fp.begin() + j * Nc, fp.begin() + (j + 1) * Nc, spec.p_out + i * Nc);
    if (spec.u_out) std::copy(fu.begin() + j * 3 * Nc, fu.begin() + (j + 1) * 3 * Nc, spec.u_out + i * 3 * Nc);
  }
  return ps;
}

}  // namespace fvs
