// Line preconditioner (declared in la.cuh): tridiagonal solves along chains
// of strongly coupled cells.  Used for the energy system, whose couplings
// across thin cells exceed its mass term several times over, so that
// point-Jacobi needs many Krylov iterations.
#include <vector>

#include "la.cuh"
#include "lines_host.h"

namespace fvs {

namespace {

constexpr int kMaxLine = 512;   // longer chains are cut (a dropped coupling keeps P a valid preconditioner)

// Thomas factors of every line with the current values: row k of a line
// reads lo_k x_{k-1} + b_k x_k + up_k x_{k+1}; pivots d_k = b_k - lo_k cp_{k-1},
// cp_k = up_k / d_k.  One thread per line.
__global__ void k_line_factor(int64_t ngroups, const int64_t* __restrict__ goff, const int32_t* __restrict__ llen,
                              const int32_t* __restrict__ cell, const int8_t* __restrict__ sprev,
                              const int8_t* __restrict__ snext, int64_t n, const double* __restrict__ val,
                              const double* __restrict__ diag, const double* __restrict__ dextra,
                              double* __restrict__ lo, double* __restrict__ inv, double* __restrict__ cp) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t g = t >> 5;
  if (g >= ngroups) return;
  const int lane = (int)(t & 31);
  const int len = llen[t];
  const int64_t base = goff[g] + lane;
  double cprev = 0.0;
#pragma unroll 4
  for (int pos = 0; pos < len; ++pos) {
    const int64_t idx = base + (int64_t)pos * 32;
    const int32_t c = cell[idx];
    const int kp = sprev[idx], kn = snext[idx];
    const double a = kp >= 0 ? val[(int64_t)kp * n + c] : 0.0;
    const double u = kn >= 0 ? val[(int64_t)kn * n + c] : 0.0;
    const double d = diag[c] + (dextra ? dextra[c] : 0.0) - a * cprev;
    const double iv = d != 0.0 ? 1.0 / d : 0.0;
    lo[idx] = a;
    inv[idx] = iv;
    cprev = u * iv;
    cp[idx] = cprev;
  }
}

// z = P^-1 r: forward substitution y_k = (r_k - lo_k y_{k-1}) / d_k (kept in
// z), then back substitution x_k = y_k - cp_k x_{k+1}.
__global__ void k_line_solve(int64_t ngroups, const int64_t* __restrict__ goff, const int32_t* __restrict__ llen,
                             const int32_t* __restrict__ cell, const double* __restrict__ lo,
                             const double* __restrict__ inv, const double* __restrict__ cp, const double* r,
                             double* z) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t g = t >> 5;
  if (g >= ngroups) return;
  const int lane = (int)(t & 31);
  const int len = llen[t];
  const int64_t base = goff[g] + lane;
  double y = 0.0;
#pragma unroll 4
  for (int pos = 0; pos < len; ++pos) {
    const int64_t idx = base + (int64_t)pos * 32;
    const int32_t c = cell[idx];
    y = (r[c] - lo[idx] * y) * inv[idx];
    z[c] = y;
  }
  double x = 0.0;
#pragma unroll 4
  for (int pos = len - 1; pos >= 0; --pos) {
    const int64_t idx = base + (int64_t)pos * 32;
    const int32_t c = cell[idx];
    x = z[c] - cp[idx] * x;
    z[c] = x;
  }
}

}  // namespace

fvs_status LinePrecond::build(cudaStream_t s, const Ell& Ain) {
  ready = false;
  A = &Ain;
  n = Ain.n;
  w = Ain.w;
  built_from = Ain.col.p;
  if (n <= 0) return FVS_OK;
  if (n > 2147483647LL) {
    set_error("line preconditioner: %lld rows exceed 32-bit cell ids", (long long)n);
    return FVS_ERR_ARG;
  }
  const size_t nw = (size_t)n * (size_t)w;
  std::vector<int32_t> col(nw);
  std::vector<double> val(nw);
  FVS_CUDA(cudaMemcpyAsync(col.data(), Ain.col.p, nw * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FVS_CUDA(cudaMemcpyAsync(val.data(), Ain.val.p, nw * sizeof(double), cudaMemcpyDeviceToHost, s));
  FVS_CUDA(cudaStreamSynchronize(s));
  LineLayout L;
  build_line_layout(col.data(), val.data(), n, w, kMaxLine, L);
  nlines = L.nlines;
  ngroups = L.ngroups;
  padded = L.padded;
  max_len = L.max_len;
  FVS_TRY(goff.alloc(ngroups + 1));
  FVS_TRY(llen.alloc((size_t)ngroups * 32 + 1));
  FVS_TRY(cell.alloc(padded + 1));
  FVS_TRY(sprev.alloc(padded + 1));
  FVS_TRY(snext.alloc(padded + 1));
  FVS_TRY(lo.alloc(padded + 1));
  FVS_TRY(inv.alloc(padded + 1));
  FVS_TRY(cp.alloc(padded + 1));
  FVS_CUDA(cudaMemcpyAsync(goff.p, L.goff.data(), (ngroups + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  FVS_CUDA(cudaMemcpyAsync(llen.p, L.llen.data(), L.llen.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  FVS_CUDA(cudaMemcpyAsync(cell.p, L.cell.data(), padded * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  FVS_CUDA(cudaMemcpyAsync(sprev.p, L.sprev.data(), padded * sizeof(int8_t), cudaMemcpyHostToDevice, s));
  FVS_CUDA(cudaMemcpyAsync(snext.p, L.snext.data(), padded * sizeof(int8_t), cudaMemcpyHostToDevice, s));
  FVS_CUDA(cudaStreamSynchronize(s));   // the host arrays go out of scope
  ready = true;
  return FVS_OK;
}

fvs_status LinePrecond::factor(cudaStream_t s) {
  if (!ready || n <= 0) return FVS_OK;
  const int64_t threads = ngroups * 32;
  k_line_factor<<<grid_for(threads, 128), 128, 0, s>>>(ngroups, goff, llen, cell, sprev, snext, n, A->val,
                                                      A->diag, dextra, lo, inv, cp);
  FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

fvs_status LinePrecond::apply(cudaStream_t s, const double* r, double* z) {
  if (n <= 0) return FVS_OK;
  const int64_t threads = ngroups * 32;
  k_line_solve<<<grid_for(threads, 128), 128, 0, s>>>(ngroups, goff, llen, cell, lo, inv, cp, r, z);
  FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  return FVS_OK;
}

}  // namespace fvs
