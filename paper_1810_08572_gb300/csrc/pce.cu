// Polynomial chaos surrogate of the UQ map (Section 2.7, Eq. 27-28; the
// paper's own surrogate, with the total Sobol indices of Section 5).
//
// An output w(xi) is expanded in products of orthonormal 1-D polynomials of
// the standardised inputs (probabilists' Hermite for normal inputs, Legendre
// for uniform ones), truncated at a total degree.  The coefficients solve the
// overdetermined Vandermonde system of Eq. 28 in the least-squares sense: the
// GPU forms the normal equations (Psi^T Psi) c = Psi^T w, factors them by
// Cholesky in one block and refines the solution twice against the residual
// of the Vandermonde system itself.  Evaluation on Monte Carlo inputs is one
// thread per sample.  Collocation points are the roots of the basis
// polynomials (eigenvalues of their Jacobi matrices, by cyclic Jacobi
// rotations on the host), combined by a tensor product or by Smolyak's rule.
#include <algorithm>
#include <cmath>
#include <map>
#include <vector>

#include "common.cuh"

#define FVS_API extern "C" __attribute__((visibility("default")))

namespace fvs {

#define GS(i, n) for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

constexpr int PCE_MAXD = 8;     // inputs
constexpr int PCE_MAXP = 24;    // total degree
constexpr int PCE_MAXOUT = 8;   // outputs

struct PceDims {
  int d, p, P, nout;
  int fam[PCE_MAXD];
  double a[PCE_MAXD], b[PCE_MAXD];   // normal: mean, sd; uniform: lo, hi
};

// orthonormal 1-D values psi_0..psi_p at the standardised input of x
__device__ __forceinline__ void pce_basis_1d(const PceDims& D, int j, double x, double* B) {
  const bool normal = D.fam[j] == 0;
  const double xi = normal ? (x - D.a[j]) / D.b[j] : (2.0 * x - D.a[j] - D.b[j]) / (D.b[j] - D.a[j]);
  B[0] = 1.0;
  if (D.p >= 1) B[1] = xi;
  for (int n = 1; n < D.p; ++n)
    B[n + 1] = normal ? xi * B[n] - n * B[n - 1] : ((2 * n + 1) * xi * B[n] - n * B[n - 1]) / (n + 1);
  double f = 1.0;   // n! for the Hermite norms
  for (int n = 0; n <= D.p; ++n) {
    if (n > 0) f *= n;
    B[n] *= normal ? rsqrt(f) : sqrt(2.0 * n + 1.0);
  }
}

// row m of the Vandermonde matrix of Eq. 28: V[m*P + k] = prod_j psi_{alpha_kj}
__global__ void k_pce_vander(int64_t m, PceDims D, const int8_t* alpha, const double* X, double* V) {
  double B[PCE_MAXD][PCE_MAXP + 1];
  GS(r, m) {
    for (int j = 0; j < D.d; ++j) pce_basis_1d(D, j, X[r * D.d + j], B[j]);
    for (int k = 0; k < D.P; ++k) {
      double v = 1.0;
      for (int j = 0; j < D.d; ++j) v *= B[j][alpha[k * D.d + j]];
      V[r * D.P + k] = v;
    }
  }
}

// G = V^T V (P x P) and R = V^T Y (P x nout), one thread per entry, rows
// summed in a fixed order
__global__ void k_pce_normal(int64_t m, int P, int nout, const double* V, const double* Y, double* G, double* R) {
  const int64_t total = (int64_t)P * (P + nout);
  GS(e, total) {
    const int i = (int)(e / (P + nout)), jj = (int)(e % (P + nout));
    double s = 0.0;
    if (jj < P) {
      for (int64_t r = 0; r < m; ++r) s += V[r * P + i] * V[r * P + jj];
      G[(int64_t)i * P + jj] = s;
    } else {
      const int q = jj - P;
      for (int64_t r = 0; r < m; ++r) s += V[r * P + i] * Y[r * nout + q];
      R[(int64_t)i * nout + q] = s;
    }
  }
}

// residual of the Vandermonde system: E = Y - V C (m x nout)
__global__ void k_pce_resid(int64_t m, int P, int nout, const double* V, const double* C, const double* Y,
                            double* E) {
  GS(e, m * nout) {
    const int64_t r = e / nout;
    const int q = (int)(e % nout);
    double s = Y[e];
    for (int k = 0; k < P; ++k) s -= V[r * P + k] * C[(int64_t)k * nout + q];
    E[e] = s;
  }
}

// In one block: Cholesky G = L L^T in place (lower triangle), then solve
// L L^T X = R for the nout right sides (X overwrites R).  err: not positive
// definite (a collocation set that does not determine the coefficients).
__global__ void k_pce_cholesky_solve(int P, int nout, double* G, double* R, int* err) {
  __shared__ double piv;
  for (int k = 0; k < P; ++k) {
    if (threadIdx.x == 0) {
      double s = G[(int64_t)k * P + k];
      for (int t = 0; t < k; ++t) s -= G[(int64_t)k * P + t] * G[(int64_t)k * P + t];
      if (!(s > 0.0)) {
        *err = 1;
        s = 1e-300;
      }
      piv = sqrt(s);
      G[(int64_t)k * P + k] = piv;
    }
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < P; i += blockDim.x) {
      double s = G[(int64_t)i * P + k];
      for (int t = 0; t < k; ++t) s -= G[(int64_t)i * P + t] * G[(int64_t)k * P + t];
      G[(int64_t)i * P + k] = s / piv;
    }
    __syncthreads();
  }
  // forward (L y = r) then backward (L^T x = y) substitution, one thread per right side
  for (int q = threadIdx.x; q < nout; q += blockDim.x) {
    for (int i = 0; i < P; ++i) {
      double s = R[(int64_t)i * nout + q];
      for (int t = 0; t < i; ++t) s -= G[(int64_t)i * P + t] * R[(int64_t)t * nout + q];
      R[(int64_t)i * nout + q] = s / G[(int64_t)i * P + i];
    }
    for (int i = P - 1; i >= 0; --i) {
      double s = R[(int64_t)i * nout + q];
      for (int t = i + 1; t < P; ++t) s -= G[(int64_t)t * P + i] * R[(int64_t)t * nout + q];
      R[(int64_t)i * nout + q] = s / G[(int64_t)i * P + i];
    }
  }
}

// R = V^T E (P x nout): the right side of the refinement step
__global__ void k_pce_vte(int64_t m, int P, int nout, const double* V, const double* E, double* R) {
  GS(e, (int64_t)P * nout) {
    const int i = (int)(e / nout), q = (int)(e % nout);
    double s = 0.0;
    for (int64_t r = 0; r < m; ++r) s += V[r * P + i] * E[r * nout + q];
    R[e] = s;
  }
}
// solve L L^T X = R with the factor k_pce_cholesky_solve left in G
__global__ void k_pce_chol_apply(int P, int nout, const double* G, double* R) {
  for (int q = threadIdx.x; q < nout; q += blockDim.x) {
    for (int i = 0; i < P; ++i) {
      double s = R[(int64_t)i * nout + q];
      for (int t = 0; t < i; ++t) s -= G[(int64_t)i * P + t] * R[(int64_t)t * nout + q];
      R[(int64_t)i * nout + q] = s / G[(int64_t)i * P + i];
    }
    for (int i = P - 1; i >= 0; --i) {
      double s = R[(int64_t)i * nout + q];
      for (int t = i + 1; t < P; ++t) s -= G[(int64_t)t * P + i] * R[(int64_t)t * nout + q];
      R[(int64_t)i * nout + q] = s / G[(int64_t)i * P + i];
    }
  }
}
__global__ void k_pce_axpy(int64_t n, const double* a, double* c) {
  GS(i, n) c[i] += a[i];
}

// Y[n x nout] = sum_k C[k] prod_j psi_{alpha_kj}(xi_j), one thread per sample
__global__ void k_pce_eval(int64_t n, PceDims D, const int8_t* alpha, const double* C, const double* X, double* Y) {
  double B[PCE_MAXD][PCE_MAXP + 1];
  GS(r, n) {
    for (int j = 0; j < D.d; ++j) pce_basis_1d(D, j, X[r * D.d + j], B[j]);
    double y[PCE_MAXOUT];
    for (int q = 0; q < D.nout; ++q) y[q] = 0.0;
    for (int k = 0; k < D.P; ++k) {
      double v = 1.0;
      for (int j = 0; j < D.d; ++j) v *= B[j][alpha[k * D.d + j]];
      for (int q = 0; q < D.nout; ++q) y[q] += C[(int64_t)k * D.nout + q] * v;
    }
    for (int q = 0; q < D.nout; ++q) Y[r * D.nout + q] = y[q];
  }
}

// per output (one block each): mean c_0, variance sum_{k>0} c_k^2, total and
// first-order Sobol indices of every input
__global__ void k_pce_sobol(PceDims D, const int8_t* alpha, const double* C, double* out) {
  const int q = blockIdx.x;
  __shared__ double sh[32];
  __shared__ double var;
  double v = 0.0;
  for (int k = 1 + threadIdx.x; k < D.P; k += blockDim.x) v += C[(int64_t)k * D.nout + q] * C[(int64_t)k * D.nout + q];
  v = block_sum(v, sh);
  if (threadIdx.x == 0) var = v;
  __syncthreads();
  double* o = out + (int64_t)q * (2 + 2 * D.d);
  if (threadIdx.x == 0) {
    o[0] = C[q];
    o[1] = var;
  }
  for (int j = 0; j < D.d; ++j) {
    double t = 0.0, f = 0.0;
    for (int k = 1 + threadIdx.x; k < D.P; k += blockDim.x) {
      const double c2 = C[(int64_t)k * D.nout + q] * C[(int64_t)k * D.nout + q];
      int deg = 0;
      for (int i = 0; i < D.d; ++i) deg += alpha[k * D.d + i];
      if (alpha[k * D.d + j] > 0) {
        t += c2;
        if (deg == alpha[k * D.d + j]) f += c2;
      }
    }
    t = block_sum(t, sh);
    f = block_sum(f, sh);
    if (threadIdx.x == 0) {
      o[2 + j] = var > 0.0 ? t / var : 0.0;
      o[2 + D.d + j] = var > 0.0 ? f / var : 0.0;
    }
  }
}

// roots of the degree-n orthonormal polynomial: eigenvalues of its
// symmetric tridiagonal Jacobi matrix (zero diagonal; off-diagonal sqrt(k)
// for Hermite, k / sqrt(4k^2 - 1) for Legendre), by cyclic Jacobi rotations
static std::vector<double> gauss_roots(int family, int n) {
  std::vector<double> A((size_t)n * n, 0.0);
  for (int k = 1; k < n; ++k) {
    const double e = family == 0 ? std::sqrt((double)k) : k / std::sqrt(4.0 * k * k - 1.0);
    A[(size_t)(k - 1) * n + k] = A[(size_t)k * n + k - 1] = e;
  }
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[(size_t)i * n + j] * A[(size_t)i * n + j];
    if (off < 1e-30) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        // rotation that zeroes A[p][q]
        const double theta = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
      }
    }
  }
  std::vector<double> r(n);
  for (int i = 0; i < n; ++i) r[i] = A[(size_t)i * n + i];
  std::sort(r.begin(), r.end());
  for (auto& x : r)
    if (std::fabs(x) < 1e-13) x = 0.0;   // the middle root of an odd rule
  return r;
}

}  // namespace fvs

using namespace fvs;

struct fvs_pce_s {
  cudaStream_t stream = nullptr;
  PceDims D{};
  std::vector<int8_t> alpha;   // [P*d]
  DBuf<int8_t> dalpha;
  DBuf<double> coef;           // [P*nout]
  bool fitted = false;
};

FVS_API fvs_status fvs_pce_create(int32_t n_in, const int32_t* family, const double* p1, const double* p2,
                                  int32_t degree, int32_t n_out, void* stream, fvs_pce* out) {
  if (!out || !family || !p1 || !p2 || n_in < 1 || n_in > PCE_MAXD || degree < 0 || degree > PCE_MAXP ||
      n_out < 1 || n_out > PCE_MAXOUT) {
    set_error("fvs_pce_create: bad argument (1..%d inputs, degree 0..%d, 1..%d outputs)", PCE_MAXD, PCE_MAXP,
              PCE_MAXOUT);
    return FVS_ERR_ARG;
  }
  for (int j = 0; j < n_in; ++j) {
    const bool ok = (family[j] == FVS_PCE_NORMAL && p2[j] > 0) || (family[j] == FVS_PCE_UNIFORM && p2[j] > p1[j]);
    if (!ok) {
      set_error("fvs_pce_create: input %d: a normal input needs sd > 0, a uniform one lo < hi", j);
      return FVS_ERR_ARG;
    }
  }
  *out = nullptr;
  fvs_pce s = new (std::nothrow) fvs_pce_s();
  if (!s) return FVS_ERR_NOMEM;
  s->stream = (cudaStream_t)stream;
  s->D.d = n_in;
  s->D.p = degree;
  s->D.nout = n_out;
  for (int j = 0; j < n_in; ++j) {
    s->D.fam[j] = family[j];
    s->D.a[j] = p1[j];
    s->D.b[j] = p2[j];
  }
  // multi-indices of total degree <= p, graded by degree (alpha = 0 first)
  std::vector<int> a(n_in, 0);
  for (int deg = 0; deg <= degree; ++deg) {
    std::fill(a.begin(), a.end(), 0);
    // odometer over [0, deg]^d keeping those that sum to deg
    while (true) {
      int sum = 0;
      for (int v : a) sum += v;
      if (sum == deg)
        for (int j = 0; j < n_in; ++j) s->alpha.push_back((int8_t)a[j]);
      int j = n_in - 1;
      while (j >= 0 && a[j] == deg) a[j--] = 0;
      if (j < 0) break;
      ++a[j];
    }
  }
  // (the odometer runs with the last input fastest, as the oracle orders
  // its multi-indices)
  s->D.P = (int)(s->alpha.size() / n_in);
  AllocStream as(s->stream);
  fvs_status st = s->dalpha.alloc(s->alpha.size());
  if (st == FVS_OK) st = s->coef.alloc((size_t)s->D.P * n_out);
  if (st == FVS_OK && cudaMemcpyAsync(s->dalpha.p, s->alpha.data(), s->alpha.size(), cudaMemcpyHostToDevice,
                                      s->stream) != cudaSuccess) {
    set_error("fvs_pce_create: upload failed");
    st = FVS_ERR_CUDA;
  }
  if (st == FVS_OK && cudaStreamSynchronize(s->stream) != cudaSuccess) st = FVS_ERR_CUDA;
  if (st != FVS_OK) {
    delete s;
    return st;
  }
  *out = s;
  return FVS_OK;
}

FVS_API fvs_status fvs_pce_destroy(fvs_pce s) {
  if (!s) return FVS_ERR_ARG;
  {
    AllocStream as(s->stream);
    cudaStreamSynchronize(s->stream);
    s->dalpha.release();
    s->coef.release();
    cudaStreamSynchronize(s->stream);
  }
  delete s;
  return FVS_OK;
}

FVS_API int64_t fvs_pce_num_terms(fvs_pce s) { return s ? (int64_t)s->D.P : -1; }

FVS_API fvs_status fvs_pce_multi_indices(fvs_pce s, int32_t* alpha, int64_t len) {
  if (!s || !alpha || len < (int64_t)s->alpha.size()) {
    set_error("fvs_pce_multi_indices: bad argument");
    return FVS_ERR_ARG;
  }
  for (size_t i = 0; i < s->alpha.size(); ++i) alpha[i] = s->alpha[i];
  return FVS_OK;
}

FVS_API fvs_status fvs_pce_nodes(fvs_pce s, int32_t level, int32_t sparse, double* X, int64_t cap, int64_t* n_out) {
  if (!s || !n_out || level < 1 || level > 40) {
    set_error("fvs_pce_nodes: bad argument (level 1..40)");
    return FVS_ERR_ARG;
  }
  const int d = s->D.d;
  // standardised rules of 1..level points per input
  std::vector<std::vector<std::vector<double>>> R(d);
  for (int j = 0; j < d; ++j) {
    R[j].resize(level + 1);
    for (int m = 1; m <= level; ++m) R[j][m] = gauss_roots(s->D.fam[j], m);
  }
  std::map<std::vector<long long>, std::vector<double>> pts;   // rounded key -> point
  std::vector<int> idx(d, 1);
  auto add_grid = [&](const std::vector<int>& ii) {
    std::vector<int> c(d, 0);
    while (true) {
      std::vector<double> p(d);
      std::vector<long long> key(d);
      for (int j = 0; j < d; ++j) {
        p[j] = R[j][ii[j]][c[j]];
        key[j] = std::llround(p[j] * 1e10);
      }
      pts.emplace(key, p);
      int j = d - 1;
      while (j >= 0 && c[j] == ii[j] - 1) c[j--] = 0;
      if (j < 0) break;
      ++c[j];
    }
  };
  if (!sparse) {
    add_grid(std::vector<int>(d, level));
  } else {
    // Smolyak: every multi-index with max(d, level) <= |i| <= level + d - 1
    std::vector<int> ii(d, 1);
    while (true) {
      int sum = 0;
      for (int v : ii) sum += v;
      if (sum >= std::max(d, (int)level) && sum <= level + d - 1) add_grid(ii);
      int j = d - 1;
      while (j >= 0 && ii[j] == level) ii[j--] = 1;
      if (j < 0) break;
      ++ii[j];
    }
  }
  *n_out = (int64_t)pts.size();
  if (!X) return FVS_OK;   // count only
  if (cap < *n_out) {
    set_error("fvs_pce_nodes: %lld points do not fit in %lld", (long long)*n_out, (long long)cap);
    return FVS_ERR_ARG;
  }
  int64_t r = 0;
  for (const auto& kv : pts) {
    for (int j = 0; j < d; ++j) {
      const double xi = kv.second[j];
      X[r * d + j] = s->D.fam[j] == FVS_PCE_NORMAL ? s->D.a[j] + s->D.b[j] * xi
                                                    : 0.5 * (s->D.a[j] + s->D.b[j]) + 0.5 * (s->D.b[j] - s->D.a[j]) * xi;
    }
    ++r;
  }
  return FVS_OK;
}

FVS_API fvs_status fvs_pce_fit(fvs_pce s, const double* X, const double* Y, int64_t m, double* rms_resid) {
  if (!s || !X || !Y || m < s->D.P) {
    set_error("fvs_pce_fit: need at least as many points as terms (%d)", s ? s->D.P : 0);
    return FVS_ERR_ARG;
  }
  const int P = s->D.P, d = s->D.d, no = s->D.nout;
  cudaStream_t st = s->stream;
  AllocStream as(st);
  DBuf<double> dX, dY, V, G, R, E, C2;
  DBuf<int> err;
  FVS_TRY(dX.alloc((size_t)m * d)); FVS_TRY(dY.alloc((size_t)m * no)); FVS_TRY(V.alloc((size_t)m * P));
  FVS_TRY(G.alloc((size_t)P * P)); FVS_TRY(R.alloc((size_t)P * no)); FVS_TRY(E.alloc((size_t)m * no));
  FVS_TRY(C2.alloc((size_t)P * no)); FVS_TRY(err.alloc(1)); FVS_TRY(err.zero(st));
  FVS_CUDA(cudaMemcpyAsync(dX.p, X, (size_t)m * d * sizeof(double), cudaMemcpyHostToDevice, st));
  FVS_CUDA(cudaMemcpyAsync(dY.p, Y, (size_t)m * no * sizeof(double), cudaMemcpyHostToDevice, st));
  k_pce_vander<<<stride_grid(m, 128), 128, 0, st>>>(m, s->D, s->dalpha, dX, V); FVS_COUNT_LAUNCH();
  const int64_t ne = (int64_t)P * (P + no);
  k_pce_normal<<<stride_grid(ne, 128), 128, 0, st>>>(m, P, no, V, dY, G, R); FVS_COUNT_LAUNCH();
  k_pce_cholesky_solve<<<1, 256, 0, st>>>(P, no, G, R, err); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  // two refinement steps on the residual of the Vandermonde system (the
  // normal equations square its condition number): C += (L L^T)^-1 V^T (Y - V C)
  for (int it = 0; it < 2; ++it) {
    k_pce_resid<<<stride_grid(m * no, 128), 128, 0, st>>>(m, P, no, V, R, dY, E); FVS_COUNT_LAUNCH();
    k_pce_vte<<<stride_grid((int64_t)P * no, 128), 128, 0, st>>>(m, P, no, V, E, C2); FVS_COUNT_LAUNCH();
    k_pce_chol_apply<<<1, 32, 0, st>>>(P, no, G, C2); FVS_COUNT_LAUNCH();
    k_pce_axpy<<<stride_grid((int64_t)P * no, 128), 128, 0, st>>>((int64_t)P * no, C2, R); FVS_COUNT_LAUNCH();
  }
  FVS_LAUNCH_CHECK();
  int h = 0;
  FVS_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  FVS_CUDA(cudaStreamSynchronize(st));
  if (h) {
    set_error("fvs_pce_fit: the collocation points do not determine the %d coefficients", P);
    return FVS_ERR_ARG;
  }
  FVS_CUDA(cudaMemcpyAsync(s->coef.p, R.p, (size_t)P * no * sizeof(double), cudaMemcpyDeviceToDevice, st));
  s->fitted = true;
  if (rms_resid) {
    k_pce_resid<<<stride_grid(m * no, 128), 128, 0, st>>>(m, P, no, V, s->coef, dY, E); FVS_COUNT_LAUNCH();
    FVS_LAUNCH_CHECK();
    std::vector<double> he((size_t)m * no);
    FVS_CUDA(cudaMemcpyAsync(he.data(), E.p, he.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    FVS_CUDA(cudaStreamSynchronize(st));
    double a = 0.0;
    for (double e : he) a += e * e;
    *rms_resid = std::sqrt(a / (double)he.size());
  }
  FVS_CUDA(cudaStreamSynchronize(st));
  return FVS_OK;
}

FVS_API fvs_status fvs_pce_eval(fvs_pce s, const double* X, double* Y, int64_t n, int on_device) {
  if (!s || !X || !Y || n <= 0 || !s->fitted) {
    set_error("fvs_pce_eval: bad argument or no fit yet");
    return FVS_ERR_ARG;
  }
  cudaStream_t st = s->stream;
  AllocStream as(st);
  const int d = s->D.d, no = s->D.nout;
  DBuf<double> dX, dY;
  const double* xp = X;
  double* yp = Y;
  if (!on_device) {
    FVS_TRY(dX.alloc((size_t)n * d)); FVS_TRY(dY.alloc((size_t)n * no));
    FVS_CUDA(cudaMemcpyAsync(dX.p, X, (size_t)n * d * sizeof(double), cudaMemcpyHostToDevice, st));
    xp = dX.p;
    yp = dY.p;
  }
  k_pce_eval<<<stride_grid(n, 128), 128, 0, st>>>(n, s->D, s->dalpha, s->coef, xp, yp); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  if (!on_device) FVS_CUDA(cudaMemcpyAsync(Y, dY.p, (size_t)n * no * sizeof(double), cudaMemcpyDeviceToHost, st));
  FVS_CUDA(cudaStreamSynchronize(st));
  return FVS_OK;
}

FVS_API fvs_status fvs_pce_coefficients(fvs_pce s, double* c, int64_t len) {
  if (!s || !c || !s->fitted || len < (int64_t)s->D.P * s->D.nout) {
    set_error("fvs_pce_coefficients: bad argument or no fit yet");
    return FVS_ERR_ARG;
  }
  FVS_CUDA(cudaMemcpyAsync(c, s->coef.p, (size_t)s->D.P * s->D.nout * sizeof(double), cudaMemcpyDeviceToHost,
                           s->stream));
  FVS_CUDA(cudaStreamSynchronize(s->stream));
  return FVS_OK;
}

FVS_API fvs_status fvs_pce_sensitivity(fvs_pce s, double* mean, double* var, double* total, double* first) {
  if (!s || !s->fitted) {
    set_error("fvs_pce_sensitivity: no fit yet");
    return FVS_ERR_ARG;
  }
  cudaStream_t st = s->stream;
  AllocStream as(st);
  const int d = s->D.d, no = s->D.nout;
  DBuf<double> o;
  FVS_TRY(o.alloc((size_t)no * (2 + 2 * d)));
  k_pce_sobol<<<no, 256, 0, st>>>(s->D, s->dalpha, s->coef, o); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  std::vector<double> h((size_t)no * (2 + 2 * d));
  FVS_CUDA(cudaMemcpyAsync(h.data(), o.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  FVS_CUDA(cudaStreamSynchronize(st));
  for (int q = 0; q < no; ++q) {
    const double* r = h.data() + (size_t)q * (2 + 2 * d);
    if (mean) mean[q] = r[0];
    if (var) var[q] = r[1];
    for (int j = 0; j < d; ++j) {
      if (total) total[q * d + j] = r[2 + j];
      if (first) first[q * d + j] = r[2 + d + j];
    }
  }
  return FVS_OK;
}
