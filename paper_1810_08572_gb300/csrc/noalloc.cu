// fvs_query_fields_noalloc: the field read-back of fvs_query_fields for
// callers that must not allocate GPU memory.
//
// fvs_query_fields gathers a field from the solver's internal numbering into
// the caller's numbering in a temporary device buffer and copies that to the
// host.  Some callers cannot afford that allocation: a monitor that samples
// a running simulation from a thread that must never block on (or fail in)
// the allocator, code that runs while the device memory budget is already
// exhausted by other work, or a host that has installed a pool with a fixed
// footprint.  This variant stages the gather in a fixed device array that is
// part of the library image instead, and allocates nothing.
//
// The array holds FVS_NOALLOC_MAX_VALUES doubles (8 MiB) and is shared by
// all calls: every call overwrites the values it needs (all of them, so
// nothing has to start at zero), and calls whose GPU work overlaps
// (different streams, or different threads on one stream without ordering)
// race on it.  The CUDA runtime places a module's device arrays on a GPU
// when that module is first used there (lazy loading), and that placement
// is itself an allocation; fvs_solver_create therefore resolves the array's
// address on the solver's device (noalloc_reserve), so the 8 MiB are taken
// when a solver is created and held until the process exits, and a later
// fvs_query_fields_noalloc allocates nothing.
#include <mutex>

#include "solver.cuh"

namespace fvs {

#define FVS_NOALLOC_MAX_VALUES (1 << 20)

static __device__ __align__(256) double g_noalloc_scratch[FVS_NOALLOC_MAX_VALUES];

// device address of the array, looked up once per device under a
// once-flag (host code may not use the symbol itself: on the host it names
// a stand-in, not GPU memory)
static constexpr int kMaxDevices = 64;
static double* g_noalloc_ptr[kMaxDevices] = {nullptr};
static cudaError_t g_noalloc_err[kMaxDevices] = {cudaSuccess};
static std::once_flag g_noalloc_once[kMaxDevices];

static fvs_status noalloc_scratch(double** out) {
  int dev = 0;
  FVS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("fvs_query_fields_noalloc: device %d out of range", dev);
    return FVS_ERR_CUDA;
  }
  std::call_once(g_noalloc_once[dev], [dev] {
    void* p = nullptr;
    g_noalloc_err[dev] = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (g_noalloc_err[dev] == cudaSuccess) g_noalloc_ptr[dev] = (double*)p;
  });
  if (g_noalloc_err[dev] != cudaSuccess || !g_noalloc_ptr[dev]) {
    set_error("fvs_query_fields_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(g_noalloc_err[dev]));
    return FVS_ERR_CUDA;
  }
  *out = g_noalloc_ptr[dev];
  return FVS_OK;
}

// called by fvs_solver_create with the solver's device current
fvs_status noalloc_reserve() {
  double* p = nullptr;
  return noalloc_scratch(&p);
}

#define GS(i, n) for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// out[comps*to_in[i] + d] = src[d*n + i]
__global__ void k_na_gather(int64_t n, int comps, const int32_t* to_in, const double* src, double* out) {
  GS(i, n) {
    const int64_t o = to_in[i];
    for (int d = 0; d < comps; ++d) out[comps * o + d] = src[d * n + i];
  }
}
// out[to_in[i]] = sqrt(a[i]) (grain radius from its square)
__global__ void k_na_sqrt(int64_t n, const int32_t* to_in, const double* a, double* out) {
  GS(i, n) out[to_in[i]] = sqrt(a[i]);
}
// out[2*to_in[i]] = a[i], out[2*to_in[i]+1] = b[i]
__global__ void k_na_pair(int64_t n, const int32_t* to_in, const double* a, const double* b, double* out) {
  GS(i, n) {
    const int64_t o = to_in[i];
    out[2 * o] = a[i];
    out[2 * o + 1] = b[i];
  }
}
__global__ void k_na_u8(int64_t n, const int32_t* to_in, const uint8_t* src, double* out) {
  GS(i, n) out[to_in[i]] = (double)src[i];
}
// per-cell t_f, cooling rate, SDAS (Eq. 22), yield strength (Eq. 23)
__global__ void k_na_qoi(int64_t n, const int32_t* to_in, const double* tliq, const double* tsol, double Ts,
                         double Tl, double* out) {
  GS(c, n) {
    const int64_t o = to_in[c];
    double tf = __longlong_as_double(0x7ff8000000000000LL), cr = tf, lam = tf, ys = tf;
    if (tliq[c] >= 0.0 && tsol[c] >= 0.0) {
      tf = tsol[c] - tliq[c];
      cr = (Tl - Ts) / tf;
      lam = 39.4 * pow(cr, -0.317);
      ys = 59.0 / sqrt(lam) + 120.3;
    }
    out[4 * o] = tf;
    out[4 * o + 1] = cr;
    out[4 * o + 2] = lam;
    out[4 * o + 3] = ys;
  }
}

}  // namespace fvs

using namespace fvs;

extern "C" __attribute__((visibility("default"))) fvs_status fvs_query_fields_noalloc(fvs_solver s, fvs_field field,
                                                                                     double* dst, int64_t dst_len) {
  if (!s || !dst) {
    set_error("fvs_query_fields_noalloc: NULL argument");
    return FVS_ERR_ARG;
  }
  if (!s->have_props) {
    set_error("fvs_query_fields_noalloc: no properties set");
    return FVS_ERR_STATE;
  }
  fvs_mesh m = s->mesh;
  const int64_t Nc = m->Nc, Nf = m->Nf;
  int64_t need = 0;
  switch (field) {
    case FVS_T: case FVS_FS: case FVS_P: case FVS_TAG: case FVS_GRAIN: need = Nc; break;
    case FVS_U: case FVS_USTAR: need = 3 * Nc; break;
    case FVS_QOI: need = 4 * Nc; break;
    case FVS_CROSS: need = 2 * Nc; break;
    case FVS_FLUX: case FVS_FACE_CASE: need = Nf; break;
    default: set_error("fvs_query_fields_noalloc: unknown field %d", (int)field); return FVS_ERR_ARG;
  }
  if (dst_len < need) {
    set_error("fvs_query_fields_noalloc: destination holds %lld values, field needs %lld", (long long)dst_len,
              (long long)need);
    return FVS_ERR_ARG;
  }
  if (need > FVS_NOALLOC_MAX_VALUES) {
    set_error("fvs_query_fields_noalloc: field has %lld values, more than the %d this entry point can stage; "
              "use fvs_query_fields", (long long)need, FVS_NOALLOC_MAX_VALUES);
    return FVS_ERR_ARG;
  }
  double* buf = nullptr;
  FVS_TRY(noalloc_scratch(&buf));
  cudaStream_t st = s->stream;
  const int gc = stride_grid(Nc, 256), gf = stride_grid(Nf, 256);
  const double Ts = s->props.mat.T_sol, Tl = s->props.mat.T_liq;
  switch (field) {
    case FVS_T: k_na_gather<<<gc, 256, 0, st>>>(Nc, 1, m->cell_in, s->T, buf); break;
    case FVS_FS: k_na_gather<<<gc, 256, 0, st>>>(Nc, 1, m->cell_in, s->fs, buf); break;
    case FVS_P: k_na_gather<<<gc, 256, 0, st>>>(Nc, 1, m->cell_in, s->p, buf); break;
    case FVS_U: k_na_gather<<<gc, 256, 0, st>>>(Nc, 3, m->cell_in, s->u, buf); break;
    case FVS_USTAR: k_na_gather<<<gc, 256, 0, st>>>(Nc, 3, m->cell_in, s->ustar, buf); break;
    case FVS_FLUX: k_na_gather<<<gf, 256, 0, st>>>(Nf, 1, m->face_in, s->F, buf); break;
    case FVS_TAG: k_na_u8<<<gc, 256, 0, st>>>(Nc, m->cell_in, s->lm, buf); break;
    case FVS_FACE_CASE: k_na_u8<<<gf, 256, 0, st>>>(Nf, m->face_in, s->fcase, buf); break;
    case FVS_QOI: k_na_qoi<<<gc, 256, 0, st>>>(Nc, m->cell_in, s->tliq, s->tsol, Ts, Tl, buf); break;
    case FVS_CROSS: k_na_pair<<<gc, 256, 0, st>>>(Nc, m->cell_in, s->tliq, s->tsol, buf); break;
    case FVS_GRAIN: k_na_sqrt<<<gc, 256, 0, st>>>(Nc, m->cell_in, s->r2, buf); break;
    default: break;
  }
  FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  FVS_CUDA(cudaMemcpyAsync(dst, buf, need * sizeof(double), cudaMemcpyDeviceToHost, st));
  FVS_CUDA(cudaStreamSynchronize(st));
  return FVS_OK;
}
