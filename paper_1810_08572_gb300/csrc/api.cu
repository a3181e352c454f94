// extern "C" entry points of include/fvs.h: argument checks, object
// lifetime, error messages.  All numerical work is in the kernels of the
// other translation units.
#include <stdarg.h>

#include <new>

#include "batch.cuh"
#include "fslaw.cuh"
#include "solver.cuh"

namespace fvs {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

thread_local Prof* g_prof = nullptr;
thread_local cudaStream_t g_alloc_stream = nullptr;
unsigned long long g_launches = 0;

Prof::~Prof() {
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
}
void Prof::label(const void* key, const char* name) {
  for (auto& kv : labels)
    if (kv.first == key) { kv.second = name; return; }
  labels.emplace_back(key, name);
}
const char* Prof::label_of(const void* key) const {
  for (auto& kv : labels)
    if (kv.first == key) return kv.second.c_str();
  return nullptr;
}
int Prof::begin(const void* key, const char* kernel, double bytes, cudaStream_t s) {
  const char* lab = label_of(key);
  if (!lab) return -1;
  std::string name = std::string(kernel) + "@" + lab;
  int cls = -1;
  for (size_t i = 0; i < classes.size(); ++i)
    if (classes[i].name == name) { cls = (int)i; break; }
  if (cls < 0) {
    classes.push_back(Cls());
    classes.back().name = name;
    cls = (int)classes.size() - 1;
  }
  while (pool.size() < used + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    pool.push_back(e);
  }
  Rec r{cls, bytes, pool[used], pool[used + 1]};
  used += 2;
  cudaEventRecord(r.a, s);
  recs.push_back(r);
  return (int)recs.size() - 1;
}
void Prof::end(int token, cudaStream_t s) { cudaEventRecord(recs[token].b, s); }
fvs_status Prof::collect() {
  for (const Rec& r : recs) {
    FVS_CUDA(cudaEventSynchronize(r.b));
    float ms = 0.f;
    FVS_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    classes[r.cls].launches += 1;
    classes[r.cls].ms += ms;
    classes[r.cls].bytes += r.bytes;
  }
  recs.clear();
  used = 0;
  return FVS_OK;
}
void Prof::reset() {
  recs.clear();
  used = 0;
  classes.clear();
}

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cached[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 132;
    cached[dev] = n;
  }
  return cached[dev];
}

static fvs_status check_device() {
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    set_error("no CUDA device available (%s)", e != cudaSuccess ? cudaGetErrorString(e) : "count 0");
    return FVS_ERR_CUDA;
  }
  return FVS_OK;
}

}  // namespace fvs

using namespace fvs;

#define FVS_API extern "C" __attribute__((visibility("default")))

FVS_API const char* fvs_last_error(void) { return g_err; }

FVS_API const char* fvs_version(void) { return "fvs 0.1 sm_103a"; }

FVS_API int64_t fvs_launch_count(void) { return (int64_t)__atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

FVS_API fvs_status fvs_mesh_create(const double* nodes_xyz, int64_t n_nodes, const int32_t* cell_nodes,
                                   int64_t n_cells, const int32_t* face_nodes, int64_t n_faces,
                                   const int32_t* face_cells, const int32_t* boundary_patch, int reorder,
                                   void* stream, fvs_mesh* out) {
  if (!out || !nodes_xyz || !cell_nodes || !face_nodes || !face_cells || !boundary_patch || n_nodes <= 0 ||
      n_cells <= 0 || n_faces <= 0) {
    set_error("fvs_mesh_create: NULL pointer or empty mesh");
    return FVS_ERR_ARG;
  }
  if (n_cells > 100000000 || n_faces > 400000000 || n_nodes > 200000000) {
    set_error("fvs_mesh_create: mesh too large for 32-bit ids");
    return FVS_ERR_ARG;
  }
  *out = nullptr;
  FVS_TRY(check_device());
  fvs_mesh m = new (std::nothrow) fvs_mesh_s();
  if (!m) return FVS_ERR_NOMEM;
  m->stream = (cudaStream_t)stream;
  AllocStream as(m->stream);
  cudaGetDevice(&m->device);
  fvs_status s = mesh_build(m, nodes_xyz, n_nodes, cell_nodes, n_cells, face_nodes, n_faces, face_cells,
                            boundary_patch, reorder);
  if (s != FVS_OK) {
    delete m;
    return s;
  }
  *out = m;
  return FVS_OK;
}

FVS_API fvs_status fvs_mesh_destroy(fvs_mesh mesh) {
  if (!mesh) return FVS_ERR_ARG;
  cudaStream_t st = mesh->stream;
  {
    AllocStream as(st);
    cudaStreamSynchronize(st);
    delete mesh;
  }
  cudaStreamSynchronize(st);
  return FVS_OK;
}

FVS_API fvs_status fvs_mesh_get_info(fvs_mesh m, fvs_mesh_info* info) {
  if (!m || !info) {
    set_error("fvs_mesh_get_info: NULL argument");
    return FVS_ERR_ARG;
  }
  info->n_cells = m->Nc;
  info->n_faces = m->Nf;
  info->n_nodes = m->Nv;
  info->n_interior_faces = m->Nfi;
  info->max_cell_neighbours = m->W;
  info->max_face_neighbours = m->WF;
  info->n_patches = m->npatch;
  info->orthogonal = m->orthogonal;
  info->total_volume = m->total_volume;
  return FVS_OK;
}

__global__ void k_unpermute(int64_t n, const int32_t* to_in, const double* src, double* dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[to_in[i]] = src[i];
}

FVS_API fvs_status fvs_mesh_geometry(fvs_mesh m, int which, double* dst, int64_t dst_len) {
  if (!m || !dst || (which != 0 && which != 1)) {
    set_error("fvs_mesh_geometry: bad argument");
    return FVS_ERR_ARG;
  }
  const int64_t n = which == 0 ? m->Nc : m->Nf;
  if (dst_len < n) {
    set_error("fvs_mesh_geometry: destination too small");
    return FVS_ERR_ARG;
  }
  AllocStream as(m->stream);
  DBuf<double> tmp;
  FVS_TRY(tmp.alloc(n));
  k_unpermute<<<stride_grid(n, 256), 256, 0, m->stream>>>(n, which == 0 ? m->cell_in.p : m->face_in.p,
                                                          which == 0 ? m->V.p : m->A.p, tmp.p); FVS_COUNT_LAUNCH();
  FVS_LAUNCH_CHECK();
  FVS_CUDA(cudaMemcpyAsync(dst, tmp.p, n * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  FVS_CUDA(cudaStreamSynchronize(m->stream));
  return FVS_OK;
}

FVS_API fvs_status fvs_solver_create(fvs_mesh mesh, void* stream, fvs_solver* out) {
  if (!mesh || !out) {
    set_error("fvs_solver_create: NULL argument");
    return FVS_ERR_ARG;
  }
  *out = nullptr;
  fvs_solver s = new (std::nothrow) fvs_solver_s();
  if (!s) return FVS_ERR_NOMEM;
  s->mesh = mesh;
  s->stream = (cudaStream_t)stream;
  AllocStream as(s->stream);
  fvs_status st = solver_alloc(s);
  if (st == FVS_OK) st = noalloc_reserve();
  if (st != FVS_OK) {
    delete s;
    return st;
  }
  *out = s;
  return FVS_OK;
}

FVS_API fvs_status fvs_solver_destroy(fvs_solver s) {
  if (!s) return FVS_ERR_ARG;
  cudaStream_t st = s->stream;
  {
    AllocStream as(st);
    cudaStreamSynchronize(st);
    delete s;
  }
  cudaStreamSynchronize(st);
  return FVS_OK;
}

FVS_API fvs_status fvs_set_properties(fvs_solver s, const fvs_props* p) {
  if (!s || !p) {
    set_error("fvs_set_properties: NULL argument");
    return FVS_ERR_ARG;
  }
  AllocStream as(s->stream);
  return solver_set_properties(s, p);
}

FVS_API fvs_status fvs_mesh_set_zones(fvs_mesh mesh, const int32_t* zone) {
  if (!mesh || !zone) {
    set_error("fvs_mesh_set_zones: NULL argument");
    return FVS_ERR_ARG;
  }
  AllocStream as(mesh->stream);
  return mesh_set_zones(mesh, zone);
}

FVS_API fvs_status fvs_set_mold(fvs_solver s, double rho, double cp, double k, double h, double T_init) {
  if (!s) {
    set_error("fvs_set_mold: NULL solver");
    return FVS_ERR_ARG;
  }
  AllocStream as(s->stream);
  return solver_set_mold(s, rho, cp, k, h, T_init);
}

FVS_API fvs_status fvs_set_grain_growth(fvs_solver s, double kp, double D_s, double r0) {
  if (!s) {
    set_error("fvs_set_grain_growth: NULL solver");
    return FVS_ERR_ARG;
  }
  AllocStream as(s->stream);
  return solver_set_grain(s, kp, D_s, r0);
}

FVS_API fvs_status fvs_set_state(fvs_solver s, const double* T, const double* u, int on_device) {
  if (!s || !T) {
    set_error("fvs_set_state: NULL argument");
    return FVS_ERR_ARG;
  }
  AllocStream as(s->stream);
  return solver_set_state(s, T, u, on_device);
}

FVS_API fvs_status fvs_step(fvs_solver s, double dt, int32_t n_steps, fvs_step_stats* last) {
  if (!s || n_steps < 0) {
    set_error("fvs_step: bad argument");
    return FVS_ERR_ARG;
  }
  fvs_status worst = FVS_OK;
  AllocStream as(s->stream);
  g_prof = &s->prof;
  for (int i = 0; i < n_steps; ++i) {
    fvs_status r = solver_step(s, dt, last);
    if (r == FVS_ERR_NOT_CONVERGED) worst = r;
    else if (r != FVS_OK) { g_prof = nullptr; return r; }
  }
  g_prof = nullptr;
  return worst;
}

FVS_API fvs_status fvs_profile_enable(fvs_solver s, int on) {
  if (!s) {
    set_error("fvs_profile_enable: NULL solver");
    return FVS_ERR_ARG;
  }
  s->prof.reset();
  s->prof.on = on != 0;
  s->prof.label(&s->K, "pressure");
  s->prof.label(&s->Kp, "pressure");   // the V-cycle on the compact operator
  s->prof.label(&s->Ke, "energy");
  s->prof.label(&s->M, "momentum");
  return FVS_OK;
}

FVS_API fvs_status fvs_profile_read(fvs_solver s, fvs_kernel_time* out, int32_t max_records, int32_t* n_records) {
  if (!s || !n_records || (max_records > 0 && !out)) {
    set_error("fvs_profile_read: bad argument");
    return FVS_ERR_ARG;
  }
  FVS_TRY(s->prof.collect());
  const int n = (int)s->prof.classes.size();
  *n_records = n;
  for (int i = 0; i < n && i < max_records; ++i) {
    const Prof::Cls& c = s->prof.classes[i];
    snprintf(out[i].name, sizeof(out[i].name), "%s", c.name.c_str());
    out[i].launches = c.launches;
    out[i].total_ms = c.ms;
    out[i].bytes = c.bytes;
  }
  return FVS_OK;
}

FVS_API fvs_status fvs_pressure_solve(fvs_solver s, const double* rhs, double* p_out, double rtol, int32_t* iters,
                                      double* relres) {
  if (!s || !rhs || !p_out || !(rtol > 0)) {
    set_error("fvs_pressure_solve: bad argument");
    return FVS_ERR_ARG;
  }
  int it = 0;
  AllocStream as(s->stream);
  fvs_status r = solver_pressure_solve(s, rhs, p_out, rtol, &it, relres);
  if (iters) *iters = it;
  return r;
}

FVS_API fvs_status fvs_query_fields(fvs_solver s, fvs_field field, double* dst, int64_t dst_len, int dst_on_device) {
  if (!s || !dst) {
    set_error("fvs_query_fields: NULL argument");
    return FVS_ERR_ARG;
  }
  if (!s->have_props) {
    set_error("fvs_query_fields: no properties set");
    return FVS_ERR_STATE;
  }
  AllocStream as(s->stream);
  return solver_query(s, field, dst, dst_len, dst_on_device);
}

FVS_API fvs_status fvs_get_time(fvs_solver s, double* time, int64_t* steps) {
  if (!s) {
    set_error("fvs_get_time: NULL argument");
    return FVS_ERR_ARG;
  }
  if (time) *time = s->time;
  if (steps) *steps = s->nstep;
  return FVS_OK;
}

FVS_API fvs_status fvs_uq_batch(fvs_mesh mesh, const fvs_props* base, int64_t n_samples, const double* inputs,
                                double dt, int32_t max_steps, const fvs_uq_options* opt_in, double* qoi_out,
                                int64_t* steps_out) {
  if (!mesh || !base || !inputs || !qoi_out || n_samples <= 0 || !(dt > 0) || max_steps <= 0) {
    set_error("fvs_uq_batch: bad argument");
    return FVS_ERR_ARG;
  }
  fvs_uq_options opt{};
  if (opt_in) opt = *opt_in;
  const int mode = opt.mode;
  if (mode != FVS_UQ_LOCKSTEP && mode != FVS_UQ_STREAMS && mode != FVS_UQ_SURROGATE) {
    set_error("fvs_uq_batch: mode %d is not available (0 lockstep batch, 1 independent solves, 2 surrogate)", mode);
    return FVS_ERR_ARG;
  }
  if (opt.qoi_kind != FVS_QOI_MEANS && opt.qoi_kind != FVS_QOI_EXTREMES) {
    set_error("fvs_uq_batch: qoi_kind %d is not available", opt.qoi_kind);
    return FVS_ERR_ARG;
  }
  if (opt.grain_Ds < 0.0 || (opt.grain_Ds > 0.0 && !(opt.grain_kp > 0.0 && opt.grain_kp < 1.0 && opt.grain_r0 >= 0.0))) {
    set_error("fvs_uq_batch: invalid grain-growth data (0 < kp < 1, D_s >= 0, r0 >= 0)");
    return FVS_ERR_ARG;
  }
  UqSpec spec;
  spec.qoi_kind = opt.qoi_kind;
  spec.grain_kp = opt.grain_kp;
  spec.grain_Ds = opt.grain_Ds;
  spec.grain_r0 = opt.grain_r0;
  spec.T_out = opt.T_out;
  spec.u_out = opt.u_out;
  spec.p_out = opt.p_out;
  spec.T_liq.resize(n_samples);
  const bool shift = opt.liquidus_T0 != 0.0 || opt.liquidus_slope != 0.0;
  for (int64_t i = 0; i < n_samples; ++i) {
    const double C0 = inputs[3 * i + 2];
    spec.T_liq[i] = shift ? opt.liquidus_T0 + opt.liquidus_slope * C0 : base->mat.T_liq;
    if (!fs_law_valid(base->mat, spec.T_liq[i])) {
      set_error("fvs_uq_batch: sample %lld gives a liquidus of %.3f K that does not suit the solid-fraction law "
                "(below the solidus, or outside T_sol + T_eps < T_liq < T_f for Scheil)", (long long)i,
                spec.T_liq[i]);
      return FVS_ERR_ARG;
    }
  }
  if (mode == FVS_UQ_SURROGATE)
    return uq_surrogate(mesh, base, n_samples, inputs, dt, max_steps, opt, spec, qoi_out, steps_out);
  if (opt.used_plain)
    for (int64_t i = 0; i < n_samples; ++i) opt.used_plain[i] = 1;
  if (mode == FVS_UQ_LOCKSTEP) return batch_run(mesh, base, n_samples, inputs, dt, max_steps, spec, qoi_out, steps_out);
  return uq_batch(mesh, base, n_samples, inputs, dt, max_steps, opt.n_streams, spec, qoi_out, steps_out);
}
