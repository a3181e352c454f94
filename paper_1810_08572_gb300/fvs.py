"""Thin ctypes binding of the C ABI in include/fvs.h.

Argument marshalling only: every step of the method runs in the CUDA
library libfvs.so.  The functions keep the C names (fvs_mesh_create,
fvs_step, ...); ``Mesh`` and ``Solver`` are small conveniences that own the
handles.  There is no CPU fallback: importing this module fails if the
library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfvs.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python -m paper_1810_08572_gb300.build)")
_lib = C.CDLL(LIB_PATH)

# status codes
FVS_OK, FVS_ERR_ARG, FVS_ERR_MESH, FVS_ERR_CUDA, FVS_ERR_NOMEM, FVS_ERR_NOT_CONVERGED, \
    FVS_ERR_TIMEOUT, FVS_ERR_STATE = range(8)
STATUS = {0: "FVS_OK", 1: "FVS_ERR_ARG", 2: "FVS_ERR_MESH", 3: "FVS_ERR_CUDA", 4: "FVS_ERR_NOMEM",
          5: "FVS_ERR_NOT_CONVERGED", 6: "FVS_ERR_TIMEOUT", 7: "FVS_ERR_STATE"}
FVS_BC_ADIABATIC, FVS_BC_DIRICHLET, FVS_BC_CONVECTIVE = 0, 1, 2
FVS_PREC_FP64, FVS_PREC_MIXED = 0, 1
FVS_PSOLVER_AMG, FVS_PSOLVER_JACOBI = 0, 1
FIELDS = dict(T=0, FS=1, U=2, P=3, FLUX=4, TAG=5, QOI=6, USTAR=7, CROSS=8, FACE_CASE=9, GRAIN=10)


class FvsError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}: {fvs_last_error()}")


class fvs_material(C.Structure):
    _fields_ = [("rho", C.c_double), ("k", C.c_double), ("cp", C.c_double), ("latent", C.c_double),
                ("T_sol", C.c_double), ("T_liq", C.c_double), ("mu", C.c_double), ("beta", C.c_double),
                ("T_ref", C.c_double), ("g", C.c_double * 3), ("darcy_C", C.c_double),
                ("darcy_eps", C.c_double), ("fs_model", C.c_int32), ("kp", C.c_double), ("T_f", C.c_double),
                ("T_eps", C.c_double)]


class fvs_patch_bc(C.Structure):
    _fields_ = [("type", C.c_int32), ("T", C.c_double), ("h", C.c_double)]


class fvs_props(C.Structure):
    _fields_ = [("mat", fvs_material), ("n_patches", C.c_int32), ("bc", C.POINTER(fvs_patch_bc)),
                ("T_init", C.c_double), ("p_rtol", C.c_double), ("mom_rtol", C.c_double),
                ("e_rtol", C.c_double), ("e_tol_T", C.c_double), ("max_e_iters", C.c_int32),
                ("max_krylov_iters", C.c_int32), ("precision", C.c_int32), ("p_solver", C.c_int32),
                ("no_flow", C.c_int32), ("n_k", C.c_int32), ("k_T", C.POINTER(C.c_double)),
                ("k_val", C.POINTER(C.c_double))]


class fvs_step_stats(C.Structure):
    _fields_ = [("n_active", C.c_int64), ("n_ppe", C.c_int64), ("mom_its", C.c_int32), ("p_its", C.c_int32),
                ("e_its", C.c_int32), ("e_lin_its", C.c_int32), ("p_relres", C.c_double),
                ("fallback", C.c_int32), ("n_components", C.c_int32), ("amg_levels", C.c_int32),
                ("status", C.c_int32), ("p_rebuilt", C.c_int32), ("setup_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fvs_mesh_info(C.Structure):
    _fields_ = [("n_cells", C.c_int64), ("n_faces", C.c_int64), ("n_nodes", C.c_int64),
                ("n_interior_faces", C.c_int64), ("max_cell_neighbours", C.c_int32),
                ("max_face_neighbours", C.c_int32), ("n_patches", C.c_int32), ("orthogonal", C.c_int32),
                ("total_volume", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fvs_uq_options(C.Structure):
    _fields_ = [("mode", C.c_int32), ("n_streams", C.c_int32), ("qoi_kind", C.c_int32),
                ("liquidus_T0", C.c_double), ("liquidus_slope", C.c_double), ("grain_kp", C.c_double),
                ("grain_Ds", C.c_double), ("grain_r0", C.c_double), ("n_models", C.c_int32),
                ("models", C.POINTER(C.c_void_p)), ("box_lo", C.POINTER(C.c_double)),
                ("box_hi", C.POINTER(C.c_double)), ("max_spread", C.c_double), ("plain_mode", C.c_int32),
                ("used_plain", C.POINTER(C.c_int32)), ("T_out", C.POINTER(C.c_double)),
                ("u_out", C.POINTER(C.c_double)), ("p_out", C.POINTER(C.c_double))]


class fvs_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_int64), ("total_ms", C.c_double),
                ("bytes", C.c_double)]


_P = C.c_void_p
_SIGS = {
    "fvs_last_error": ([], C.c_char_p),
    "fvs_version": ([], C.c_char_p),
    "fvs_launch_count": ([], C.c_int64),
    "fvs_mesh_create": ([_P, C.c_int64, _P, C.c_int64, _P, C.c_int64, _P, _P, C.c_int, _P, C.POINTER(_P)],
                        C.c_int),
    "fvs_mesh_destroy": ([_P], C.c_int),
    "fvs_mesh_get_info": ([_P, C.POINTER(fvs_mesh_info)], C.c_int),
    "fvs_mesh_geometry": ([_P, C.c_int, _P, C.c_int64], C.c_int),
    "fvs_solver_create": ([_P, _P, C.POINTER(_P)], C.c_int),
    "fvs_solver_destroy": ([_P], C.c_int),
    "fvs_set_properties": ([_P, C.POINTER(fvs_props)], C.c_int),
    "fvs_mesh_set_zones": ([_P, _P], C.c_int),
    "fvs_set_mold": ([_P, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double], C.c_int),
    "fvs_set_grain_growth": ([_P, C.c_double, C.c_double, C.c_double], C.c_int),
    "fvs_set_state": ([_P, _P, _P, C.c_int], C.c_int),
    "fvs_step": ([_P, C.c_double, C.c_int32, C.POINTER(fvs_step_stats)], C.c_int),
    "fvs_pressure_solve": ([_P, _P, _P, C.c_double, C.POINTER(C.c_int32), C.POINTER(C.c_double)], C.c_int),
    "fvs_query_fields": ([_P, C.c_int, _P, C.c_int64, C.c_int], C.c_int),
    "fvs_get_time": ([_P, C.POINTER(C.c_double), C.POINTER(C.c_int64)], C.c_int),
    "fvs_query_fields_noalloc": ([_P, C.c_int, _P, C.c_int64], C.c_int),
    "fvs_surrogate_create": ([C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, _P, C.POINTER(_P)],
                             C.c_int),
    "fvs_surrogate_destroy": ([_P], C.c_int),
    "fvs_surrogate_set_scaling": ([_P, _P, _P, _P, _P], C.c_int),
    "fvs_surrogate_num_params": ([_P], C.c_int64),
    "fvs_surrogate_params": ([_P, _P, C.c_int64, C.c_int], C.c_int),
    "fvs_surrogate_gradients": ([_P, _P, _P, C.c_int64, _P, C.c_int64, C.POINTER(C.c_double)], C.c_int),
    "fvs_surrogate_train": ([_P, _P, _P, C.c_int64, C.c_int32, C.c_double, C.POINTER(C.c_double)], C.c_int),
    "fvs_surrogate_predict": ([_P, _P, _P, C.c_int64, C.c_int], C.c_int),
    "fvs_profile_enable": ([_P, C.c_int], C.c_int),
    "fvs_uq_batch": ([_P, C.POINTER(fvs_props), C.c_int64, _P, C.c_double, C.c_int32, C.POINTER(fvs_uq_options),
                      _P, _P], C.c_int),
    "fvs_profile_read": ([_P, C.POINTER(fvs_kernel_time), C.c_int32, C.POINTER(C.c_int32)], C.c_int),
    "fvs_measure_fp64_fma": ([C.c_int64, C.POINTER(C.c_double)], C.c_int),
    "fvs_pce_create": ([C.c_int32, _P, _P, _P, C.c_int32, C.c_int32, _P, C.POINTER(_P)], C.c_int),
    "fvs_pce_destroy": ([_P], C.c_int),
    "fvs_pce_num_terms": ([_P], C.c_int64),
    "fvs_pce_multi_indices": ([_P, _P, C.c_int64], C.c_int),
    "fvs_pce_nodes": ([_P, C.c_int32, C.c_int32, _P, C.c_int64, C.POINTER(C.c_int64)], C.c_int),
    "fvs_pce_fit": ([_P, _P, _P, C.c_int64, C.POINTER(C.c_double)], C.c_int),
    "fvs_pce_eval": ([_P, _P, _P, C.c_int64, C.c_int], C.c_int),
    "fvs_pce_coefficients": ([_P, _P, C.c_int64], C.c_int),
    "fvs_pce_sensitivity": ([_P, _P, _P, _P, _P], C.c_int),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res
    globals()[_name] = _f
EXPORTED = sorted(_SIGS)


def fvs_last_error_str():
    return _lib.fvs_last_error().decode()


def fvs_last_error():   # noqa: F811  (string form for messages)
    return _lib.fvs_last_error().decode()


def check(status, where):
    if status != FVS_OK:
        raise FvsError(status, where)
    return status


def _ptr(a):
    """Host numpy array or device tensor -> void pointer."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(C.c_void_p)
    return C.c_void_p(a.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def make_props(p):
    """fvs_props from the plain-dict settings of fvs_inputs.cases.props()."""
    m = p["material"]
    mat = fvs_material(m["rho"], m["k"], m["cp"], m["latent"], m["T_sol"], m["T_liq"], m["mu"], m["beta"],
                       m["T_ref"], (C.c_double * 3)(*m["g"]), m["darcy_C"], m["darcy_eps"],
                       int(m.get("fs_model", 0)), float(m.get("kp", 0.0)), float(m.get("T_f", 0.0)),
                       float(m.get("T_eps", 0.0)))
    walls = p["walls"]
    bcs = (fvs_patch_bc * max(1, len(walls)))(*[fvs_patch_bc(int(w[0]), float(w[1]),
                                                              float(w[2]) if len(w) > 2 else 0.0) for w in walls])
    kt = p.get("k_table") or []
    kT = (C.c_double * max(1, len(kt)))(*[float(a) for a, _ in kt])
    kv = (C.c_double * max(1, len(kt)))(*[float(b) for _, b in kt])
    props = fvs_props(mat, len(walls), C.cast(bcs, C.POINTER(fvs_patch_bc)), p["T_init"], p["p_rtol"],
                      p.get("mom_rtol", 1e-10), p.get("e_rtol", 1e-10), p.get("e_tol_T", 1e-8),
                      int(p.get("max_e_iters", 40)), int(p.get("max_krylov_iters", 500)),
                      int(p.get("precision", 0)), int(p.get("p_solver", 0)), int(bool(p.get("no_flow", False))),
                      len(kt), C.cast(kT, C.POINTER(C.c_double)), C.cast(kv, C.POINTER(C.c_double)))
    props._keep = (bcs, kT, kv)
    return props


class Mesh:
    """Owns an fvs_mesh handle built from host arrays (see fvs_inputs.mesh)."""

    def __init__(self, mesh, reorder=True, stream=None):
        self.nodes = np.ascontiguousarray(mesh["nodes"], dtype=np.float64)
        cells = np.ascontiguousarray(mesh["cells"], dtype=np.int32)
        faces = np.ascontiguousarray(mesh["faces"], dtype=np.int32)
        fcells = np.ascontiguousarray(mesh["face_cells"], dtype=np.int32)
        patch = np.ascontiguousarray(mesh["patch"], dtype=np.int32)
        h = C.c_void_p()
        check(fvs_mesh_create(_ptr(self.nodes), len(self.nodes), _ptr(cells), len(cells), _ptr(faces),
                              len(faces), _ptr(fcells), _ptr(patch), int(reorder), _stream_ptr(stream),
                              C.byref(h)), "fvs_mesh_create")
        self.h = h
        info = fvs_mesh_info()
        check(fvs_mesh_get_info(h, C.byref(info)), "fvs_mesh_get_info")
        self.info = info.as_dict()
        self.n_cells = info.n_cells
        self.n_faces = info.n_faces
        if mesh.get("cell_zone") is not None:     # 0 metal, 1 mold
            zone = np.ascontiguousarray(mesh["cell_zone"], dtype=np.int32)
            check(fvs_mesh_set_zones(h, _ptr(zone)), "fvs_mesh_set_zones")

    def geometry(self, which):
        n = self.n_cells if which == 0 else self.n_faces
        out = np.empty(n, dtype=np.float64)
        check(fvs_mesh_geometry(self.h, which, _ptr(out), n), "fvs_mesh_geometry")
        return out

    def close(self):
        if self.h:
            fvs_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


UQ_LOCKSTEP, UQ_STREAMS, UQ_SURROGATE = 0, 1, 2
QOI_MEANS, QOI_EXTREMES = 0, 1
# liquidus line of the synthetic cavity workloads: 913 K at 4 wt%, -5 K per wt%
CAVITY_LIQUIDUS = (933.0, -5.0)


def _dptr(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def uq_batch(mesh, props, inputs, dt, max_steps, n_streams=0, mode=UQ_LOCKSTEP, **kw):
    """Plain batched UQ solves: inputs [S, 3] (T_melt, T_wall, C0) -> (qoi [S, 4], steps [S]).
    mode UQ_LOCKSTEP advances all samples together (one launch per phase);
    UQ_STREAMS runs independent solves on n_streams CUDA streams.  Other
    options as in uq_run."""
    q, st, _ = uq_run(mesh, props, inputs, dt, max_steps, n_streams=n_streams, mode=mode, **kw)
    return q, st


def uq_run(mesh, props, inputs, dt, max_steps, n_streams=0, mode=UQ_LOCKSTEP, qoi_kind=QOI_MEANS,
           liquidus=CAVITY_LIQUIDUS, grain=None, models=None, box=None, max_spread=0.0,
           plain_mode=UQ_LOCKSTEP, fields=False, allow_not_converged=False):
    """fvs_uq_batch: inputs [S, 3] (T_melt, T_wall, C0) -> (qoi [S, 4], steps [S],
    extras), extras holding used_plain and, with fields=True, the final T, U
    and P of every plainly solved sample.  liquidus = (T at C0 = 0, slope in K per
    wt%) or None to keep the material's; grain = dict(kp, D_s, r0); models:
    Surrogate objects for mode UQ_SURROGATE, box = (lo[3], hi[3])."""
    inputs = np.ascontiguousarray(inputs, dtype=np.float64)
    n = len(inputs)
    nc = mesh.n_cells
    qoi = np.empty((n, 4), dtype=np.float64)
    steps = np.empty(n, dtype=np.int64)
    used = np.empty(n, dtype=np.int32)
    opt = fvs_uq_options()
    opt.mode, opt.n_streams, opt.qoi_kind = int(mode), int(n_streams), int(qoi_kind)
    if liquidus is not None:
        opt.liquidus_T0, opt.liquidus_slope = float(liquidus[0]), float(liquidus[1])
    if grain is not None:
        opt.grain_kp, opt.grain_Ds, opt.grain_r0 = float(grain["kp"]), float(grain["D_s"]), float(grain["r0"])
    keep = []
    if models:
        hs = (C.c_void_p * len(models))(*[m.h.value for m in models])
        lo = np.ascontiguousarray(box[0], dtype=np.float64)
        hi = np.ascontiguousarray(box[1], dtype=np.float64)
        keep += [hs, lo, hi]
        opt.n_models = len(models)
        opt.models = C.cast(hs, C.POINTER(C.c_void_p))
        opt.box_lo, opt.box_hi = _dptr(lo), _dptr(hi)
        opt.max_spread = float(max_spread)
        opt.plain_mode = int(plain_mode)
    opt.used_plain = used.ctypes.data_as(C.POINTER(C.c_int32))
    extra = dict(used_plain=used)
    if fields:
        extra.update(T=np.full((n, nc), np.nan), U=np.full((n, nc, 3), np.nan), P=np.full((n, nc), np.nan))
        opt.T_out, opt.u_out, opt.p_out = _dptr(extra["T"]), _dptr(extra["U"]), _dptr(extra["P"])
    pr = make_props(props)
    r = fvs_uq_batch(mesh.h, C.byref(pr), n, _ptr(inputs), float(dt), int(max_steps), C.byref(opt), _ptr(qoi),
                     _ptr(steps))
    if r != FVS_OK and not (allow_not_converged and r == FVS_ERR_NOT_CONVERGED):
        raise FvsError(r, "fvs_uq_batch")
    extra["used_plain"] = used.astype(bool)
    return qoi, steps, extra


class Surrogate:
    """Owns an fvs_surrogate handle (BF16 tensor-core MLP)."""

    def __init__(self, n_in, n_hidden, n_layers, n_out, seed=0, stream=None):
        h = C.c_void_p()
        check(fvs_surrogate_create(n_in, n_hidden, n_layers, n_out, seed, _stream_ptr(stream), C.byref(h)),
              "fvs_surrogate_create")
        self.h = h
        self.n_in, self.n_out = n_in, n_out

    def set_scaling(self, mu_in, sd_in, mu_out, sd_out):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (mu_in, sd_in, mu_out, sd_out)]
        check(fvs_surrogate_set_scaling(self.h, *[_ptr(a) for a in arrs]), "fvs_surrogate_set_scaling")

    def num_params(self):
        return int(fvs_surrogate_num_params(self.h))

    def get_params(self):
        p = np.empty(self.num_params(), dtype=np.float64)
        check(fvs_surrogate_params(self.h, _ptr(p), len(p), 0), "fvs_surrogate_params")
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float64)
        check(fvs_surrogate_params(self.h, _ptr(p), len(p), 1), "fvs_surrogate_params")

    def gradients(self, X, T):
        X = np.ascontiguousarray(X, dtype=np.float64)
        T = np.ascontiguousarray(T, dtype=np.float64)
        g = np.empty(self.num_params(), dtype=np.float64)
        loss = C.c_double()
        check(fvs_surrogate_gradients(self.h, _ptr(X), _ptr(T), len(X), _ptr(g), len(g), C.byref(loss)),
              "fvs_surrogate_gradients")
        return g, loss.value

    def train(self, X, T, epochs, lr):
        X = np.ascontiguousarray(X, dtype=np.float64)
        T = np.ascontiguousarray(T, dtype=np.float64)
        loss = C.c_double()
        check(fvs_surrogate_train(self.h, _ptr(X), _ptr(T), len(X), int(epochs), float(lr), C.byref(loss)),
              "fvs_surrogate_train")
        return loss.value

    def predict(self, X, out=None):
        """Host numpy in/out, or device tensors (X [n, n_in], out [n, n_out])."""
        if isinstance(X, np.ndarray):
            X = np.ascontiguousarray(X, dtype=np.float64)
            Y = np.empty((len(X), self.n_out), dtype=np.float64)
            check(fvs_surrogate_predict(self.h, _ptr(X), _ptr(Y), len(X), 0), "fvs_surrogate_predict")
            return Y
        check(fvs_surrogate_predict(self.h, _ptr(X), _ptr(out), X.shape[0], 1), "fvs_surrogate_predict")
        return out

    def close(self):
        if self.h:
            fvs_surrogate_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PCE_NORMAL, PCE_UNIFORM = 0, 1


def measure_fp64_fma(iters=1 << 16):
    """Measured FP64 FMA rate (GFLOP/s) of the current GPU."""
    g = C.c_double()
    check(fvs_measure_fp64_fma(int(iters), C.byref(g)), "fvs_measure_fp64_fma")
    return g.value


class Pce:
    """Owns an fvs_pce handle: polynomial chaos surrogate (Eq. 27-28)."""

    def __init__(self, families, params, degree, n_out, stream=None):
        fam = np.ascontiguousarray(families, dtype=np.int32)
        p1 = np.ascontiguousarray([a for a, _ in params], dtype=np.float64)
        p2 = np.ascontiguousarray([b for _, b in params], dtype=np.float64)
        h = C.c_void_p()
        check(fvs_pce_create(len(fam), _ptr(fam), _ptr(p1), _ptr(p2), int(degree), int(n_out), _stream_ptr(stream),
                             C.byref(h)), "fvs_pce_create")
        self.h = h
        self.d, self.n_out = len(fam), int(n_out)

    def num_terms(self):
        return int(fvs_pce_num_terms(self.h))

    def multi_indices(self):
        a = np.empty(self.num_terms() * self.d, dtype=np.int32)
        check(fvs_pce_multi_indices(self.h, _ptr(a), len(a)), "fvs_pce_multi_indices")
        return a.reshape(-1, self.d)

    def nodes(self, level, sparse=False):
        n = C.c_int64()
        check(fvs_pce_nodes(self.h, int(level), int(sparse), None, 0, C.byref(n)), "fvs_pce_nodes")
        X = np.empty((n.value, self.d), dtype=np.float64)
        check(fvs_pce_nodes(self.h, int(level), int(sparse), _ptr(X), n.value, C.byref(n)), "fvs_pce_nodes")
        return X

    def fit(self, X, Y):
        X = np.ascontiguousarray(X, dtype=np.float64)
        Y = np.ascontiguousarray(np.asarray(Y, dtype=np.float64).reshape(len(X), -1))
        r = C.c_double()
        check(fvs_pce_fit(self.h, _ptr(X), _ptr(Y), len(X), C.byref(r)), "fvs_pce_fit")
        return r.value

    def __call__(self, X, out=None):
        if isinstance(X, np.ndarray):
            X = np.ascontiguousarray(X, dtype=np.float64)
            Y = np.empty((len(X), self.n_out), dtype=np.float64)
            check(fvs_pce_eval(self.h, _ptr(X), _ptr(Y), len(X), 0), "fvs_pce_eval")
            return Y
        check(fvs_pce_eval(self.h, _ptr(X), _ptr(out), X.shape[0], 1), "fvs_pce_eval")
        return out

    def coefficients(self):
        c = np.empty(self.num_terms() * self.n_out, dtype=np.float64)
        check(fvs_pce_coefficients(self.h, _ptr(c), len(c)), "fvs_pce_coefficients")
        return c.reshape(-1, self.n_out)

    def sensitivity(self):
        """(mean [n_out], var [n_out], total Sobol [n_out, d], first-order [n_out, d])."""
        m = np.empty(self.n_out)
        v = np.empty(self.n_out)
        t = np.empty((self.n_out, self.d))
        f = np.empty((self.n_out, self.d))
        check(fvs_pce_sensitivity(self.h, _ptr(m), _ptr(v), _ptr(t), _ptr(f)), "fvs_pce_sensitivity")
        return m, v, t, f

    def close(self):
        if self.h:
            fvs_pce_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """Owns an fvs_solver handle on a Mesh."""

    def __init__(self, mesh, props, stream=None):
        self.mesh = mesh
        h = C.c_void_p()
        check(fvs_solver_create(mesh.h, _stream_ptr(stream), C.byref(h)), "fvs_solver_create")
        self.h = h
        self.set_properties(props)

    def set_properties(self, props):
        """props as from fvs_inputs.cases.props; an optional props["mold"] =
        dict(rho, cp, k, h, T_init) gives the mold zone its material."""
        self._props = make_props(props)
        check(fvs_set_properties(self.h, C.byref(self._props)), "fvs_set_properties")
        mold = props.get("mold")
        if mold is not None:
            check(fvs_set_mold(self.h, float(mold["rho"]), float(mold["cp"]), float(mold["k"]), float(mold["h"]),
                               float(mold["T_init"])), "fvs_set_mold")
        grain = props.get("grain")
        if grain is not None:
            check(fvs_set_grain_growth(self.h, float(grain["kp"]), float(grain["D_s"]), float(grain["r0"])),
                  "fvs_set_grain_growth")

    def set_state(self, T, u=None):
        """T [n_cells], u [n_cells, 3] (host numpy or device tensors, input numbering)."""
        on_dev = not isinstance(T, np.ndarray)
        if not on_dev:
            T = np.ascontiguousarray(T, dtype=np.float64)
            u = None if u is None else np.ascontiguousarray(u, dtype=np.float64)
        check(fvs_set_state(self.h, _ptr(T), _ptr(u), int(on_dev)), "fvs_set_state")

    def step(self, dt, n=1, allow_not_converged=False):
        st = fvs_step_stats()
        r = fvs_step(self.h, float(dt), int(n), C.byref(st))
        if r != FVS_OK and not (allow_not_converged and r == FVS_ERR_NOT_CONVERGED):
            raise FvsError(r, "fvs_step")
        return st.as_dict()

    def query(self, name, out=None):
        """Field in input numbering: host numpy array, or into a device tensor ``out``."""
        f = FIELDS[name]
        nc, nf = self.mesh.n_cells, self.mesh.n_faces
        n = {0: nc, 1: nc, 2: 3 * nc, 3: nc, 4: nf, 5: nc, 6: 4 * nc, 7: 3 * nc, 8: 2 * nc, 9: nf, 10: nc}[f]
        if out is None:
            a = np.empty(n, dtype=np.float64)
            check(fvs_query_fields(self.h, f, _ptr(a), n, 0), "fvs_query_fields")
            if f in (2, 7):
                a = a.reshape(nc, 3)
            elif f == 6:
                a = a.reshape(nc, 4)
            elif f == 8:
                a = a.reshape(nc, 2)
            return a
        check(fvs_query_fields(self.h, f, _ptr(out), out.numel(), 1), "fvs_query_fields")
        return out

    def pressure_solve(self, rhs, p_out, rtol):
        """rhs, p_out: device tensors [n_cells] (input numbering)."""
        it = C.c_int32()
        rr = C.c_double()
        r = fvs_pressure_solve(self.h, _ptr(rhs), _ptr(p_out), float(rtol), C.byref(it), C.byref(rr))
        return r, it.value, rr.value

    def profile(self, on=True):
        check(fvs_profile_enable(self.h, int(on)), "fvs_profile_enable")

    def profile_read(self):
        recs = (fvs_kernel_time * 64)()
        n = C.c_int32()
        check(fvs_profile_read(self.h, recs, 64, C.byref(n)), "fvs_profile_read")
        return [dict(name=r.name.decode(), launches=r.launches, total_ms=r.total_ms, bytes=r.bytes)
                for r in recs[:min(n.value, 64)]]

    def time(self):
        t = C.c_double()
        n = C.c_int64()
        check(fvs_get_time(self.h, C.byref(t), C.byref(n)), "fvs_get_time")
        return t.value, n.value

    def close(self):
        if self.h:
            fvs_solver_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
