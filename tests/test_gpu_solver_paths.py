"""Solver paths beyond the default one: the single-grid pressure solve on a
system of several liquid pockets, a refused non-finite right side, the
bench workload's jittered mesh at a size no oracle can follow (checked
through identities that hold at any size), and three choices that must not
change the answer: face-only stencils on orthogonal meshes, the AMG
hierarchy built on the face couplings of the pressure matrix, and the
Chebyshev smoother in place of weighted Jacobi."""
import numpy as np
import pytest

from fvs_inputs import box_mesh, cases
from oracle.fv import Oracle
from tests.helpers import set_state

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

TIGHT = dict(p_rtol=1e-13, mom_rtol=1e-12, e_rtol=1e-13, e_tol_T=1e-11, max_krylov_iters=4000)


@pytest.fixture(scope="module")
def fvs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import os
    from paper_1810_08572_gb300 import LIB_PATH, build
    if not os.path.exists(LIB_PATH):
        build()
    from paper_1810_08572_gb300 import fvs as f
    return f


def rel(a, b):
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


def pockets_field(m, seed=0):
    """Melt split into three pockets by two solid bands two cells wide across
    the whole mesh (no vertex is shared between pockets), plus a lone solid
    cell inside the last pocket."""
    ijk = m["cell_ijk"]
    nx, ny, nz = m["shape"]
    rng = np.random.default_rng(seed)
    T = 950.0 - rng.uniform(0.0, 20.0, len(ijk))
    band = ((ijk[:, 0] >= 4) & (ijk[:, 0] <= 5)) | ((ijk[:, 0] >= 10) & (ijk[:, 0] <= 11))
    T[band] = 800.0
    T[(ijk[:, 0] == nx - 2) & (ijk[:, 1] == ny // 2) & (ijk[:, 2] == 0)] = 800.0
    return T


@pytest.mark.parametrize("p_solver,precision", [(1, 0), (0, 0), (0, 1)])
def test_liquid_pockets_match_oracle(fvs, p_solver, precision):
    """Jittered, permuted 16x16x2 mesh with three liquid pockets (Section 2.5:
    each pocket is a separate singular block).  p_solver 1 is the paper's
    single-grid fallback (Jacobi BiCGStab), whose parts are labelled on the
    GPU from the matrix pattern; p_solver 0 is the AMG path with the labels of
    its coarsest level.  Two steps against the oracle at 1e-10 (FP64; 1e-8
    with the FP32 V-cycle at the same tight residual)."""
    m = box_mesh(16, 16, 2, cases.CAVITY, jitter=0.2, jitter_seed=41, permute_seed=42)
    T0 = pockets_field(m)
    rng = np.random.default_rng(7)
    u0 = rng.normal(scale=2e-3, size=(len(T0), 3))
    props = cases.props(p_solver=p_solver, precision=precision, **TIGHT)
    o = Oracle(m, props)
    set_state(o, T0, u0)
    M = fvs.Mesh(m)
    S = fvs.Solver(M, props)
    S.set_state(T0, u0)
    tol = 1e-10 if precision == 0 else 1e-8
    for _ in range(2):
        st_o = o.step(1e-3)
        st = S.step(1e-3)
        assert st_o["ncomp"] == 3 and st["n_components"] == 3, (st_o["ncomp"], st["n_components"])
        assert st["fallback"] == 0 and st["p_relres"] <= 1e-12
        if p_solver == 1:
            assert st["amg_levels"] == 0
        for name, ref in (("T", o.T), ("U", o.u), ("P", o.p), ("USTAR", o.u_star)):
            assert rel(S.query(name), ref) <= tol, name
        # each pocket's pressure has zero mean
        P = S.query("P")
        ijk = m["cell_ijk"][:, 0]
        for lo, hi in ((0, 3), (6, 9), (12, 15)):
            sel = (ijk >= lo) & (ijk <= hi) & o.ppe
            assert abs(P[sel].mean()) <= 1e-12 * np.abs(P).max()


def test_pressure_solve_refuses_non_finite_right_side(fvs):
    """A NaN in the right side is reported as FVS_ERR_ARG before any
    iteration runs, and the solver stays usable."""
    import torch
    m = box_mesh(10, 10, 2, cases.CAVITY, jitter=0.2, jitter_seed=3, permute_seed=4)
    M = fvs.Mesh(m)
    S = fvs.Solver(M, cases.props(**TIGHT))
    S.step(1e-3)
    rhs = torch.randn(M.n_cells, dtype=torch.float64, device="cuda")
    p = torch.zeros_like(rhs)
    rhs[17] = float("nan")
    status, its, _ = S.pressure_solve(rhs, p, 1e-10)
    assert status == fvs.FVS_ERR_ARG and its == 0
    assert "non-finite" in fvs.fvs_last_error()
    rhs[17] = float("inf")
    assert S.pressure_solve(rhs, p, 1e-10)[0] == fvs.FVS_ERR_ARG
    rhs[17] = 0.0
    status, its, rr = S.pressure_solve(rhs, p, 1e-10)
    assert status == fvs.FVS_OK and rr <= 1e-10 and torch.isfinite(p).all()
    st = S.step(1e-3)
    assert st["status"] == 0


def _wall_flux_weights(m, faces_sel):
    """For Dirichlet wall faces whose four vertices all hold the wall value,
    Eq. 11-12 reduce the conductive flux to k A (1/(n.d) + w0)(T_w - T_c);
    returns A (1/(n.d) + w0) per selected face (w0 the xi weight of the
    cross-diffusion vector J^-T (n - d/(n.d)))."""
    X = np.asarray(m["nodes"])
    f = np.asarray(m["faces"])[faces_sel]
    own = np.asarray(m["face_cells"])[faces_sel, 0]
    cells = np.asarray(m["cells"])
    Sf = 0.5 * np.cross(X[f[:, 2]] - X[f[:, 0]], X[f[:, 3]] - X[f[:, 1]])
    A = np.linalg.norm(Sf, axis=1)
    n = Sf / A[:, None]
    xf = X[f].mean(axis=1)
    xc = X[cells[own]].mean(axis=1)
    d = xf - xc
    nd = np.einsum("fi,fi->f", n, d)
    J = np.stack([d, X[f[:, 2]] - X[f[:, 0]], X[f[:, 3]] - X[f[:, 1]]], axis=1)
    t = n - d / nd[:, None]
    w = np.einsum("fij,fi->fj", np.linalg.inv(J), t)
    return A * (1.0 / nd + w[:, 0]), own


def test_jittered_full_size_identities(fvs):
    """96^3 jittered, permuted cavity (the bench workload's mesh family; BiCGStab
    on 27-point rows, AMG hierarchy with refreshes), p_rtol 1e-8, three steps
    in FP64 and in mixed precision after 30 steps of cooling.  Each step: the face-flux divergence is dt
    times the pressure residual cell by cell (Eq. 17), so its norm is at most
    p_rtol times the predictor divergence; the sensible-minus-latent energy
    change equals dt times the mean of the wall heat flows at both time
    levels (Crank-Nicolson; convection telescopes, walls carry no flow); no
    velocity in solid cells.  After the 33 steps the mixed-precision fields
    are within 1e-6 of the FP64 ones."""
    n = 96
    c = cases.config_jittered(n=n)
    m = c["mesh"]
    dt = c["dt"]
    mat = cases.AL_ALLOY
    own = np.asarray(m["face_cells"])[:, 0]
    nei = np.asarray(m["face_cells"])[:, 1]
    inner = nei >= 0
    X = np.asarray(m["nodes"])
    fc = np.asarray(m["faces"])[inner]
    Sf = 0.5 * np.cross(X[fc[:, 2]] - X[fc[:, 0]], X[fc[:, 3]] - X[fc[:, 1]])
    oi, ni = own[inner], nei[inner]
    patch = np.asarray(m["patch"])
    walls = cases.cavity_walls()
    dirichlet = [(pid, T) for pid, (typ, T) in enumerate(walls) if typ == cases.BC_DIRICHLET]
    wall_w = [(_wall_flux_weights(m, patch == pid), T) for pid, T in dirichlet]

    def wall_heat(T):
        return sum(float((mat["k"] * g * (Tw - T[o])).sum()) for (g, o), Tw in wall_w)

    out = {}
    for precision in (0, 1):
        props = cases.props(p_rtol=1e-8, mom_rtol=1e-10, e_rtol=1e-13, e_tol_T=1e-10, max_krylov_iters=2000,
                            precision=precision)
        M = fvs.Mesh(m)
        V = M.geometry(0)
        S = fvs.Solver(M, props)
        T, fs = S.query("T"), S.query("FS")
        # cool the melt near the cold wall until its first cells freeze
        # (about 25 steps at this cell size), so that the steps below renumber
        # or refresh the pressure hierarchy
        S.step(dt, 30, allow_not_converged=False)
        T, fs = S.query("T"), S.query("FS")
        for _ in range(3):
            T0, fs0 = T, fs
            st = S.step(dt)
            assert st["status"] == 0 and st["fallback"] == 0 and st["p_relres"] <= 1e-8
            T, fs = S.query("T"), S.query("FS")
            U, US, F, case = S.query("U"), S.query("USTAR"), S.query("FLUX"), S.query("FACE_CASE")
            solid = T0 <= mat["T_sol"]
            assert np.abs(U[solid]).max(initial=0.0) == 0.0
            flow = ((case == 1) | (case == 2))[inner]
            Fstar = np.einsum("fi,fi->f", Sf[flow], 0.5 * (US[oi[flow]] + US[ni[flow]]))
            divF = (np.bincount(own, weights=F, minlength=len(T))
                    - np.bincount(ni, weights=F[inner], minlength=len(T)))
            divS = (np.bincount(oi[flow], weights=Fstar, minlength=len(T))
                    - np.bincount(ni[flow], weights=Fstar, minlength=len(T)))
            assert np.linalg.norm(divF) <= 1.05e-8 * np.linalg.norm(divS)
            dE = float((V * (mat["rho"] * mat["cp"] * (T - T0) - mat["rho"] * mat["latent"] * (fs - fs0))).sum())
            gross = float((V * np.abs(mat["rho"] * mat["cp"] * (T - T0))).sum())
            Q = 0.5 * (wall_heat(T0) + wall_heat(T))
            assert abs(dE - dt * Q) <= 1e-6 * gross, (dE, dt * Q, gross)
        assert (S.query("TAG") == 0).any()
        out[precision] = {k: S.query(k) for k in ("T", "U", "P")}
        S.close()
        M.close()
    assert np.abs(out[1]["T"] - out[0]["T"]).max() <= 1e-6
    assert rel(out[1]["U"], out[0]["U"]) <= 1e-6
    assert rel(out[1]["P"], out[0]["P"]) <= 1e-6


def test_bench_workload_in_its_launch_configuration(fvs):
    """The timed workload itself: the 128^3 jittered, permuted cavity with the
    solver settings, side stream and CUDA graphs of the step benchmark, 3 + 20
    steps (cells start to freeze at step 11, after which the hierarchy is
    refreshed).  Every step converges (no step of the measured run is taken
    unconverged) without the fallback; in each of the last three the flux
    carries no divergence beyond the pressure residual (Eq. 17), only flowing
    faces carry flux and solid cells do not move.  After the 23 steps the
    mixed-precision fields are within 1e-6 of the FP64 ones."""
    import torch
    c = cases.config_jittered(n=128)
    m, dt = c["mesh"], c["dt"]
    own = np.asarray(m["face_cells"])[:, 0]
    nei = np.asarray(m["face_cells"])[:, 1]
    inner = nei >= 0
    X = np.asarray(m["nodes"])
    fc = np.asarray(m["faces"])[inner]
    Sf = 0.5 * np.cross(X[fc[:, 2]] - X[fc[:, 0]], X[fc[:, 3]] - X[fc[:, 1]])
    oi, ni = own[inner], nei[inner]
    nc = len(m["cells"])
    out = {}
    for precision in (0, 1):
        # the step benchmark's settings
        props = cases.props(p_rtol=1e-8, mom_rtol=1e-10, e_rtol=1e-10, e_tol_T=1e-6, max_e_iters=40,
                            max_krylov_iters=1000, precision=precision)
        stream = torch.cuda.Stream()
        M = fvs.Mesh(m, stream=stream)
        S = fvs.Solver(M, props, stream=stream)
        refreshed = 0
        for k in range(23):
            T0 = S.query("T") if k >= 20 else None
            st = S.step(dt)
            assert st["status"] == 0 and st["fallback"] == 0 and st["p_relres"] <= 1e-8, (k, st)
            refreshed += st["p_rebuilt"] == 2
            if T0 is None:
                continue
            U, US, F, case = S.query("U"), S.query("USTAR"), S.query("FLUX"), S.query("FACE_CASE")
            assert np.abs(U[T0 <= cases.AL_ALLOY["T_sol"]]).max(initial=0.0) == 0.0
            flowing = (case == 1) | (case == 2)
            assert np.abs(F[~flowing]).max(initial=0.0) == 0.0
            flow = flowing[inner]
            Fstar = np.einsum("fi,fi->f", Sf[flow], 0.5 * (US[oi[flow]] + US[ni[flow]]))
            divF = np.bincount(own, weights=F, minlength=nc) - np.bincount(ni, weights=F[inner], minlength=nc)
            divS = (np.bincount(oi[flow], weights=Fstar, minlength=nc)
                    - np.bincount(ni[flow], weights=Fstar, minlength=nc))
            assert np.linalg.norm(divF) <= 1.05e-8 * np.linalg.norm(divS)
        assert refreshed > 0 and (S.query("TAG") == 0).any()
        out[precision] = {k: S.query(k) for k in ("T", "U", "P")}
        S.close()
        M.close()
    # measured on this workload by the step benchmark: 3.3e-7 K, 2.5e-7, 1.4e-8
    assert np.abs(out[1]["T"] - out[0]["T"]).max() <= 1e-6
    assert rel(out[1]["U"], out[0]["U"]) <= 1e-6
    assert rel(out[1]["P"], out[0]["P"]) <= 1e-6


def _run(fvs, m, props, T0, u0, steps, dt=1e-3):
    M = fvs.Mesh(m)
    S = fvs.Solver(M, props)
    S.set_state(T0, u0)
    for _ in range(steps):
        st = S.step(dt)
        assert st["status"] == 0 and st["fallback"] == 0
    out = {k: S.query(k) for k in ("T", "U", "P", "FLUX")}
    width = M.info["max_cell_neighbours"]
    S.close()
    M.close()
    return out, width


def test_face_only_stencil_changes_nothing(fvs, monkeypatch):
    """On an orthogonal mesh the neighbour lists keep only the cells across
    the faces (7 slots); the couplings left out were exact zeros, so three
    steps with convection and a frozen band equal the 27-slot stencil's to
    rounding of the Krylov iterates (both solved to 1e-13)."""
    m = box_mesh(12, 10, 6, cases.CAVITY, permute_seed=5)
    ijk = m["cell_ijk"]
    rng = np.random.default_rng(9)
    T0 = 940.0 - rng.uniform(0.0, 10.0, len(ijk))
    T0[ijk[:, 0] == 5] = 800.0
    u0 = rng.normal(scale=2e-3, size=(len(T0), 3))
    props = cases.props(**TIGHT)
    face, wf = _run(fvs, m, props, T0, u0, 3)
    monkeypatch.setenv("FVS_FULL_STENCIL", "1")
    full, ww = _run(fvs, m, props, T0, u0, 3)
    assert wf == 7 and ww == 27
    for k in ("T", "U", "P", "FLUX"):
        assert rel(face[k], full[k]) <= 1e-11, k


def test_hierarchy_on_face_couplings_changes_only_the_iterations(fvs, monkeypatch):
    """The AMG hierarchy built on the face-coupling part of the pressure
    matrix (vertex couplings lumped into the diagonal) preconditions the same
    Krylov solve as one built on the full matrix: on a jittered mesh with
    two pockets, three steps agree to the solve tolerance."""
    m = box_mesh(40, 36, 2, cases.CAVITY, jitter=0.2, jitter_seed=81, permute_seed=82)
    T0 = pockets_field(m, seed=4)
    rng = np.random.default_rng(10)
    u0 = rng.normal(scale=2e-3, size=(len(T0), 3))
    props = cases.props(**TIGHT)
    compact, _ = _run(fvs, m, props, T0, u0, 3)
    monkeypatch.setenv("FVS_PC_COMPACT", "0")
    full, _ = _run(fvs, m, props, T0, u0, 3)
    for k in ("T", "U", "P", "FLUX"):
        assert rel(compact[k], full[k]) <= 1e-10, k


def _steps_with_stats(fvs, m, props, T0, u0, steps, dt=1e-3):
    M = fvs.Mesh(m)
    S = fvs.Solver(M, props)
    S.set_state(T0, u0)
    its = []
    for _ in range(steps):
        st = S.step(dt)
        assert st["status"] == 0 and st["fallback"] == 0 and st["p_relres"] <= 1e-12
        assert st["amg_levels"] >= 2
        its.append(st["p_its"])
    out = {k: S.query(k) for k in ("T", "U", "P", "FLUX")}
    S.close()
    M.close()
    return out, its


@pytest.mark.parametrize("jitter,precision", [(0.2, 0), (0.2, 1), (0.0, 0)])
def test_chebyshev_smoother_changes_only_the_iterations(fvs, monkeypatch, jitter, precision):
    """The Chebyshev smoother (FVS_AMG_SMOOTHER=1: on every level a
    Chebyshev polynomial in D^-1 A on [b/4, b], b the level's Gershgorin
    bound; degree 1 before and 2 after the coarse correction under BiCGStab,
    1 and 1 under CG) preconditions the same solves as weighted Jacobi: three
    steps of a multi-level hierarchy with three liquid pockets agree to the
    solve tolerance, jittered (BiCGStab, FP64 and the FP32 V-cycle) and
    orthogonal (CG), with a comparable number of iterations."""
    m = box_mesh(32, 32, 8, cases.CAVITY, jitter=jitter, jitter_seed=91, permute_seed=92)
    T0 = pockets_field(m, seed=5)
    rng = np.random.default_rng(11)
    u0 = rng.normal(scale=2e-3, size=(len(T0), 3))
    props = cases.props(precision=precision, **TIGHT)
    jac, its_j = _steps_with_stats(fvs, m, props, T0, u0, 3)
    monkeypatch.setenv("FVS_AMG_SMOOTHER", "1")
    che, its_c = _steps_with_stats(fvs, m, props, T0, u0, 3)
    tol = 1e-10 if precision == 0 else 1e-8
    for k in ("T", "U", "P"):
        assert rel(che[k], jac[k]) <= tol, (k, rel(che[k], jac[k]))
    assert sum(its_c) <= 2 * sum(its_j), (its_c, its_j)


def test_energy_line_preconditioner_changes_only_the_iterations(fvs, monkeypatch):
    """FVS_ENERGY_LINES=1: the energy system preconditioned by tridiagonal
    solves along chains of strongly coupled cells (on this mesh of thin
    cells, the z columns) instead of point-Jacobi solves the same equations:
    three steps with flow and two frozen bands agree to the solve tolerance,
    in fewer inner iterations (a CPU prototype of the same system: 18
    against 5 to 1e-13)."""
    m = box_mesh(12, 12, 64, cases.CAVITY, jitter=0.2, jitter_seed=21, permute_seed=22)
    T0 = pockets_field(m, seed=8)
    rng = np.random.default_rng(12)
    u0 = rng.normal(scale=2e-3, size=(len(T0), 3))
    props = cases.props(**TIGHT)

    def run():
        M = fvs.Mesh(m)
        S = fvs.Solver(M, props)
        S.set_state(T0, u0)
        its = 0
        for _ in range(3):
            st = S.step(1e-3)
            assert st["status"] == 0 and st["fallback"] == 0
            its += st["e_lin_its"]
        out = {k: S.query(k) for k in ("T", "U", "P", "FS")}
        S.close()
        M.close()
        return out, its

    jac, its_j = run()
    monkeypatch.setenv("FVS_ENERGY_LINES", "1")
    lin, its_l = run()
    for k in ("T", "U", "P", "FS"):
        assert rel(lin[k], jac[k]) <= 1e-10, (k, rel(lin[k], jac[k]))
    assert its_l <= 0.6 * its_j, (its_l, its_j)
