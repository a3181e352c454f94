"""The casting-like workload on the GPU: a voxelised plate with ribs and a
riser in a conduction-only steel shell (metal-mold interface coefficient,
Section 2.4.4 energy on all cells).  Small meshes against the oracle element
by element; the full-size mesh (about 4.4M metal and 2.1M mold cells) through
properties that hold at any size."""
import numpy as np
import pytest

from fvs_inputs import cases, casting_mesh
from oracle.fv import Oracle

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

TIGHT = dict(p_rtol=1e-13, mom_rtol=1e-12, e_rtol=1e-13, e_tol_T=1e-11, max_krylov_iters=2000)


@pytest.fixture(scope="module")
def fvs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1810_08572_gb300 import LIB_PATH, build
    import os
    if not os.path.exists(LIB_PATH):
        build()
    from paper_1810_08572_gb300 import fvs as f
    return f


def rel(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / (scale if scale > 0 else 1.0)


@pytest.mark.parametrize("precision", [0, 1])
def test_small_casting_matches_oracle(fvs, precision):
    """5 mm voxels (plate, ribs and riser in a one-voxel shell): the first
    step within 1e-10 of the oracle (FP64) and fifteen steps within 1e-8 K,
    FP64 or with the FP32 V-cycle at the same tight outer tolerance."""
    m = casting_mesh(0.005)
    props = cases.casting_props(precision=precision, **TIGHT)
    o = Oracle(m, props)
    M = fvs.Mesh(m)
    S = fvs.Solver(M, props)
    assert (~o.metal).sum() > 0 and o.interface.sum() > 0
    o.step(1e-3)
    S.step(1e-3)
    tol = 1e-10 if precision == 0 else 1e-8
    assert rel(S.query("T"), o.T) <= tol
    assert rel(S.query("U"), o.u) <= tol
    assert rel(S.query("P"), o.p) <= tol
    for _ in range(14):
        o.step(1e-3)
    S.step(1e-3, 14)
    assert np.abs(S.query("T") - o.T).max() <= 1e-8
    assert rel(S.query("U"), o.u) <= 1e-8
    assert np.abs(S.query("U")[~o.metal]).max() == 0.0
    assert np.abs(S.query("FS")[~o.metal]).max() == 0.0


def _face_vectors(m, sel):
    """Face vector areas 1/2 (x3 - x1) x (x4 - x2) of the selected faces."""
    X = np.asarray(m["nodes"])
    f = np.asarray(m["faces"])[sel]
    return 0.5 * np.cross(X[f[:, 2]] - X[f[:, 0]], X[f[:, 3]] - X[f[:, 1]])


def test_full_size_casting_properties(fvs):
    """The workload at its full size (0.46 mm voxels), mixed precision,
    p_rtol 1e-8, a few steps from the initial state.  Each step: pressure
    residual at target; no flow and no solid fraction in the mold; no flow in
    solid metal; flux only on flowing faces; the face-flux divergence is dt
    times the pressure residual (Eq. 17), so its norm is bounded by p_rtol
    times the predictor divergence; and the energy change of the whole
    casting plus mold equals dt times the mean heat flow through the shell's
    outer surface (orthogonal voxel walls: 2 k h (T_wall - T_cell) per face)."""
    h = 0.46e-3
    c = cases.config_casting(h)
    m = c["mesh"]
    zone = m["cell_zone"]
    nmetal, nmold = int((zone == 0).sum()), int((zone == 1).sum())
    assert 4.0e6 < nmetal < 4.8e6 and 1.8e6 < nmold < 2.6e6
    props = cases.casting_props(precision=1, p_rtol=1e-8, e_rtol=1e-13, e_tol_T=1e-10, max_krylov_iters=2000)
    M = fvs.Mesh(m)
    S = fvs.Solver(M, props)
    dt = c["dt"]
    metal = zone == 0
    mold = props["mold"]
    mat = props["material"]
    rcp = np.where(metal, mat["rho"] * mat["cp"], mold["rho"] * mold["cp"])
    rL = np.where(metal, mat["rho"] * mat["latent"], 0.0)
    own = np.asarray(m["face_cells"])[:, 0]
    nei = np.asarray(m["face_cells"])[:, 1]
    wall = nei < 0
    T_wall = props["walls"][0][1]
    inner = ~wall
    Sf = _face_vectors(m, inner)
    oi, ni = own[inner], nei[inner]

    def wall_heat(T):
        return float((2.0 * mold["k"] * h * (T_wall - T[own[wall]])).sum())

    T = S.query("T")
    fs = S.query("FS")
    assert np.all(T[metal] == 950.0) and np.all(T[~metal] == 500.0)
    for _ in range(3):
        T0, fs0 = T, fs
        st = S.step(dt)
        assert st["status"] == 0 and st["fallback"] == 0
        assert st["p_relres"] <= 1e-8
        T, fs = S.query("T"), S.query("FS")
        U, US, F = S.query("U"), S.query("USTAR"), S.query("FLUX")
        case = S.query("FACE_CASE")
        assert np.all(np.isfinite(T)) and np.all(np.isfinite(U))
        assert np.abs(U[~metal]).max() == 0.0 and np.abs(fs[~metal]).max() == 0.0
        solid = T0 <= mat["T_sol"]
        assert np.abs(U[solid]).max() == 0.0
        flow = (case == 1) | (case == 2)
        assert np.abs(F[~flow]).max() == 0.0
        # Eq. 17: div F^{n+1} = div F* - dt div(grad p) = dt (b - A p) cell by cell
        fl = flow[inner]
        Fstar = np.einsum("fi,fi->f", Sf[fl], 0.5 * (US[oi[fl]] + US[ni[fl]]))
        divF = np.bincount(own, weights=F, minlength=len(T)) - np.bincount(nei[inner], weights=F[inner],
                                                                          minlength=len(T))
        divS = (np.bincount(oi[fl], weights=Fstar, minlength=len(T))
                - np.bincount(ni[fl], weights=Fstar, minlength=len(T)))
        assert np.linalg.norm(divF) <= 1.05e-8 * np.linalg.norm(divS)
        # energy: sensible minus latent change against the wall heat flow
        dE = float((h ** 3 * (rcp * (T - T0) - rL * (fs - fs0))).sum())
        gross = float((h ** 3 * np.abs(rcp * (T - T0))).sum())
        Q = 0.5 * (wall_heat(T0) + wall_heat(T))
        assert abs(dE - dt * Q) <= 1e-6 * gross
    assert (T[metal] < 950.0).any() and (T[~metal] > 500.0).any()
