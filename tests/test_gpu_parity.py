"""GPU path against the CPU oracle, element by element, through the C ABI.

Bar (FP64 path): <= 1e-10 relative after one step, <= 1e-6 K in temperature
after 200 steps of the 32x32x4 cavity.  Relative errors are measured against
the largest magnitude of each field.
"""
import numpy as np
import pytest

from fvs_inputs import box_mesh, cases, zones_inner_box
from oracle.fv import Oracle
from tests.helpers import frozen_corner_field, set_state

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


def make_pair(fvs, mesh, props, T0=None, u0=None, reorder=True):
    o = Oracle(mesh, props)
    M = fvs.Mesh(mesh, reorder=reorder)
    S = fvs.Solver(M, props)
    if T0 is not None:
        set_state(o, T0, u0)
        S.set_state(T0, u0)
    return o, M, S


def compare(o, S, tol, fields=("T", "U", "P", "FLUX", "USTAR")):
    """Max-abs error over the largest magnitude of each field.  The face flux
    of Eq. 17 is a difference of two nearly equal terms (A n.u*_f and the
    pressure term), so its error is measured against the larger of the two."""
    ref = dict(T=o.T, U=o.u, P=o.p, FLUX=o.F, USTAR=o.u_star, FS=o.fs)
    out = {}
    for name in fields:
        got = S.query(name)
        if name == "FLUX":
            g = o.g
            fstar = g.Af * np.einsum("fi,fi->f", g.n, g.Avg @ o.u_star)
            out[name] = np.abs(got - o.F).max() / max(np.abs(fstar).max(), np.abs(o.F).max(), 1e-300)
        else:
            out[name] = rel(got, ref[name])
    bad = {k: v for k, v in out.items() if not v <= tol}
    assert not bad, out
    return out


def test_geometry_matches(fvs):
    m = box_mesh(9, 7, 5, cases.CAVITY, jitter=0.2, jitter_seed=4, permute_seed=5)
    o = Oracle(m, cases.props())
    M = fvs.Mesh(m)
    assert rel(M.geometry(0), o.g.V) < 1e-13
    assert rel(M.geometry(1), o.g.Af) < 1e-13
    assert M.info["orthogonal"] == 0
    assert abs(M.info["total_volume"] - 0.1 * 0.1 * 0.0125) < 1e-15
    # an orthogonal mesh couples a cell to the cells across its faces only
    M2 = fvs.Mesh(box_mesh(6, 5, 4, cases.CAVITY))
    assert M2.info["orthogonal"] == 1 and M2.info["max_cell_neighbours"] == 7


def test_one_step_cavity(fvs):
    """32x32x4 cavity, cold x = 0 wall: one step from rest at 950 K."""
    c = cases.config_small()
    props = cases.props(**TIGHT)
    o, M, S = make_pair(fvs, c["mesh"], props)
    o.step(1e-3)
    S.step(1e-3)
    compare(o, S, 1e-10)


@pytest.mark.parametrize("reorder", [True, False])
def test_one_step_jittered_with_solid(fvs, reorder):
    """Jittered, permuted 16x16x2 mesh with a frozen block and a lone solid
    cell, a random initial velocity: every face case, cross diffusion,
    smearing and renumbering are exercised."""
    m = box_mesh(16, 16, 2, cases.CAVITY, jitter=0.2, jitter_seed=21, permute_seed=22)
    T0 = frozen_corner_field(m)
    rng = np.random.default_rng(3)
    u0 = rng.normal(scale=2e-3, size=(len(T0), 3))
    props = cases.props(**TIGHT)
    o, M, S = make_pair(fvs, m, props, T0, u0, reorder=reorder)
    o.step(1e-3)
    st = S.step(1e-3)
    assert st["n_active"] == int(o.lm.sum())
    assert st["n_ppe"] == int(o.ppe.sum())
    cases_gpu = S.query("FACE_CASE")
    assert np.array_equal(cases_gpu.astype(int), o.case)
    assert np.array_equal(S.query("TAG").astype(bool), o.lm)
    compare(o, S, 1e-10)
    # a second step uses the Adams-Bashforth history of the first
    o.step(1e-3)
    S.step(1e-3)
    compare(o, S, 1e-10)


def test_pressure_solve_matches_oracle(fvs):
    """fvs_pressure_solve on the oracle's right side of the last step."""
    import torch
    m = box_mesh(12, 12, 3, cases.CAVITY, jitter=0.2, jitter_seed=31, permute_seed=32)
    T0 = frozen_corner_field(m, seed=2)
    rng = np.random.default_rng(5)
    u0 = rng.normal(scale=2e-3, size=(len(T0), 3))
    o, M, S = make_pair(fvs, m, cases.props(**TIGHT), T0, u0)
    o.step(1e-3)
    S.step(1e-3)
    rhs = torch.tensor(o.b_ppe, dtype=torch.float64, device="cuda")
    p = torch.zeros_like(rhs)
    status, its, rr = S.pressure_solve(rhs, p, 1e-13)
    assert status == 0 and rr <= 1e-12
    assert rel(p.cpu().numpy(), o.p) < 1e-10


def test_large_coarsest_level(fvs, monkeypatch):
    """A coarsest AMG level far above the shared-memory size (several hundred rows
    here) is inverted in global memory by the whole GPU; one step still
    matches the oracle."""
    monkeypatch.setenv("FVS_AMG_COARSEST", "1000")
    m = box_mesh(24, 24, 6, cases.CAVITY, jitter=0.2, jitter_seed=71, permute_seed=72)
    T0 = frozen_corner_field(m, seed=7)
    rng = np.random.default_rng(8)
    u0 = rng.normal(scale=2e-3, size=(len(T0), 3))
    o, M, S = make_pair(fvs, m, cases.props(**TIGHT), T0, u0)
    o.step(1e-3)
    st = S.step(1e-3)
    assert st["amg_levels"] >= 2 and st["fallback"] == 0 and st["p_its"] < 200, st
    compare(o, S, 1e-10)


MOLD = dict(rho=7800.0, cp=500.0, k=30.0, h=2000.0, T_init=500.0)


def mold_case():
    """Jittered cavity: a metal column through the middle, mold around it,
    every outer wall (mold surface) held at 500 K."""
    m = box_mesh(12, 12, 4, cases.CAVITY, jitter=0.2, jitter_seed=91, permute_seed=92)
    m = dict(m, cell_zone=zones_inner_box(m, (0.025, 0.025, -1.0), (0.075, 0.075, 1.0)))
    props = cases.props(walls=cases.all_walls(500.0), T_init=950.0, mold=MOLD, **TIGHT)
    return m, props


def test_mold_one_step(fvs):
    """Metal in a mold (conduction-only cells, interface coefficient h): one
    step equals the oracle's, fields within 1e-10."""
    m, props = mold_case()
    o, M, S = make_pair(fvs, m, props)
    assert (~o.metal).sum() > 0 and o.interface.sum() > 0
    o.step(1e-3)
    S.step(1e-3)
    compare(o, S, 1e-10)


def test_mold_forty_steps(fvs):
    """Forty steps of the metal column in its mold: temperature within 1e-8 K
    of the oracle everywhere (metal and mold), velocity within 1e-8 relative,
    no velocity in the mold."""
    m, props = mold_case()
    o, M, S = make_pair(fvs, m, props)
    for _ in range(40):
        o.step(2e-3)
    S.step(2e-3, 40)
    assert np.abs(S.query("T") - o.T).max() <= 1e-8
    U = S.query("U")
    assert rel(U, o.u) <= 1e-8
    assert np.abs(U[~o.metal]).max() == 0.0
    np.testing.assert_allclose(S.query("CROSS"), np.stack([o.t_liq, o.t_sol], 1), atol=1e-9)


def test_two_hundred_steps_cavity(fvs):
    """The 32x32x4 configuration for its 200 steps: temperature within 1e-6 K."""
    c = cases.config_small()
    props = cases.props(**dict(TIGHT, p_rtol=1e-12))
    o, M, S = make_pair(fvs, c["mesh"], props)
    for _ in range(200):
        o.step(1e-3)
    S.step(1e-3, 200)
    assert np.abs(S.query("T") - o.T).max() <= 1e-6
    assert rel(S.query("U"), o.u) <= 1e-6
    np.testing.assert_allclose(S.query("CROSS"), np.stack([o.t_liq, o.t_sol], 1), atol=1e-9)


def test_crossings_and_microstructure(fvs):
    """A small cavity cooled on all walls freezes within the run; per-cell
    solidification times, cooling rates, SDAS and yield strength (Eq. 22-23)
    follow the oracle's."""
    m = box_mesh(8, 8, 2, (0.01, 0.01, 0.0025))
    props = cases.props(walls=cases.all_walls(700.0), T_init=920.0, **TIGHT)
    o, M, S = make_pair(fvs, m, props)
    for _ in range(120):
        o.step(2e-3)
    S.step(2e-3, 120)
    q = S.query("QOI")
    ref = o.qoi()
    done = np.isfinite(ref["t_f"])
    assert done.sum() > 20
    assert np.array_equal(np.isfinite(q[:, 0]), done)
    for k, name in enumerate(("t_f", "cooling_rate", "sdas", "yield_strength")):
        assert rel(q[done, k], ref[name][done]) < 1e-8, name


def test_mixed_precision_matches_fp64(fvs):
    """FP32 AMG V-cycle inside the FP64 Krylov method: at the same 1e-8
    pressure residual the fields stay within 1e-6 (relative) of the FP64 path
    and of the tightly solved oracle."""
    m = box_mesh(24, 24, 6, cases.CAVITY, jitter=0.2, jitter_seed=41, permute_seed=42)
    T0 = frozen_corner_field(m, seed=4)
    rng = np.random.default_rng(6)
    u0 = rng.normal(scale=2e-3, size=(len(T0), 3))
    runs = {}
    for prec in (0, 1):
        props = cases.props(p_rtol=1e-8, mom_rtol=1e-12, e_rtol=1e-13, e_tol_T=1e-10, precision=prec)
        M = fvs.Mesh(m)
        S = fvs.Solver(M, props)
        S.set_state(T0, u0)
        st = [S.step(1e-3) for _ in range(3)]
        assert all(s["p_relres"] <= 1e-8 for s in st)
        assert all(s["amg_levels"] >= 2 for s in st)
        runs[prec] = {k: S.query(k) for k in ("T", "U", "P", "FLUX")}
    o = Oracle(m, cases.props(**TIGHT))
    set_state(o, T0, u0)
    o.run(1e-3, 3)
    ref = dict(T=o.T, U=o.u, P=o.p, FLUX=o.F)
    for k in ("T", "U", "P"):
        assert rel(runs[1][k], runs[0][k]) <= 1e-6, (k, rel(runs[1][k], runs[0][k]))
        assert rel(runs[1][k], ref[k]) <= 1e-6, (k, rel(runs[1][k], ref[k]))


def oracle_uq(m, props, inputs, dt, max_steps):
    """Per-sample oracle runs to full solidification: (qoi means, steps)."""
    out, nsteps = [], []
    for Tm, Tw, C0 in inputs:
        mat = dict(props["material"], T_liq=913.0 - 5.0 * (C0 - 4.0))
        o = Oracle(m, cases.props(material=mat, walls=cases.all_walls(Tw), T_init=Tm, **TIGHT))
        k = 0
        while k < max_steps:
            st = o.step(dt)
            k += 1
            if st["n_active"] == 0:
                break
        q = o.qoi()
        done = np.isfinite(q["t_f"])
        out.append([q[name][done].mean() for name in ("t_f", "cooling_rate", "sdas", "yield_strength")])
        nsteps.append(k)
    return np.array(out), np.array(nsteps)


@pytest.mark.parametrize("mode", [0, 1])
def test_uq_batch_matches_oracle(fvs, mode):
    """fvs_uq_batch: each sample is a plain solve with its own melt and wall
    temperatures and liquidus; per-sample means of t_f, cooling rate, SDAS and
    yield equal the oracle's runs of the same samples to full solidification.
    Mode 0 advances the samples in lockstep (one launch per phase), mode 1
    runs independent solves on streams."""
    m = box_mesh(8, 8, 2, (0.01, 0.01, 0.0025))
    inputs = np.array([[930.0, 700.0, 4.0], [955.0, 680.0, 3.2], [942.0, 735.0, 4.8]])
    props = cases.props(**TIGHT)
    M = fvs.Mesh(m)
    qoi, steps = fvs.uq_batch(M, props, inputs, 2e-3, 400, n_streams=2, mode=mode)
    ref, ref_steps = oracle_uq(m, props, inputs, 2e-3, 400)
    assert np.array_equal(steps, ref_steps)
    np.testing.assert_allclose(qoi, ref, rtol=1e-8)


def test_lockstep_batch_multilevel_matches_oracle(fvs):
    """Lockstep batch on a mesh whose pressure hierarchy has several levels
    (per-sample Galerkin values on the shared aggregation, per-sample
    coarsest inverses) against the oracle, sample by sample, to full
    solidification."""
    m = box_mesh(16, 16, 4, (0.02, 0.02, 0.005))
    inputs = np.array([[930.0, 700.0, 4.0], [948.0, 690.0, 3.4]])
    props = cases.props(**TIGHT)
    M = fvs.Mesh(m)
    qoi, steps = fvs.uq_batch(M, props, inputs, 2e-3, 300, mode=0)
    ref, ref_steps = oracle_uq(m, props, inputs, 2e-3, 300)
    assert np.array_equal(steps, ref_steps)
    np.testing.assert_allclose(qoi, ref, rtol=1e-8)


def test_lockstep_batch_mixed_precision_matches_oracle(fvs):
    """Lockstep batch with the FP32 V-cycle inside the FP64 Krylov method:
    at the same (tight) outer tolerance the per-sample QoIs equal the
    oracle's."""
    m = box_mesh(16, 16, 4, (0.02, 0.02, 0.005))
    inputs = np.array([[930.0, 700.0, 4.0], [948.0, 690.0, 3.4]])
    props = cases.props(**dict(TIGHT, precision=1))
    M = fvs.Mesh(m)
    qoi, steps = fvs.uq_batch(M, props, inputs, 2e-3, 300, mode=0)
    ref, ref_steps = oracle_uq(m, cases.props(**TIGHT), inputs, 2e-3, 300)
    assert np.array_equal(steps, ref_steps)
    np.testing.assert_allclose(qoi, ref, rtol=1e-8)


def test_lockstep_batch_skewed_mesh_matches_oracle(fvs):
    """Jittered (non-orthogonal) hexes: BiCGStab pressure solves, vertex
    cross terms and smeared coefficients in the per-sample pressure rows.
    Forty steps (the outer shell solidified) against the oracle."""
    m = box_mesh(16, 16, 4, (0.02, 0.02, 0.005), jitter=0.15, jitter_seed=81, permute_seed=82)
    inputs = np.array([[930.0, 700.0, 4.0], [948.0, 690.0, 3.4]])
    props = cases.props(**TIGHT)
    M = fvs.Mesh(m)
    qoi, steps = fvs.uq_batch(M, props, inputs, 2e-3, 40, mode=0)
    ref, ref_steps = oracle_uq(m, props, inputs, 2e-3, 40)
    assert np.array_equal(steps, ref_steps) and (steps == 40).all()
    np.testing.assert_allclose(qoi, ref, rtol=1e-8)


def test_lockstep_batch_many_samples_matches_independent_solves(fvs):
    """Forty samples (two tiles of 32, the second one partly padding):
    lockstep and independent solves give the same QoIs and step counts."""
    m = box_mesh(8, 8, 2, (0.01, 0.01, 0.0025))
    inputs = cases.uq_inputs(40, seed=7)
    props = cases.props(**TIGHT)
    M = fvs.Mesh(m)
    q0, s0 = fvs.uq_batch(M, props, inputs, 2e-3, 400, mode=0)
    q1, s1 = fvs.uq_batch(M, props, inputs, 2e-3, 400, n_streams=4, mode=1)
    assert np.array_equal(s0, s1)
    np.testing.assert_allclose(q0, q1, rtol=1e-9)


@pytest.mark.parametrize("precision", [0, 1])
def test_refreshed_hierarchy_while_cells_freeze(fvs, monkeypatch, precision):
    """Cells that freeze keep the system numbering: their rows turn into
    identity rows and the AMG hierarchy is re-formed on its old aggregates
    (p_rebuilt == 2) instead of aggregated anew.  Fifty steps of a cavity
    cooled on every wall, freezing from about step 8, match the oracle."""
    monkeypatch.setenv("FVS_REFRESH_FRACTION", "1.0")
    m = box_mesh(16, 16, 4, (0.02, 0.02, 0.005), jitter=0.2, jitter_seed=61, permute_seed=62)
    props = cases.props(walls=cases.all_walls(700.0), T_init=920.0, **dict(TIGHT, precision=precision))
    o, M, S = make_pair(fvs, m, props)
    kinds = []
    for _ in range(50):
        o.step(2e-3)
        st = S.step(2e-3)
        assert st["p_relres"] <= 1e-12
        kinds.append(st["p_rebuilt"])
    assert kinds.count(2) >= 5, kinds
    assert np.abs(S.query("T") - o.T).max() <= 1e-8
    compare(o, S, 1e-9, fields=("U", "P", "FLUX"))


def remelt_field(m, full_band):
    """Melt at 940 K with a two-cell solid band just below the solidus (it
    re-melts in the first step), either across the whole mesh (two pockets
    that merge when it melts) or across half of it (one pocket)."""
    ijk = m["cell_ijk"]
    nx, ny, _ = m["shape"]
    rng = np.random.default_rng(11)
    T = 940.0 - rng.uniform(0.0, 5.0, len(ijk))
    band = (ijk[:, 0] >= nx // 2) & (ijk[:, 0] <= nx // 2 + 1)
    if not full_band:
        band &= ijk[:, 1] < ny // 2
    T[band] = cases.AL_ALLOY["T_sol"] - 1e-3
    return T, band


@pytest.mark.parametrize("full_band", [False, True])
def test_margin_cells_that_melt(fvs, full_band):
    """The numbering also holds the solid cells across a face from the melt.
    When they melt (here a band just below the solidus, heated from both
    sides) their rows join the aggregates of their neighbours and the
    hierarchy is refreshed, not rebuilt (p_rebuilt == 2), unless they join
    two pockets: then the labels conflict and the step rebuilds
    (p_rebuilt == 1).  Both against the oracle at 1e-10."""
    m = box_mesh(24, 24, 4, cases.CAVITY, jitter=0.2, jitter_seed=71, permute_seed=72)
    T0, band = remelt_field(m, full_band)
    props = cases.props(**TIGHT)
    o, M, S = make_pair(fvs, m, props, T0)
    st = S.step(1e-3)
    o.step(1e-3)
    assert st["p_rebuilt"] == 1 and st["n_components"] == (2 if full_band else 1)
    assert (S.query("T")[band] > cases.AL_ALLOY["T_sol"]).all()
    st = S.step(1e-3)
    o.step(1e-3)
    assert st["p_rebuilt"] == (1 if full_band else 2), st["p_rebuilt"]
    assert st["n_components"] == 1 and st["p_relres"] <= 1e-12
    compare(o, S, 1e-10)
    for _ in range(3):
        st = S.step(1e-3)
        o.step(1e-3)
        assert st["p_relres"] <= 1e-12
    compare(o, S, 1e-10)


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replayed_iterations_on_a_stream(fvs, precision):
    """On a non-default stream the Krylov iterations are captured once and
    replayed as CUDA graphs; results still match the oracle."""
    import torch
    m = box_mesh(20, 20, 4, cases.CAVITY, jitter=0.2, jitter_seed=51, permute_seed=52)
    T0 = frozen_corner_field(m, seed=5)
    rng = np.random.default_rng(7)
    u0 = rng.normal(scale=2e-3, size=(len(T0), 3))
    props = cases.props(**dict(TIGHT, precision=precision))
    st = torch.cuda.Stream()
    M = fvs.Mesh(m, stream=st)
    S = fvs.Solver(M, props, stream=st)
    S.set_state(T0, u0)
    o = Oracle(m, props)
    set_state(o, T0, u0)
    for _ in range(3):
        o.step(1e-3)
        S.step(1e-3)
    torch.cuda.synchronize()
    compare(o, S, 1e-10)


SCHEIL = cases.AL_SI_SCHEIL


def test_scheil_one_step(fvs):
    """Smeared Gulliver-Scheil solid fraction (Eq. 21) on a jittered,
    permuted mesh whose cells span the liquid, Scheil, smear and solid
    pieces: one step equals the oracle's within 1e-10, solid fraction too."""
    m = box_mesh(10, 10, 4, cases.CAVITY, jitter=0.2, jitter_seed=61, permute_seed=62)
    rng = np.random.default_rng(3)
    T0 = 826.0 + 130.0 * m["cell_ijk"][:, 0] / 9.0 + rng.uniform(-6.0, 6.0, len(m["cells"]))
    u0 = rng.normal(scale=1e-3, size=(len(T0), 3))
    props = cases.props(material=SCHEIL, **TIGHT)
    o, M, S = make_pair(fvs, m, props, T0, u0)
    assert ((T0 > 831.0) & (T0 < 835.0)).any()
    o.step(1e-3)
    S.step(1e-3)
    compare(o, S, 1e-10, fields=("T", "U", "P", "FLUX", "USTAR", "FS"))


@pytest.mark.parametrize("precision", [0, 1])
def test_scheil_forty_steps(fvs, precision):
    """Forty steps of the Scheil alloy cooled through its freezing range on
    every wall: temperature within 1e-8 K of the oracle, solid fraction within
    1e-8, velocity within 1e-8 relative, crossing times equal; the FP32
    V-cycle (precision 1) reaches the same solution at the same outer
    tolerance."""
    m = box_mesh(12, 12, 4, cases.CAVITY, jitter=0.2, jitter_seed=63, permute_seed=64)
    rng = np.random.default_rng(5)
    T0 = 836.0 + 110.0 * m["cell_ijk"][:, 0] / 11.0 + rng.uniform(-3.0, 3.0, len(m["cells"]))
    props = cases.props(material=SCHEIL, walls=cases.all_walls(700.0), **dict(TIGHT, precision=precision))
    o, M, S = make_pair(fvs, m, props, T0)
    for _ in range(40):
        o.step(2e-3)
    S.step(2e-3, 40)
    assert np.abs(S.query("T") - o.T).max() <= 1e-8
    assert np.abs(S.query("FS") - o.fs).max() <= 1e-8
    assert rel(S.query("U"), o.u) <= 1e-8
    np.testing.assert_allclose(S.query("CROSS"), np.stack([o.t_liq, o.t_sol], 1), atol=1e-9)
    assert (o.fs > 0.0).any() and ((o.fs > 0.0) & (o.fs < 1.0)).any() and (o.t_sol > 0.0).any()


@pytest.mark.parametrize("mode", [0, 1])
def test_scheil_uq_batch_matches_oracle(fvs, mode):
    """fvs_uq_batch with the Scheil law and a liquidus per sample (the Scheil
    curve moves with it): per-sample QoIs equal the oracle's runs to full
    solidification, lockstep batch and independent solves."""
    m = box_mesh(8, 8, 2, (0.01, 0.01, 0.0025))
    inputs = np.array([[930.0, 700.0, 4.0], [952.0, 690.0, 3.3]])
    props = cases.props(material=SCHEIL, **TIGHT)
    M = fvs.Mesh(m)
    qoi, steps = fvs.uq_batch(M, props, inputs, 2e-3, 400, n_streams=2, mode=mode)
    ref, ref_steps = oracle_uq(m, props, inputs, 2e-3, 400)
    assert np.array_equal(steps, ref_steps)
    np.testing.assert_allclose(qoi, ref, rtol=1e-8)


@pytest.mark.parametrize("material", ["linear", "scheil"])
def test_grain_growth_matches_oracle(fvs, material):
    """Grain growth (Eq. 24-26) while a jittered cavity cools through its
    freezing range from every wall: the grain radius of every cell equals the
    oracle's within 1e-10 relative after twenty steps, cells that never
    turned mushy keep r0, and the mold-free cavity has no zero radius."""
    m = box_mesh(10, 10, 3, cases.CAVITY, jitter=0.2, jitter_seed=71, permute_seed=72)
    mat = cases.AL_ALLOY if material == "linear" else SCHEIL
    grain = dict(kp=0.13, D_s=3e-9, r0=1e-6)
    props = cases.props(material=mat, walls=cases.all_walls(700.0), T_init=915.0, grain=grain, **TIGHT)
    o, M, S = make_pair(fvs, m, props)
    np.testing.assert_allclose(S.query("GRAIN"), o.grain_radius(), rtol=1e-15)
    for _ in range(20):
        o.step(2e-3)
    S.step(2e-3, 20)
    r = S.query("GRAIN")
    assert rel(r, o.grain_radius()) <= 1e-10
    assert (r > 1.001e-6).any() and np.isclose(r, 1e-6, rtol=1e-14, atol=0).any()


def test_heated_slot_against_the_cubic_and_the_oracle(fvs):
    """The buoyant flow between a hot and a cold wall of
    ``tests/test_oracle_convection.py`` (32 cells across, 80 steps of 8 ms
    from rest): every field of the GPU path matches the oracle, and its
    mid-height profile is the closed-form cubic of the fully developed flow
    to the discretisation error the oracle shows (0.72 % of the peak)."""
    from tests.test_oracle_convection import T_C, T_H, T_REF, D, mid_rows, slot_case, slot_exact
    mesh, mat, walls = slot_case(32)
    props = cases.props(material=mat, walls=walls, T_init=T_REF, **dict(TIGHT, p_rtol=1e-12))
    o = Oracle(mesh, props)
    T0 = T_C + (T_H - T_C) * o.g.xc[:, 0] / D
    set_state(o, T0)
    S = fvs.Solver(fvs.Mesh(mesh), props)
    S.set_state(T0)
    for _ in range(80):
        o.step(8e-3)
    S.step(8e-3, 80)
    compare(o, S, 1e-7, fields=("T", "U", "P"))
    v_ex = slot_exact(o.g.xc[:, 0], mat)
    mid = mid_rows(mesh)
    err = np.abs(S.query("U")[mid, 1] - v_ex[mid]).max() / np.abs(v_ex).max()
    assert err < 0.008, err


def test_freezing_out_and_fully_solid(fvs):
    """Degenerate active sets: a small cavity with cold walls freezes out
    within ten steps of 2 ms and is stepped on with no liquid or mushy cell
    (empty momentum and pressure systems, pure conduction); a cavity that
    starts below the solidus has no active cell from its first step.  The
    active counts follow the oracle's step by step, the flow fields are zero
    once nothing is active, and the temperatures match."""
    m = box_mesh(8, 8, 2, (0.01, 0.01, 0.0025))
    props = cases.props(walls=cases.all_walls(500.0), T_init=915.0, **TIGHT)
    o, M, S = make_pair(fvs, m, props)
    counts = []
    for _ in range(16):
        st_o = o.step(2e-3)
        st = S.step(2e-3)
        assert st["n_active"] == st_o["n_active"] == int(o.lm.sum())
        counts.append(st["n_active"])
    assert counts[0] > 0 and counts[-6:] == [0] * 6, counts
    assert rel(S.query("T"), o.T) <= 1e-10
    for name in ("U", "P", "FLUX"):
        assert np.abs(S.query(name)).max() == 0.0, name
    q, ref = S.query("QOI"), o.qoi()
    assert np.isfinite(ref["t_f"]).all() and np.isfinite(q[:, 0]).all()
    assert rel(q[:, 0], ref["t_f"]) < 1e-8

    props = cases.props(walls=cases.all_walls(700.0), T_init=800.0, **TIGHT)
    o, M, S = make_pair(fvs, m, props)
    for _ in range(3):
        o.step(2e-3)
        st = S.step(2e-3)
        assert st["n_active"] == 0 and st["n_ppe"] == 0
    assert rel(S.query("T"), o.T) <= 1e-10
    for name in ("U", "P", "FLUX"):
        assert np.abs(S.query(name)).max() == 0.0, name
