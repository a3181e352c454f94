"""Physics pins of the oracle (Eq. 2-6, Eq. 18-23; Section 2.4.4).  CPU only."""
import json
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from fvs_inputs import box_mesh, cases, casting_mesh, zones_inner_box
from oracle.analytic import neumann_isothermal, stefan_linear
from oracle.fv import Oracle, darcy_coefficient, sdas_um, solid_fraction, yield_strength_mpa
from tests.helpers import mushy_field, set_state

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_darcy_single_cell_closed_form():
    """One closed cube of side h in the mushy zone: no pressure coupling, so
    Eq. 6 reduces to one equation per component,
    (rho V/dt + D V + 6 mu h) u* = rho V/dt u^n - 6 mu h u^n - rho beta (T - T_ref) g V
    (each wall face adds mu A (0 - u)/(h/2) = -2 mu h u; Crank-Nicolson halves it)."""
    h = 0.01
    m = box_mesh(1, 1, 1, (h, h, h))
    mat = cases.AL_ALLOY
    o = Oracle(m, cases.props(walls=[(0, 0.0)] * 6))
    T = 873.0
    u0 = np.array([[0.01, -0.02, 0.005]])
    set_state(o, [T], u=u0)
    dt = 1e-3
    o.step(dt)
    V = h ** 3
    fs = solid_fraction(T, mat["T_sol"], mat["T_liq"])
    assert fs == pytest.approx(0.5)
    D = mat["darcy_C"] * fs ** 2 / ((1 - fs) ** 3 + mat["darcy_eps"])
    buoy = -mat["rho"] * mat["beta"] * (T - mat["T_ref"]) * np.array(mat["g"]) * V
    lhs = mat["rho"] * V / dt + D * V + 6 * mat["mu"] * h
    rhs = mat["rho"] * V / dt * u0[0] - 6 * mat["mu"] * h * u0[0] + buoy
    np.testing.assert_allclose(o.u[0], rhs / lhs, rtol=1e-12)
    assert darcy_coefficient(0.0, 1e8, 1e-3) == 0.0


@pytest.mark.parametrize("T0", [960.0, 905.0, 840.0])
def test_energy_single_cell_closed_form(T0):
    """One cube with one fixed-temperature face: the energy equation of a
    step is a scalar piecewise-linear equation in T,
    rho cp V (T - T0)/dt = k h (T_w - T) + k h (T_w - T0) + rho L V (fs(T) - fs(T0))/dt,
    solved here region by region; the oracle's latent-heat iteration must
    land on that root."""
    h = 0.01
    m = box_mesh(1, 1, 1, (h, h, h))
    mat = cases.AL_ALLOY
    Tw = 700.0
    o = Oracle(m, cases.props(walls=[(1, Tw)] + [(0, 0.0)] * 5))
    set_state(o, [T0])
    dt = 0.05
    o.step(dt)
    rho, cp, k, L = mat["rho"], mat["cp"], mat["k"], mat["latent"]
    Ts, Tl = mat["T_sol"], mat["T_liq"]
    V = h ** 3
    a = rho * cp * V / dt
    fs0 = solid_fraction(T0, Ts, Tl)
    b = rho * L * V / dt
    roots = []
    # solid: fs = 1; liquid: fs = 0; mushy: fs = (Tl - T)/(Tl - Ts)
    for lo, hi, fsa, fsb in ((-np.inf, Ts, 1.0, 0.0), (Tl, np.inf, 0.0, 0.0),
                             (Ts, Tl, Tl / (Tl - Ts), -1.0 / (Tl - Ts))):
        # a (T - T0) = k h (Tw - T) + k h (Tw - T0) + b (fsa + fsb T - fs0)
        T = (a * T0 + k * h * Tw + k * h * (Tw - T0) + b * (fsa - fs0)) / (a + k * h - b * fsb)
        if lo - 1e-9 <= T <= hi + 1e-9:
            roots.append(T)
    assert len(roots) >= 1
    assert o.T[0] == pytest.approx(roots[0], rel=1e-12)
    # the paper reports 5-10 passes of the latent-heat iteration (Section 2.4.4)
    assert o.stats["e_its"] <= 10


def test_stefan_three_region_limit_is_neumann():
    """The linear-fs similarity solution tends to the classical Neumann
    solution as the freezing interval closes (error ~ T_liq - T_sol)."""
    x = np.linspace(0.0, 0.01, 201)
    Tn, Xn = neumann_isothermal(x, 0.2, 700.0, 950.0, 913.0, 150.0, 2700.0, 900.0, 3.9e5)
    errs = []
    for dT in (1.0, 0.1, 0.01):
        T, (X1, X2) = stefan_linear(x, 0.2, 700.0, 950.0, 913.0 - dT, 913.0, 150.0, 2700.0, 900.0, 3.9e5)
        assert X1 < Xn < X2
        errs.append(np.abs(T - Tn).max())
    assert errs[1] < 0.15 * errs[0] and errs[2] < 0.15 * errs[1] and errs[2] < 0.005


def test_stefan_linear_solid_fraction():
    """1-D freezing with a linear solid fraction against the three-region
    similarity solution, started from the exact profile at t = 0.05 s; the
    error over the run shrinks under refinement of dx and dt (the enthalpy
    kink at the solidus front limits the rate to about first order)."""
    mat = dict(cases.AL_ALLOY, g=(0.0, 0.0, 0.0))
    ex = lambda x, t: stefan_linear(x, t, 700.0, 950.0, mat["T_sol"], mat["T_liq"],
                                    mat["k"], mat["rho"], mat["cp"], mat["latent"])[0]
    worst = []
    for n, dt in ((60, 1e-3), (120, 5e-4), (240, 2.5e-4)):
        m = box_mesh(n, 1, 1, (0.03, 1e-3, 1e-3))
        o = Oracle(m, cases.props(material=mat, walls=cases.cavity_walls(700.0, 950.0)))
        x = o.g.xc[:, 0]
        set_state(o, ex(x, 0.05))
        e = 0.0
        for i in range(int(round(0.1 / dt))):
            o.step(dt)
            e = max(e, np.abs(o.T - ex(x, 0.05 + (i + 1) * dt)).max())
        worst.append(e)
    assert worst[0] > worst[1] > worst[2]
    assert worst[2] < 0.8 and worst[0] / worst[2] > 5.0, worst


@pytest.mark.parametrize("with_mold,scheil", [(False, False), (True, False), (False, True), ("casting", False)])
def test_global_energy_balance(with_mold, scheil):
    """Summed over the cavity, the energy change of a step (sensible minus
    latent) equals dt times the mean of the wall heat flow at both time
    levels: convective and interior diffusive fluxes telescope, including the
    series flux through a metal-mold interface; the latent part follows the
    solid-fraction law in use (linear or Eq. 21)."""
    m = box_mesh(8, 8, 3, cases.CAVITY, jitter=0.15, jitter_seed=2)
    extra = {}
    if with_mold == "casting":
        # voxelised plate with ribs and riser in its steel shell
        m = casting_mesh(0.005)
        extra = dict(mold=dict(cases.STEEL_MOLD))
    elif with_mold:
        m = dict(m, cell_zone=zones_inner_box(m, (0.02, 0.02, -1.0), (0.08, 0.08, 1.0)))
        extra = dict(mold=dict(rho=7800.0, cp=500.0, k=30.0, h=2000.0, T_init=600.0))
    if scheil:
        extra["material"] = cases.AL_SI_SCHEIL
    o = Oracle(m, cases.props(oracle_tol_T=1e-12, **extra))
    rng = np.random.default_rng(4)
    set_state(o, mushy_field(m), u=rng.normal(scale=1e-3, size=(len(m["cells"]), 3)))
    if with_mold:
        assert o.interface.sum() > 0 and (~o.metal).sum() > 0
    for _ in range(3):
        T0, fs0 = o.T.copy(), o.fs.copy()
        q0 = (o.LTk @ T0 + o.lTk).sum()
        o.step(1e-3)
        q1 = (o.LTk @ o.T + o.lTk).sum()
        dE = (o.g.V * (o.rcp * (o.T - T0) - o.rL * (o.fs - fs0))).sum()
        assert abs(dE - 1e-3 * 0.5 * (q0 + q1)) <= 1e-9 * abs(dE)


def test_mirror_symmetry():
    """Gravity along -y and identical z walls: the solution on the mesh
    reflected in z is the reflection of the solution (w changes sign)."""
    kw = dict(jitter=0.2, jitter_seed=9)
    a = box_mesh(6, 6, 4, cases.CAVITY, **kw)
    b = box_mesh(6, 6, 4, cases.CAVITY, mirror_z=True, **kw)
    T0 = mushy_field(a, seed=3)
    runs = []
    for m in (a, b):
        o = Oracle(m, cases.props(oracle_tol_T=1e-12))
        set_state(o, T0)
        o.run(1e-3, 4)
        runs.append(o)
    oa, ob = runs
    assert np.abs(oa.u).max() > 0
    np.testing.assert_allclose(ob.T, oa.T, rtol=1e-12)
    np.testing.assert_allclose(ob.u[:, :2], oa.u[:, :2], atol=1e-10 * np.abs(oa.u).max())
    np.testing.assert_allclose(ob.u[:, 2], -oa.u[:, 2], atol=1e-10 * np.abs(oa.u).max())
    np.testing.assert_allclose(ob.p, oa.p, atol=1e-10 * np.abs(oa.p).max())


def test_microstructure_worked_example():
    with open(os.path.join(GOLDEN, "qoi_worked_example.json")) as fh:
        g = json.load(fh)
    lam = sdas_um(g["cooling_rate_K_per_s"])
    assert lam == pytest.approx(g["sdas_um"], rel=1e-12)
    assert yield_strength_mpa(lam) == pytest.approx(g["yield_MPa"], abs=1e-6)
    # tenfold cooling rate scales SDAS by 10^-0.317
    assert sdas_um(10.0) / sdas_um(1.0) == pytest.approx(10 ** -0.317, rel=1e-14)


def test_crossing_times_linear_in_time():
    """A cell passing the liquidus within a step is stamped at the linear
    interpolation point; the local solidification time and cooling rate follow."""
    m = box_mesh(1, 1, 1, (0.01, 0.01, 0.01))
    o = Oracle(m, cases.props())
    set_state(o, [950.0])
    o.time = 1.0
    o.update_crossings(np.array([920.0]), np.array([900.0]), 0.1)   # passes 913
    assert o.t_liq[0] == pytest.approx(1.0 + 0.1 * 7.0 / 20.0, rel=1e-14)
    assert o.t_sol[0] < 0
    o.time = 2.0
    o.update_crossings(np.array([840.0]), np.array([830.0]), 0.1)   # passes 833
    assert o.t_sol[0] == pytest.approx(2.07, rel=1e-14)
    q = o.qoi()
    tf = 2.07 - 1.035
    assert q["t_f"][0] == pytest.approx(tf, rel=1e-12)
    assert q["cooling_rate"][0] == pytest.approx(80.0 / tf, rel=1e-12)


@pytest.mark.parametrize("h", [500.0, 2000.0, 1e12])
def test_metal_mold_interface_steady_conduction(h):
    """Steady conduction through a metal slab and a mold slab held at two
    temperatures: the conductive operator's steady solution is the
    series-resistance profile q = (T1 - T2) / (a/k_metal + 1/h + a/k_mold),
    linear in each slab with a jump of q/h at the interface, exact at the
    cell centres (two-point fluxes are exact for linear profiles)."""
    nx, Lx = 20, 0.04
    m = box_mesh(nx, 1, 1, (Lx, 2e-3, 2e-3))
    m = dict(m, cell_zone=zones_inner_box(m, (-1.0, -1.0, -1.0), (0.5 * Lx, 1.0, 1.0)))
    mat = dict(cases.AL_ALLOY)
    mold = dict(rho=7800.0, cp=500.0, k=30.0, h=h, T_init=500.0)
    T1, T2 = 600.0, 400.0
    o = Oracle(m, cases.props(material=mat, walls=cases.cavity_walls(T1, T2), mold=mold))
    assert o.interface.sum() == 1
    T = spla.spsolve(o.LTk.tocsc(), -o.lTk)
    x = o.g.xc[:, 0]
    a = 0.5 * Lx
    q = (T1 - T2) / (a / mat["k"] + 1.0 / h + a / mold["k"])
    exact = np.where(x < a, T1 - q * x / mat["k"], T2 + q * (Lx - x) / mold["k"])
    assert np.abs(T - exact).max() <= 1e-9 * (T1 - T2)
