"""Pins of the oracle's convective walls, temperature-dependent conductivity
and natural-convection-off mode.

* A convective wall (film coefficient h, ambient T_inf) in series with a slab
  has the closed-form steady profile T(x) = T_inf + q/h + q x/k with
  q = (T_b - T_inf)/(1/h + L/k); the discrete steady state equals it at the
  cell centres (linear profiles are exact), so a dropped half-cell
  resistance, a wrong film term or a sign slip fails.
* With k linear in T the Kirchhoff potential Phi(T) = int k dT is linear in
  x at steady state, and a face flux with k at the mean of its two
  temperatures is exactly (Phi(T_2) - Phi(T_1))/distance, so the discrete
  steady state equals Phi^-1 of the linear potential at every cell centre.
  Evaluating k at one owner instead of the mean fails (planted and checked).
  The conductivity table is the paper's Sn-Bi one (Section 3).
* The global energy balance with both features, computed from wall fluxes
  written out independently of the oracle's operator.
* Natural convection off (Section 4) equals the full method whenever the
  melt cannot move (no buoyancy, at rest).
"""
import numpy as np

from fvs_inputs import box_mesh, cases, strip_mesh
from oracle.fv import BC_ADIABATIC, BC_CONVECTIVE, BC_DIRICHLET, Oracle

# Section 3, Sn-Bi validation: mean conductivity (W/m K) at four temperatures (K)
SN_BI_K = [(273.2, 61.282), (373.2, 57.42), (573.2, 30.1), (973.2, 37.7)]
HOT = dict(cases.AL_ALLOY, beta=0.0, T_sol=300.0, T_liq=310.0, latent=0.0)   # liquid throughout, no latent heat


def _steady(o, iters=60):
    """Steady state of the conduction operator by Picard iteration on k(T)."""
    T = o.T.copy()
    for _ in range(iters):
        L, l = o.conduction(T)
        T_next = np.linalg.solve(L.toarray(), -l)
        if np.abs(T_next - T).max() < 1e-12:
            return T_next
        T = T_next
    return T


def test_convective_wall_steady_slab():
    n, Lx = 20, 0.04
    m = strip_mesh(n, length=Lx)
    h, T_inf, T_b = 800.0, 400.0, 900.0
    walls = [(BC_CONVECTIVE, T_inf, h), (BC_DIRICHLET, T_b)] + [(BC_ADIABATIC, 0.0)] * 4
    o = Oracle(m, cases.props(material=HOT, walls=walls, T_init=700.0, no_flow=True))
    T = _steady(o)
    k = HOT["k"]
    q = (T_b - T_inf) / (1.0 / h + Lx / k)
    x = o.g.xc[:, 0]
    exact = T_inf + q / h + q * x / k
    assert np.abs(T - exact).max() <= 1e-10 * T_b


def test_kirchhoff_steady_state_with_linear_k():
    n, Lx = 16, 0.02
    m = strip_mesh(n, length=Lx)
    Ta, Tb = 600.0, 950.0                   # inside the table's last linear piece
    walls = [(BC_DIRICHLET, Ta), (BC_DIRICHLET, Tb)] + [(BC_ADIABATIC, 0.0)] * 4
    o = Oracle(m, cases.props(material=HOT, walls=walls, T_init=800.0, no_flow=True, k_table=SN_BI_K))
    T = _steady(o)
    (T1, k1), (T2, k2) = SN_BI_K[2], SN_BI_K[3]
    b = (k2 - k1) / (T2 - T1)
    a = k1 - b * T1
    phi = lambda t: a * t + 0.5 * b * t * t
    x = o.g.xc[:, 0]
    target = phi(Ta) + (phi(Tb) - phi(Ta)) * x / Lx
    exact = (-a + np.sqrt(a * a + 2.0 * b * target)) / b
    assert np.abs(T - exact).max() <= 1e-10 * Tb
    # a constant conductivity would give the straight line, far from this
    assert np.abs(exact - (Ta + (Tb - Ta) * x / Lx)).max() > 1.0


def test_constant_table_is_constant_k():
    m = box_mesh(6, 5, 2, cases.CAVITY, jitter=0.2, jitter_seed=2, permute_seed=3)
    walls = cases.cavity_walls()
    a = Oracle(m, cases.props(walls=walls, T_init=930.0))
    b = Oracle(m, cases.props(walls=walls, T_init=930.0, k_table=[(300.0, 150.0), (1200.0, 150.0)]))
    for _ in range(3):
        a.step(1e-3)
        b.step(1e-3)
    assert np.abs(a.T - b.T).max() <= 1e-12 * 930.0
    assert np.abs(a.u - b.u).max() <= 1e-12 * max(np.abs(a.u).max(), 1e-300)


def test_energy_balance_with_convective_wall_and_k_of_T():
    """Orthogonal box cooling through its freezing range: x = 0 convective,
    x = L fixed, the rest adiabatic, k(T) from a table.  Each step the
    sensible-minus-latent change equals dt/2 (Q^n + Q^{n+1}) with the wall
    heat flows written out from their definitions: a convective face
    A (T_inf - T_c)/(d/k(T_c^n) + 1/h), a fixed face k(mean(T_c^n, T_w))
    A (T_w - T_c)/d, d the centre-to-face distance."""
    nx, ny, nz = 6, 5, 4
    dims = (0.03, 0.025, 0.02)
    m = box_mesh(nx, ny, nz, dims)
    h, T_inf, T_w = 1500.0, 450.0, 600.0
    table = [(500.0, 120.0), (850.0, 150.0), (1000.0, 90.0)]
    walls = [(BC_CONVECTIVE, T_inf, h), (BC_DIRICHLET, T_w)] + [(BC_ADIABATIC, 0.0)] * 4
    mat = cases.AL_ALLOY
    o = Oracle(m, cases.props(walls=walls, T_init=950.0, no_flow=True, k_table=table, oracle_tol_T=1e-12))
    g = o.g
    own = g.owner
    patch = np.asarray(m["patch"])
    A = g.Af
    d = g.d_own
    kf = lambda T: np.interp(T, [t for t, _ in table], [k for _, k in table])
    dt = 2e-3
    for _ in range(15):
        Tn, fsn = o.T.copy(), o.fs.copy()
        o.step(dt)
        T, fs = o.T, o.fs

        def Q(Tc):
            c0 = patch == 0
            c1 = patch == 1
            q0 = A[c0] * (T_inf - Tc[own[c0]]) / (d[c0] / kf(Tn[own[c0]]) + 1.0 / h)
            q1 = kf(0.5 * (Tn[own[c1]] + T_w)) * A[c1] * (T_w - Tc[own[c1]]) / d[c1]
            return q0.sum() + q1.sum()

        dE = (g.V * (mat["rho"] * mat["cp"] * (T - Tn) - mat["rho"] * mat["latent"] * (fs - fsn))).sum()
        gross = (g.V * np.abs(mat["rho"] * mat["cp"] * (T - Tn))).sum()
        assert abs(dE - 0.5 * dt * (Q(Tn) + Q(T))) <= 1e-9 * gross
    assert (o.fs > 0).any()


def test_no_flow_equals_full_method_when_the_melt_cannot_move():
    m = box_mesh(6, 6, 2, cases.CAVITY, jitter=0.2, jitter_seed=5, permute_seed=6)
    mat = dict(cases.AL_ALLOY, beta=0.0)
    props = dict(walls=cases.all_walls(700.0), T_init=930.0, p_rtol=1e-13)
    a = Oracle(m, cases.props(material=mat, **props))
    b = Oracle(m, cases.props(material=mat, no_flow=True, **props))
    for _ in range(5):
        a.step(1e-3)
        b.step(1e-3)
    assert np.abs(a.u).max() < 1e-14 and np.abs(b.u).max() == 0.0 and np.abs(b.F).max() == 0.0
    assert np.abs(a.T - b.T).max() <= 1e-10
    assert np.array_equal(a.lm, b.lm)
