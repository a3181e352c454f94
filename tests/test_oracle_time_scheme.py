"""Pins of the oracle's time levels and of its velocity correction.

* Adams-Bashforth convection (Eq. 6, and the same scheme in the energy
  equation): with a face flux that doubled between the two time levels and a
  field linear in x, the convective term of an interior cell is known in
  closed form, so one step gives T^{n+1} and u* by hand.  Weights 1/0 or 2/-1
  instead of 3/2 and -1/2, or the flux levels swapped, fail these tests
  (planted and checked).
* Hydrostatics (Eq. 2, Eq. 8, Section 2.4.3): an inviscid melt at a uniform
  temperature other than T_ref is pushed by a uniform buoyancy force; the
  projection must turn it into a pressure rising linearly against gravity
  and leave no flux and, in every cell whose face gradients see only
  interior vertices, no velocity.  A wrong factor dt/rho or a wrong sign in
  the cell-centre correction leaves a velocity behind (planted and checked).
"""
import numpy as np

from fvs_inputs import box_mesh, cases
from fvs_inputs.cases import BC_ADIABATIC
from oracle.fv import Oracle

ADIABATIC = [(BC_ADIABATIC, 0.0)] * 6


def _oracle(mesh, **mat):
    m = dict(cases.AL_ALLOY)
    m.update(mat)
    p = cases.props(material=m, walls=ADIABATIC, T_init=1000.0, p_rtol=1e-13)
    return Oracle(mesh, p)


def _x_flux(o, U):
    """Volume flux of a uniform velocity U along x through every interior face
    (walls carry no flux)."""
    g = o.g
    return np.where(g.interior, U * g.Sf[:, 0], 0.0)


def _interior_x(mesh, o):
    i = mesh["cell_ijk"][:, 0]
    return (i >= 1) & (i <= mesh["shape"][0] - 2)


def test_energy_convection_adams_bashforth():
    """T^n = T^{n-1} - 7 = 1000 + a x, F^n = U A n_x, F^{n-1} = F^n / 2:
    interior cells see Conv(T^n, F^n) = a U V and Conv(T^{n-1}, F^{n-1}) =
    a U V / 2, so (no conduction, all liquid) T^{n+1} = T^n - dt a U (3/2 - 1/4)."""
    mesh = box_mesh(8, 3, 2, (0.08, 0.03, 0.02))
    o = _oracle(mesh, k=1e-12, beta=0.0)
    a, U, dt = 1000.0, 1e-2, 1e-2
    x = o.g.xc[:, 0]
    o.T = 1000.0 + a * x
    o.T_old = o.T - 7.0
    o.fs = o.fs_of(o.T)
    o.F = _x_flux(o, U)
    o.F_old = 0.5 * o.F
    T_n = o.T.copy()
    o.step(dt)
    sel = _interior_x(mesh, o)
    expect = T_n - dt * a * U * (1.5 - 0.25)
    assert np.abs(o.T[sel] - expect[sel]).max() < 1e-9
    # the same step with weights 1/0 would land 0.25 dt a U = 0.025 K away
    assert 0.25 * dt * a * U > 1e6 * 1e-9


def test_momentum_convection_adams_bashforth():
    """u_x^n = u_x^{n-1} = a x, F^n = U A n_x, F^{n-1} = F^n / 2, no viscosity,
    no buoyancy, no drag: interior u*_x = u^n_x - dt a U (3/2 - 1/4)."""
    mesh = box_mesh(8, 3, 2, (0.08, 0.03, 0.02))
    o = _oracle(mesh, mu=0.0, beta=0.0)
    a, U, dt = 0.5, 1e-2, 1e-2
    x = o.g.xc[:, 0]
    o.u = np.zeros((o.g.Nc, 3))
    o.u[:, 0] = a * x
    o.u_old = o.u.copy()
    o.F = _x_flux(o, U)
    o.F_old = 0.5 * o.F
    u_n = o.u.copy()
    o.step(dt)
    sel = _interior_x(mesh, o)
    expect = u_n[:, 0] - dt * a * U * (1.5 - 0.25)
    assert np.abs(o.u_star[sel, 0] - expect[sel]).max() < 1e-13
    assert np.abs(o.u_star[:, 1:]).max() < 1e-15


def _hydrostatic(mesh, dT=37.0):
    o = _oracle(mesh, mu=0.0)
    o.T[:] = o.m["T_ref"] + dT
    o.T_old = o.T.copy()
    o.fs = o.fs_of(o.T)
    o.step(1e-3)
    return o


def test_hydrostatic_balance_regular_mesh():
    """Uniform T = T_ref + 37 K, inviscid: the buoyancy force per volume is
    f = -rho beta (T - T_ref) g, u* = dt f / rho everywhere, and the
    projection gives p = f . x + c and F^{n+1} = 0 (face normal gradients
    are exact for linear p on an orthogonal mesh).  The cell-centre
    correction averages whole face gradients, whose tangential parts come
    from vertex values; a vertex value is the mean of the cells around it,
    which is exact for linear p at interior vertices only.  So u^{n+1} = 0
    exactly in the cells none of whose faces has a wall vertex, and near the
    walls only the tangential part of the gradient is off (by up to half)."""
    mesh = box_mesh(6, 7, 5, (0.06, 0.07, 0.05))
    o = _hydrostatic(mesh)
    m = o.m
    f = -m["rho"] * m["beta"] * 37.0 * np.asarray(m["g"])
    ustar = 1e-3 * f / m["rho"]
    np.testing.assert_allclose(o.u_star, np.broadcast_to(ustar, o.u_star.shape), rtol=1e-12)
    y = o.g.xc[:, 1]
    p_lin = f[1] * (y - y.mean())
    assert np.abs(o.p - o.p.mean() - p_lin).max() <= 1e-9 * np.abs(p_lin).max()
    umax = np.abs(ustar).max()
    ijk, shape = mesh["cell_ijk"], np.array(mesh["shape"])
    inner = np.all((ijk >= 1) & (ijk <= shape - 2), axis=1)
    assert inner.sum() == 4 * 5 * 3
    assert np.abs(o.u[inner]).max() <= 1e-9 * umax
    # near the walls the normal part of every face gradient is still exact:
    # the velocity left there is tangential to the wall it touches
    assert np.abs(o.u).max() <= 0.5 * umax
    assert np.abs(o.F).max() <= 1e-9 * umax * o.g.Af.max()


def test_hydrostatic_balance_converges_on_distorted_meshes():
    """On a smoothly distorted (non-orthogonal) mesh the cell means that give
    the vertex values (Section 2.3) miss a linear field by O(h^2) even at
    interior vertices, so the velocity left after the projection is not zero;
    away from the walls it must shrink under refinement (measured: 1.3 %,
    0.47 %, 0.17 % of u* in the RMS at n = 6, 12, 24), and the flux still
    balances in every cell (Eq. 17)."""
    errs = []
    for n in (6, 12):
        mesh = box_mesh(n, n, n // 2, (0.06, 0.06, 0.03), distort=0.04)
        o = _hydrostatic(mesh)
        umax = np.abs(o.u_star).max()
        ijk, shape = mesh["cell_ijk"], np.array(mesh["shape"])
        inner = np.all((ijk >= 1) & (ijk <= shape - 2), axis=1)
        errs.append(np.sqrt((o.u[inner] ** 2).mean()) / umax)
        div = o.g.Div @ o.F
        assert np.abs(div).max() <= 1e-10 * umax * o.g.Af.max()
    assert errs[0] < 0.02 and errs[1] < errs[0] / 2.4, errs
