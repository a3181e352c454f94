"""Pin of the coupled flow path: buoyant flow between a hot and a cold wall.

A tall slot, width d along x, height 6 d along y (gravity along -y), the
x = 0 wall held at T_c and the x = d wall at T_h, the other walls adiabatic,
all walls no-slip, one cell across a very wide z extent (W = 1000 d).  With
the Boussinesq force of Eq. 2 taken about T_ref = (T_c + T_h) / 2 and a melt
slow enough that convection cannot bend the isotherms (Peclet and Reynolds
numbers ~1e-4), conduction keeps T linear in x, and far from the top and
bottom the flow is parallel and vertical.  There the y-momentum balance
reduces to

    mu v''(x) = -rho beta g (T(x) - T_ref) + dp/dy,

and the zero net flux through any horizontal section (the slot is closed)
makes dp/dy = 0, because the force is odd about the mid-plane.  With
xi = x - d/2 and G = rho beta g (T_h - T_c) / (mu d), integrating twice with
v(+-d/2) = 0 gives the cubic

    v(xi) = G / 6 (xi d^2 / 4 - xi^3),

rising on the hot side.  The oracle steps the full method (AB2/CN predictor
of Eq. 6, pressure equation, flux and cell corrections of Eq. 8 and Eq. 17)
from rest to a steady state; the mid-height profile must approach the cubic
at second order in the cell width (the wall faces take a one-sided gradient
over half a cell, exact for straight profiles only, so the error is O(h^2)
rather than zero).  The z walls, one cell across W, add a drag of
4 mu v / W^2 per volume, a relative change of about 4 (d / W)^2 / 10 = 4e-7,
far below the discretisation error.

Planted and checked: the buoyancy sign flipped, the implicit half of the
Crank-Nicolson viscous term dropped, and the wall faces of the velocity
diffusion taken over a whole cell instead of half a cell each fail this test.
"""
import numpy as np

from fvs_inputs import box_mesh, cases
from fvs_inputs.cases import BC_ADIABATIC, BC_DIRICHLET
from oracle.fv import Oracle

D = 0.01
T_C, T_H, T_REF = 990.0, 1010.0, 1000.0
MU, BETA = 1.0, 1e-6


def slot_case(nx):
    """Mesh, material and walls of the heated slot with nx cells across."""
    mesh = box_mesh(nx, 3 * nx, 1, (D, 6 * D, 1000 * D))
    mat = dict(cases.AL_ALLOY, T_ref=T_REF, mu=MU, beta=BETA)
    walls = [(BC_DIRICHLET, T_C), (BC_DIRICHLET, T_H)] + [(BC_ADIABATIC, 0.0)] * 4
    return mesh, mat, walls


def slot_exact(x, mat):
    """The cubic profile of the fully developed slot flow."""
    G = mat["rho"] * mat["beta"] * abs(mat["g"][1]) * (T_H - T_C) / (mat["mu"] * D)
    xi = x - D / 2
    return G / 6.0 * (xi * D * D / 4.0 - xi ** 3)


def mid_rows(mesh):
    j = mesh["cell_ijk"][:, 1]
    ny = mesh["shape"][1]
    return (j == ny // 2 - 1) | (j == ny // 2)


def _run(nx, steps=80, dt=8e-3):
    mesh, mat, walls = slot_case(nx)
    o = Oracle(mesh, cases.props(material=mat, walls=walls, T_init=T_REF, p_rtol=1e-13, oracle_tol_T=1e-12))
    x = o.g.xc[:, 0]
    o.T[:] = T_C + (T_H - T_C) * x / D
    o.T_old = o.T.copy()
    o.fs = o.fs_of(o.T)
    for _ in range(steps):
        o.step(dt)
    return o, mesh, mat


def test_heated_slot_converges_to_the_cubic_profile():
    errs = []
    for nx in (8, 16, 32):
        o, mesh, mat = _run(nx)
        x = o.g.xc[:, 0]
        v_ex = slot_exact(x, mat)
        vmax = np.abs(v_ex).max()
        mid = mid_rows(mesh)
        errs.append(np.abs(o.u[mid, 1] - v_ex[mid]).max() / vmax)
    # measured: 0.108, 0.0285, 0.0072
    assert errs[0] < 0.12 and errs[2] < 0.008, errs
    for a, b in zip(errs, errs[1:]):
        assert 3.5 < a / b < 4.5, errs

    # the finest run: the hot side rises, the profile is odd about the
    # mid-plane, the flow is vertical and the isotherms stay straight
    v = o.u[mid, 1]
    xm = x[mid]
    assert (v[xm > D / 2] > 0).all() and (v[xm < D / 2] < 0).all()
    order = np.argsort(xm)
    vs = v[order].reshape(-1, 2).mean(axis=1)       # the two mid rows, by x
    assert np.abs(vs + vs[::-1]).max() <= 1e-6 * vmax
    assert np.abs(o.u[mid, 0]).max() <= 1e-4 * vmax
    assert np.abs(o.u[mid, 2]).max() <= 1e-9 * vmax
    assert np.abs(o.T - (T_C + (T_H - T_C) * x / D)).max() <= 1e-5 * (T_H - T_C)
