"""Pins of the oracle's geometry and face gradients (Section 2.3, Eq. 11-12).

CPU only.  Each check compares with something the mathematics fixes: closed
surfaces, exact volumes, closed-form values on regular meshes, exactness of
the local-frame gradient for linear fields, and convergence on distorted
meshes.
"""
import numpy as np
import pytest

from fvs_inputs import box_mesh, cases
from oracle.analytic import conduction_series
from oracle.fv import Geometry, Oracle, solid_fraction, temperature_diffusion

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def geom(m):
    return Geometry(m["nodes"], m["cells"], m["faces"], m["face_cells"], m["patch"])


@pytest.fixture(scope="module")
def jittered():
    return geom(box_mesh(6, 5, 4, (0.3, 0.25, 0.2), jitter=0.25, jitter_seed=3, permute_seed=11))


def test_closed_surfaces(jittered):
    """The outward face vectors of every cell sum to zero (closed surface)."""
    g = jittered
    s = g.Div @ g.Sf
    scale = np.abs(g.Div) @ g.Af
    assert np.all(np.abs(s).max(axis=1) <= 1e-14 * scale)


def test_total_volume(jittered):
    """Interior faces cancel in 1/3 sum x_f . S_f, the walls stay planar, so
    the volumes add up to the box exactly and are all positive."""
    g = jittered
    assert np.all(g.V > 0)
    assert abs(g.V.sum() - 0.3 * 0.25 * 0.2) <= 1e-14 * 0.015


def test_regular_closed_forms():
    hx, hy, hz = 0.1 / 8, 0.1 / 6, 0.0125 / 4
    g = geom(box_mesh(8, 6, 4, (0.1, 0.1, 0.0125)))
    np.testing.assert_allclose(g.V, hx * hy * hz, rtol=1e-13)
    h = np.abs(g.n) @ np.array([hx, hy, hz])
    np.testing.assert_allclose(g.ndotd, np.where(g.interior, h, h / 2), rtol=1e-13)
    A = np.abs(g.n) @ np.array([hy * hz, hx * hz, hx * hy])
    np.testing.assert_allclose(g.Af, A, rtol=1e-13)
    # orthogonal hexahedra: no cross diffusion
    assert np.abs(g.w).max() < 1e-9 * np.abs(1 / g.ndotd).min()


def test_face_gradient_exact_for_linear_fields(jittered):
    """Eq. 12: with exact vertex and centre values the local-frame gradient
    reproduces the gradient of a linear field, and the split of Eq. 11
    reproduces its normal component."""
    g = jittered
    rng = np.random.default_rng(0)
    a, grad = rng.normal(), rng.normal(size=3)
    phi = lambda x: a + x @ grad
    c2 = np.where(g.interior[:, None], g.xc[np.maximum(g.neigh, 0)], g.xf)
    delta = np.stack([phi(c2) - phi(g.xc[g.owner]),
                      phi(g.nodes[g.faces[:, 2]]) - phi(g.nodes[g.faces[:, 0]]),
                      phi(g.nodes[g.faces[:, 3]]) - phi(g.nodes[g.faces[:, 1]])], axis=1)
    gf = np.einsum("fij,fj->fi", g.Jinv, delta)
    np.testing.assert_allclose(gf, np.broadcast_to(grad, gf.shape), rtol=1e-9, atol=1e-9)
    nd = (1 / g.ndotd + g.w[:, 0]) * delta[:, 0] + g.w[:, 1] * delta[:, 1] + g.w[:, 2] * delta[:, 2]
    np.testing.assert_allclose(nd, g.n @ grad, rtol=1e-9, atol=1e-9)


def test_laplacian_of_quadratic_on_regular_mesh():
    """On an orthogonal mesh the face-sum operator is the 7-point Laplacian,
    exact for quadratics away from the walls: (L phi)/V = 6 for |x|^2."""
    m = box_mesh(7, 6, 5, (0.7, 0.6, 0.5))
    o = Oracle(m, cases.props())
    g = o.g
    phi = (g.xc ** 2).sum(axis=1)
    lap = (o.Lu @ phi) / g.V
    ijk = m["cell_ijk"]
    inner = np.all((ijk > 0) & (ijk < np.array([6, 5, 4])), axis=1)
    np.testing.assert_allclose(lap[inner], 6.0, rtol=1e-10)


def test_temperature_walls_on_regular_mesh():
    """A linear profile between two fixed-temperature walls is a steady state
    of the temperature operator with adiabatic side walls."""
    m = box_mesh(9, 4, 3, (0.09, 0.04, 0.03))
    g = geom(m)
    walls = cases.cavity_walls(700.0, 950.0)
    L, l = temperature_diffusion(g, walls)
    T = 700.0 + 250.0 * g.xc[:, 0] / 0.09
    r = L @ T + l
    assert np.abs(r).max() <= 1e-9 * np.abs(l).max()


@pytest.mark.parametrize("distort", [0.0, 0.05])
def test_conduction_converges_on_distorted_slab(distort):
    """Pure conduction (no latent heat) in a slab with fixed end temperatures,
    against the Fourier series, on orthogonal and on smoothly distorted
    meshes.  On the distorted mesh the cross-diffusion terms of Eq. 11 carry
    weight: flipping their sign, swapping the eta/zeta weights or dropping
    them leaves errors of several kelvin that grow under refinement, while
    the correct operator converges.  (On randomly jittered meshes the
    vertex averaging of Section 2.3 has an O(1) consistency error, so the
    convergence check uses a smooth mapping.)"""
    mat = dict(cases.AL_ALLOY, g=(0.0, 0.0, 0.0), latent=0.0)
    alpha = mat["k"] / (mat["rho"] * mat["cp"])
    ell = 0.01
    errs = []
    for n, dt in ((6, 4e-3), (12, 2e-3), (24, 1e-3)):
        m = box_mesh(n, n // 3, n // 3, (ell, ell / 3, ell / 3), distort=distort)
        o = Oracle(m, cases.props(material=mat, walls=cases.cavity_walls(700.0, 950.0)))
        x = o.g.xc[:, 0]
        o.T = conduction_series(x, 0.1, ell, 700.0, 950.0, 950.0, alpha)
        o.fs = solid_fraction(o.T, mat["T_sol"], mat["T_liq"])
        o.T_old = o.T.copy()
        o.run(dt, int(round(0.048 / dt)))
        err = o.T - conduction_series(x, 0.148, ell, 700.0, 950.0, 950.0, alpha)
        errs.append(np.sqrt(np.mean(err ** 2)))
    if distort == 0.0:
        order = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
        assert min(order) > 1.9, (errs, order)
    else:
        assert errs[2] < 0.25 and errs[1] / errs[2] > 1.6 and errs[0] > errs[1], errs


def test_voxel_casting_mesh():
    """The voxelised casting in its mold shell: closed cell surfaces, every
    cell a cube of the voxel size, walls facing outward, metal volume equal
    to the voxel count of plate, ribs and riser, and the metal enclosed by
    the shell (no wall face on a metal cell)."""
    from fvs_inputs import casting_mesh
    h = 0.005
    m = casting_mesh(h)
    g = geom(m)
    s = g.Div @ g.Sf
    assert np.all(np.abs(s).max(axis=1) <= 1e-14 * (np.abs(g.Div) @ g.Af))
    np.testing.assert_allclose(g.V, h ** 3, rtol=1e-12)
    assert np.abs(g.w).max() < 1e-9 * np.abs(1 / g.ndotd).min()
    zone = m["cell_zone"]
    # plate 40 x 20 x 4 voxels, three ribs 1 x 20 x 2, riser 4 x 4 x 4
    assert (zone == 0).sum() == 40 * 20 * 4 + 3 * 1 * 20 * 2 + 4 * 4 * 4
    wall = ~g.interior
    assert np.all(zone[g.owner[wall]] == 1)
    # outward normals on the walls: they point away from the owner's centre
    X = np.asarray(m["nodes"])
    xc = X[np.asarray(m["cells"])].mean(axis=1)
    fc = X[np.asarray(m["faces"])].mean(axis=1)
    out = np.einsum("fi,fi->f", g.n[wall], fc[wall] - xc[g.owner[wall]])
    assert np.all(out > 0)
