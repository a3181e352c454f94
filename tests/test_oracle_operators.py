"""Pins of the oracle's pressure system and convection operator
(Section 2.4.2, Eq. 9, Eq. 15-17; Section 2.3 convection).  CPU only."""
import numpy as np
import pytest
import scipy.sparse as sp

from fvs_inputs import box_mesh, cases
from oracle.fv import Oracle, solve_singular
from tests.helpers import frozen_corner_field, set_state, small_jittered_mesh

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def ppe_after_one_step(mesh, T0, seed=0):
    o = Oracle(mesh, cases.props())
    rng = np.random.default_rng(seed)
    set_state(o, T0, u=rng.normal(scale=1e-3, size=(len(T0), 3)))
    o.step(1e-3)
    return o


@pytest.fixture(scope="module")
def frozen_jittered():
    m = small_jittered_mesh()
    return m, ppe_after_one_step(m, frozen_corner_field(m))


def assemble(o):
    g = o.g
    De, Dz = o.smeared_rows(o.case, o.ppe)
    N = g.normal_derivative_rows(g.Dxi, De, Dz)
    flow = (o.case == 1) | (o.case == 2)
    A = (g.Div @ sp.diags(flow.astype(float)) @ N).tocsr() / o.m["rho"]
    pa = np.nonzero(o.ppe)[0]
    return A[pa][:, pa].toarray(), De, Dz, pa


def test_all_face_cases_present(frozen_jittered):
    _, o = frozen_jittered
    assert {0, 1, 2, 3} <= set(np.unique(o.case).tolist())


def test_pressure_rows_and_columns_sum_to_zero(frozen_jittered):
    """Rows: a constant pressure has no gradient, and the smearing of Eq. 16
    keeps that (its divisor is the number of remaining cells).  Columns: each
    face adds equal and opposite flux to its two owners."""
    _, o = frozen_jittered
    A, _, _, _ = assemble(o)
    scale = np.abs(A).max()
    assert np.abs(A.sum(axis=1)).max() <= 1e-12 * scale
    assert np.abs(A.sum(axis=0)).max() <= 1e-12 * scale


def test_pressure_symmetric_on_orthogonal_mesh():
    m = box_mesh(6, 5, 3, cases.CAVITY)
    o = ppe_after_one_step(m, np.full(90, 950.0))
    A, _, _, _ = assemble(o)
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-12 * np.abs(A).max())


def test_smearing_equals_mean_substitution(frozen_jittered):
    """Eq. 15-16 characterised: the smeared gradient of a case-2 face is the
    original gradient evaluated with every deleted neighbour's value replaced
    by the mean of the remaining neighbours' values."""
    _, o = frozen_jittered
    g = o.g
    rng = np.random.default_rng(1)
    p = rng.normal(size=g.Nc)
    p[~o.ppe] = 0.0
    De, Dz = o.smeared_rows(o.case, o.ppe)
    NB = g.NB
    faces = np.nonzero(o.case == 2)[0]
    assert len(faces) > 10
    for f in faces:
        nbr = NB.indices[NB.indptr[f]:NB.indptr[f + 1]]
        keep = nbr[o.ppe[nbr]]
        q = p.copy()
        q[nbr[~o.ppe[nbr]]] = p[keep].mean()
        for D0, D in ((o.Deta_p, De), (o.Dzeta_p, Dz)):
            assert abs(D0[f] @ q - D[f] @ p) <= 1e-12 * (1 + np.abs(p).max())


def test_pressure_solve_matches_dense_pseudo_inverse(frozen_jittered):
    """Brute force on <= 512 cells: the pinned, projected sparse solve equals
    the minimum-norm least-squares solution of the projected system, shifted
    to zero mean on each connected part."""
    _, o = frozen_jittered
    A, _, _, pa = assemble(o)
    b = o.b_ppe[pa]
    p, ncomp = solve_singular(sp.csr_matrix(A), b)
    assert ncomp >= 1
    # for a single connected part the null space is the constants, so the
    # pseudo-inverse solution of the projected right side has zero mean
    from oracle.fv import pressure_components
    nc, lab = pressure_components(sp.csr_matrix(A))
    bp = b.copy()
    for c in range(nc):
        bp[lab == c] -= bp[lab == c].mean()
    q = np.linalg.lstsq(A, bp, rcond=1e-13)[0]
    for c in range(nc):
        q[lab == c] -= q[lab == c].mean()
    np.testing.assert_allclose(p, q, rtol=0, atol=1e-10 * np.abs(q).max())
    np.testing.assert_allclose(o.p[pa], p, rtol=0, atol=1e-10 * np.abs(q).max())


def test_convection_telescopes_and_is_exact_for_uniform_flow():
    """Sum over cells of the convective flux is zero (walls carry none); a
    constant is not convected by a divergence-free flux; on an orthogonal
    mesh a uniform flow through phi = x gives u_x V in inner cells."""
    m = box_mesh(6, 5, 4, (0.6, 0.5, 0.4))
    o = Oracle(m, cases.props())
    g = o.g
    rng = np.random.default_rng(2)
    F = np.where(g.interior, rng.normal(size=g.Nf), 0.0)
    phi = rng.normal(size=g.Nc)
    assert abs(o.conv(phi, F).sum()) <= 1e-12 * np.abs(F).sum()
    U = np.array([0.3, -0.2, 0.1])
    Fu = np.where(g.interior, g.Sf @ U, 0.0)
    ijk = m["cell_ijk"]
    inner = np.all((ijk > 0) & (ijk < np.array([5, 4, 3])), axis=1)
    assert np.abs(o.conv(np.ones(g.Nc), Fu)[inner]).max() <= 1e-14
    cx = o.conv(g.xc[:, 0], Fu)
    np.testing.assert_allclose(cx[inner], U[0] * g.V[inner], rtol=1e-12)


def test_mass_conservation_after_steps(frozen_jittered):
    """Discrete continuity: with the face flux built from the same modified
    coefficients as the pressure system (Eq. 17), every cell's net volume
    flux vanishes to the solver tolerance (<= 1e-10 of its face fluxes)."""
    m, o = frozen_jittered
    o.step(1e-3)
    g = o.g
    net = g.Div @ o.F
    tot = np.abs(g.Div) @ np.abs(o.F)
    act = tot > 0
    assert act.sum() > 100
    assert np.all(np.abs(net[act]) <= 1e-10 * tot[act])
    # blocked faces carry no flow (case 3, Section 2.4.2)
    assert np.all(o.F[o.case == 3] == 0.0)
    # solid cells are at rest (Section 2.4.1)
    assert np.all(o.u[~o.lm] == 0.0)
