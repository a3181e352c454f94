"""Plain FP64 CPU oracle of the fractional-step finite-volume solidification step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this file:
only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code with the CUDA library.

Everything is written as sparse matrices built from the definitions, assembled
with scipy.sparse and solved with a sparse direct solver, so that a reader can
check each operator against the paper by eye.  Section, equation and algorithm
numbers refer to Shahane et al., "Finite Volume Simulation Framework for Die
Casting with Uncertainty Quantification" (arXiv:1810.08572).

Readings of points the paper leaves open:
 * face vector area S_f = 1/2 (x_V3 - x_V1) x (x_V4 - x_V2); cell and face
   centres are vertex means; volume = 1/3 sum_f x_f . S_f (outward)
 * the local Jacobian of Eq. 12 has rows d = C1C2, V1V3, V2V4; on a boundary
   face C2 is the face centre
 * vertex values are arithmetic means of the cells around the vertex
   (Section 2.3); wall vertices take the wall value for velocity (no slip)
   and for temperature on fixed-temperature walls
 * convection uses the arithmetic mean of the two owner values (Section 2.3)
 * Darcy drag D = C fs^2 / ((1 - fs)^3 + eps) (Blake-Kozeny form of Eq. 3 with
   lambda folded into C)
 * the energy equation uses the same Crank-Nicolson diffusion and
   Adams-Bashforth convection as the momentum predictor (Eq. 6), with the
   flux level matching each temperature level
 * the solid fraction is linear between solidus and liquidus, or (material
   "fs_model" = 1) the Gulliver-Scheil law smeared near the solidus (Eq. 21,
   with partition coefficient kp, freezing temperature T_f and smear width
   T_eps); at each kink the derivative is taken from the side nearer the
   mushy interior (the Scheil side at T_liq and at T_sol + T_eps, the smear
   side at T_sol - T_eps); the tags stay T > T_sol in both laws
 * an LM cell none of whose faces carries flow is left out of the pressure
   system (its pressure is 0) and is treated like a solid cell when face
   gradients are smeared
 * the pressure of each connected part of the pressure system is fixed by
   zero mean; the right side is projected to zero sum on each part
 * a convective wall (heat-transfer coefficient h to an ambient T_inf)
   carries the orthogonal flux A (T_inf - T_C1)/(d_1/k_1 + 1/h) through the
   half cell and the film, d_1 the distance from the cell centre to the face
   centre; its vertices are free (cell means), as on adiabatic walls
 * a temperature-dependent conductivity k(T) of the metal (Section 3 uses a
   table; piecewise linear here, held constant outside it) is evaluated per
   face at the start of each step, at the mean of the two owner temperatures
   T^n (a fixed-temperature wall: the mean of the cell and wall values; a
   convective wall or a metal-mold interface: the metal cell's T^n), and
   used in both Crank-Nicolson halves
 * with natural convection off (Section 4: the castings are simulated
   without it) the momentum, pressure and correction steps are skipped:
   velocity, flux and pressure stay zero and the energy equation is pure
   conduction with latent heat
 * grain growth (Eq. 24-26): S takes the sign of the invariant-size
   approximation, S = 2 (C_l - C_0)/(C_s - C_l) <= 0, with the Scheil
   interface contents C_l = C_0 (1 - fs)^(kp - 1), C_s = kp C_l (as printed,
   with C_s - C_0 on top, S lies in (0, 2] and Eq. 25 has no real root);
   a cell grows only while 0 < fs < 1; d(r^2)/dt = lambda_s^2 D_s is
   integrated by the trapezoidal rule over each step, from r_0
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.sparse.csgraph import connected_components

BC_ADIABATIC = 0
BC_DIRICHLET = 1
BC_CONVECTIVE = 2


# ----------------------------------------------------------------------------
# Geometry (Section 2.3, Fig. 1, Eq. 11-12)
# ----------------------------------------------------------------------------
class Geometry:
    """Face and cell geometry of an unstructured hexahedral mesh.
    Section 2.3 (Fig. 1), the geometry behind Eq. 11-12."""

    def __init__(self, nodes, cells, faces, face_cells, patch):
        """Section 2.3: face vectors, centres, volumes and the local Jacobian of Eq. 12."""
        X = np.asarray(nodes, dtype=np.float64)
        self.nodes = X
        self.cells = np.asarray(cells, dtype=np.int64)
        self.faces = np.asarray(faces, dtype=np.int64)
        self.face_cells = np.asarray(face_cells, dtype=np.int64)
        self.patch = np.asarray(patch, dtype=np.int64)
        self.Nc, self.Nf, self.Nv = len(self.cells), len(self.faces), len(X)
        self.owner = self.face_cells[:, 0]
        self.neigh = self.face_cells[:, 1]
        self.interior = self.neigh >= 0
        Vx = [X[self.faces[:, k]] for k in range(4)]          # V1..V4
        self.Sf = 0.5 * np.cross(Vx[2] - Vx[0], Vx[3] - Vx[1])
        self.Af = np.linalg.norm(self.Sf, axis=1)
        self.n = self.Sf / self.Af[:, None]
        self.xf = X[self.faces].mean(axis=1)
        self.xc = X[self.cells].mean(axis=1)
        # volume by the divergence theorem, div x = 3
        xs = np.einsum("fi,fi->f", self.xf, self.Sf) / 3.0
        self.V = np.zeros(self.Nc)
        np.add.at(self.V, self.owner, xs)
        np.add.at(self.V, self.neigh[self.interior], -xs[self.interior])
        # d = C1 -> C2 (face centre on the boundary)
        c2 = np.where(self.interior[:, None], self.xc[np.maximum(self.neigh, 0)], self.xf)
        self.d = c2 - self.xc[self.owner]
        self.ndotd = np.einsum("fi,fi->f", self.n, self.d)
        # distances from the owner / neighbour centre to the face centre
        # (series resistance across a metal-mold interface)
        self.d_own = np.linalg.norm(self.xf - self.xc[self.owner], axis=1)
        self.d_nei = np.where(self.interior,
                              np.linalg.norm(self.xf - self.xc[np.maximum(self.neigh, 0)], axis=1), 0.0)
        # local frame xi: C1C2, eta: V1V3, zeta: V2V4 (Eq. 12); rows of J
        self.J = np.stack([self.d, Vx[2] - Vx[0], Vx[3] - Vx[1]], axis=1)
        self.Jinv = np.linalg.inv(self.J)
        # cross-diffusion vector of Eq. 11 and its weights on the local
        # differences: t . (J^-1 delta) = (J^-T t) . delta
        t = self.n - self.d / self.ndotd[:, None]
        self.w = np.einsum("fij,fi->fj", self.Jinv, t)
        # incidences
        rows = np.repeat(np.arange(self.Nc), 8)
        self.Pc = sp.csr_matrix((np.ones(8 * self.Nc), (self.cells.ravel(), rows)),
                                shape=(self.Nv, self.Nc))          # vertex x cell
        self.Pc.data[:] = 1.0                                      # repeated corners count once
        self.nv = np.asarray(self.Pc.sum(axis=1)).ravel()
        self.Pavg = sp.diags(1.0 / self.nv) @ self.Pc
        fr = np.repeat(np.arange(self.Nf), 4)
        self.Fv = sp.csr_matrix((np.ones(4 * self.Nf), (fr, self.faces.ravel())),
                                shape=(self.Nf, self.Nv))
        self.E31 = self._vdiff(2, 0)
        self.E42 = self._vdiff(3, 1)
        # neighbour set N(f): cells sharing a vertex with the face (Section 2.4.2)
        NB = (self.Fv @ self.Pc).tocsr()
        NB.data[:] = 1.0
        self.NB = NB
        # signed face -> cell sum (outward from each cell)
        fi = np.arange(self.Nf)
        r = np.concatenate([self.owner, self.neigh[self.interior]])
        c = np.concatenate([fi, fi[self.interior]])
        v = np.concatenate([np.ones(self.Nf), -np.ones(self.interior.sum())])
        self.Div = sp.csr_matrix((v, (r, c)), shape=(self.Nc, self.Nf))
        # C2 - C1 difference (boundary rows carry only -C1; the wall value is added separately)
        r = np.concatenate([fi, fi[self.interior]])
        c = np.concatenate([self.owner, self.neigh[self.interior]])
        v = np.concatenate([-np.ones(self.Nf), np.ones(self.interior.sum())])
        self.Dxi = sp.csr_matrix((v, (r, c)), shape=(self.Nf, self.Nc))
        # owner mean (1/2 each owner) used for convection and u*_f
        r = np.concatenate([fi, fi[self.interior]])
        c = np.concatenate([self.owner, self.neigh[self.interior]])
        vals = np.concatenate([np.full(self.Nf, 0.5), np.full(self.interior.sum(), 0.5)])
        self.Avg = sp.csr_matrix((vals, (r, c)), shape=(self.Nf, self.Nc))
        self.boundary_vertex = np.zeros(self.Nv, bool)
        self.boundary_vertex[self.faces[~self.interior].ravel()] = True

    def _vdiff(self, a, b):
        """Differences along a face's two diagonals: the eta and zeta derivatives of Eq. 12."""
        fi = np.arange(self.Nf)
        r = np.concatenate([fi, fi])
        c = np.concatenate([self.faces[:, a], self.faces[:, b]])
        v = np.concatenate([np.ones(self.Nf), -np.ones(self.Nf)])
        return sp.csr_matrix((v, (r, c)), shape=(self.Nf, self.Nv))

    # -- face normal derivative (Eq. 11) -------------------------------------
    def normal_derivative_rows(self, Dxi, Deta, Dzeta):
        """A_f (n . grad phi)_f as rows over cells, from the three local differences.
        Eq. 11 with the local derivatives of Eq. 12."""
        A = self.Af
        return (sp.diags(A * (1.0 / self.ndotd + self.w[:, 0])) @ Dxi
                + sp.diags(A * self.w[:, 1]) @ Deta
                + sp.diags(A * self.w[:, 2]) @ Dzeta).tocsr()


# ----------------------------------------------------------------------------
# Diffusion operators with wall data (Eq. 10-12)
# ----------------------------------------------------------------------------
def vertex_operator(g, fixed_mask, fixed_value):
    """phi_v = mean of the cells around v, or a fixed wall value where masked.
    Returns (P [Nv x Nc], c [Nv]) with phi_v = P phi + c.
    Section 2.3: a vertex value is the mean of the cells around the vertex."""
    keep = sp.diags((~fixed_mask).astype(np.float64))
    return (keep @ g.Pavg).tocsr(), np.where(fixed_mask, fixed_value, 0.0)


def diffusion_operator(g, face_mask, vP, vc, phi_b):
    """Affine operator L phi + l = sum over masked faces of sigma A_f (n . grad phi)_f.

    ``phi_b`` is the value at boundary faces (C2 := face centre).
    Eq. 11-12: direct and cross diffusion through the local Jacobian."""
    Deta = g.E31 @ vP
    Dzeta = g.E42 @ vP
    N = g.normal_derivative_rows(g.Dxi, Deta, Dzeta)
    k = g.Af * ((1.0 / g.ndotd + g.w[:, 0]) * np.where(g.interior, 0.0, phi_b)
                + g.w[:, 1] * (g.E31 @ vc) + g.w[:, 2] * (g.E42 @ vc))
    M = g.Div @ sp.diags(face_mask.astype(np.float64))
    return (M @ N).tocsr(), M @ k


def velocity_diffusion(g):
    """No-slip walls: wall vertices and wall faces carry u = 0.
    The diffusion term of Eq. 6, discretised as in Section 2.3."""
    vP, vc = vertex_operator(g, g.boundary_vertex, 0.0)
    return diffusion_operator(g, np.ones(g.Nf, bool), vP, vc, np.zeros(g.Nf))


def wall_data(g, walls):
    """Per face: wall type (-1 interior), wall temperature (or ambient
    temperature of a convective wall) and film coefficient h.
    Boundary data only (the wall conditions of Sections 3-4); no method arithmetic."""
    btype = np.full(g.Nf, -1)
    bval = np.zeros(g.Nf)
    bh = np.zeros(g.Nf)
    for pid, w in enumerate(walls):
        m = g.patch == pid
        btype[m] = w[0]
        bval[m] = w[1]
        bh[m] = w[2] if len(w) > 2 else 0.0
    return btype, bval, bh


def temperature_diffusion(g, walls, k_face=None, interface=None, G_int=None, G_conv=None):
    """Fixed-temperature walls enter through their vertices and faces;
    adiabatic walls carry no flux.

    With ``k_face`` the face flux is scaled by that face's conductivity (the
    result is the conductive flux itself).  Faces flagged in ``interface``
    (a metal cell against a mold cell) carry only the orthogonal flux
    G_int (T_C2 - T_C1) through the series resistance of the two half cells
    and the interface coefficient; convective wall faces carry
    G_conv (T_inf - T_C1) (no cross terms on either).
    The conduction term of Eq. 4, discretised by Eq. 11-12."""
    btype, bval, bh = wall_data(g, walls)
    dir_face = btype == BC_DIRICHLET
    conv_face = btype == BC_CONVECTIVE
    if conv_face.any() and k_face is None:
        raise ValueError("convective walls need face conductivities")
    # a vertex on fixed-temperature walls takes the mean of the values of the
    # fixed-temperature wall faces that contain it (each face counted once)
    cnt = np.zeros(g.Nv)
    acc = np.zeros(g.Nv)
    for f in np.nonzero(dir_face)[0]:
        for v in set(g.faces[f].tolist()):
            cnt[v] += 1
            acc[v] += bval[f]
    fixed = cnt > 0
    val = np.where(fixed, acc / np.maximum(cnt, 1), 0.0)
    vP, vc = vertex_operator(g, fixed, val)
    face_mask = g.interior | dir_face | conv_face
    bdir = np.where(dir_face, bval, 0.0)
    if k_face is None:
        return diffusion_operator(g, g.interior | dir_face, vP, vc, bdir)
    if interface is None:
        interface = np.zeros(g.Nf, bool)
    G_int = np.zeros(g.Nf) if G_int is None else G_int
    G_conv = np.zeros(g.Nf) if G_conv is None else G_conv
    Deta = g.E31 @ vP
    Dzeta = g.E42 @ vP
    N = g.normal_derivative_rows(g.Dxi, Deta, Dzeta)
    k = g.Af * ((1.0 / g.ndotd + g.w[:, 0]) * np.where(g.interior, 0.0, bdir)
                + g.w[:, 1] * (g.E31 @ vc) + g.w[:, 2] * (g.E42 @ vc))
    # conductive flux per face: k_f times the face gradient, or the series
    # flux on interface faces and convective walls (no cross terms there);
    # the wall row of Dxi carries -T_C1
    series = interface | conv_face
    G = np.where(interface, G_int, np.where(conv_face, G_conv, 0.0))
    Nk = (sp.diags(np.where(series, 0.0, k_face)) @ N + sp.diags(G) @ g.Dxi).tocsr()
    kk = np.where(series, np.where(conv_face, G_conv * bval, 0.0), k_face * k)
    M = g.Div @ sp.diags(face_mask.astype(np.float64))
    return (M @ Nk).tocsr(), M @ kk


# ----------------------------------------------------------------------------
# Material laws (Eq. 3, Eq. 5 in its linear form, Eq. 21, Eq. 22-23)
# ----------------------------------------------------------------------------
def scheil_law(m):
    """(kp, T_f, T_eps) of the smeared Gulliver-Scheil law if the material
    selects it (fs_model = 1), else None (linear solid fraction).
    Eq. 5 and its smeared form, Eq. 21."""
    if int(m.get("fs_model", 0)) == 1:
        return (float(m["kp"]), float(m["T_f"]), float(m["T_eps"]))
    return None


def _scheil_core(T, T_liq, kp, T_f):
    """Eq. 5 between the liquidus and the smear: 1 - r^(1/(kp-1)) with
    r = (T - T_f)/(T_liq - T_f) (both differences negative), and its slope."""
    e = 1.0 / (kp - 1.0)
    r = (T - T_f) / (T_liq - T_f)
    return 1.0 - r ** e, -e * r ** (e - 1.0) / (T_liq - T_f)


def solid_fraction(T, T_sol, T_liq, scheil=None):
    """fs(T): linear between T_sol and T_liq, or Eq. 21 when scheil =
    (kp, T_f, T_eps) is given."""
    T = np.asarray(T, dtype=np.float64)
    if scheil is None:
        return np.clip((T_liq - T) / (T_liq - T_sol), 0.0, 1.0)
    kp, T_f, T_eps = scheil
    T1, T2 = T_sol - T_eps, T_sol + T_eps
    f_hat = _scheil_core(T2, T_liq, kp, T_f)[0]
    Tc = np.clip(T, T2, T_liq)                      # keeps the power's base positive
    f_sch = _scheil_core(Tc, T_liq, kp, T_f)[0]
    f_smr = f_hat - (T - T2) * (1.0 - f_hat) / (2.0 * T_eps)
    return np.where(T > T_liq, 0.0, np.where(T <= T1, 1.0, np.where(T < T2, f_smr, f_sch)))


def solid_fraction_slope(T, T_sol, T_liq, scheil=None):
    """dfs/dT, taken at each kink from the side nearer the mushy interior.
    Slope of Eq. 5 / Eq. 21, used by the latent-heat linearisation of Eq. 18-20."""
    T = np.asarray(T, dtype=np.float64)
    if scheil is None:
        return np.where((T >= T_sol) & (T <= T_liq), -1.0 / (T_liq - T_sol), 0.0)
    kp, T_f, T_eps = scheil
    T1, T2 = T_sol - T_eps, T_sol + T_eps
    f_hat = _scheil_core(T2, T_liq, kp, T_f)[0]
    Tc = np.clip(T, T2, T_liq)
    d_sch = _scheil_core(Tc, T_liq, kp, T_f)[1]
    d_smr = -(1.0 - f_hat) / (2.0 * T_eps)
    return np.where((T > T_liq) | (T < T1), 0.0, np.where(T < T2, d_smr, d_sch))


def grain_supersaturation(fs, kp):
    """Eq. 26 in the sign of the invariant-size approximation:
    S = 2 (C_l - C_0)/(C_s - C_l) with C_l = C_0 (1 - fs)^(kp - 1) and
    C_s = kp C_l, so that C_0 / C_l = (1 - fs)^(1 - kp) and C_0 cancels."""
    fs = np.clip(np.asarray(fs, dtype=np.float64), 0.0, 1.0)
    c0_over_cl = (1.0 - fs) ** (1.0 - kp)
    return 2.0 * (1.0 - c0_over_cl) / (kp - 1.0)


def grain_lambda(fs, kp):
    """Eq. 25: lambda_s = -S/(2 sqrt(pi)) + sqrt(S^2/(4 pi) - S); zero
    outside the mushy range (no liquid to grow into, or no solid yet)."""
    fs = np.asarray(fs, dtype=np.float64)
    S = grain_supersaturation(fs, kp)
    lam = -S / (2.0 * np.sqrt(np.pi)) + np.sqrt(np.maximum(S * S / (4.0 * np.pi) - S, 0.0))
    return np.where((fs > 0.0) & (fs < 1.0), lam, 0.0)


def grain_update(r2, fs_a, fs_b, dt, kp, D_s):
    """One step of Eq. 24 written for r^2: d(r^2)/dt = lambda_s^2 D_s, by the
    trapezoidal rule between the solid fractions at both ends of the step."""
    la, lb = grain_lambda(fs_a, kp), grain_lambda(fs_b, kp)
    return r2 + dt * D_s * 0.5 * (la * la + lb * lb)


def darcy_coefficient(fs, C, eps):
    """Eq. 3: the Blake-Kozeny drag coefficient of Section 2.1."""
    return C * fs * fs / ((1.0 - fs) ** 3 + eps)


def sdas_um(cooling_rate):
    """Eq. 22: lambda_2 = 39.4 (dT/dt)^-0.317 micrometres."""
    return 39.4 * np.power(cooling_rate, -0.317)


def yield_strength_mpa(sdas):
    """Eq. 23: sigma_0.2 = 59.0 lambda_2^-1/2 + 120.3 MPa."""
    return 59.0 / np.sqrt(sdas) + 120.3


# ----------------------------------------------------------------------------
# Linear solves
# ----------------------------------------------------------------------------
def solve(A, b):
    """Library primitive: a sparse direct solve (no method arithmetic)."""
    x = spla.spsolve(A.tocsc(), b)
    return np.atleast_1d(x)


def pressure_components(App):
    """Connected parts of the pressure system (symmetric closure of its pattern).
    Section 2.5: the disjoint liquid pockets of the pressure system."""
    S = (abs(App) + abs(App).T).tocsr()
    S.eliminate_zeros()
    return connected_components(S, directed=False)


def solve_singular(App, b):
    """Solve A p = b on each connected part: project b to zero sum, pin the
    first unknown of each part, then shift p to zero mean (Section 2.5 notes
    the disjoint liquid pockets; each pocket is a separate singular block)."""
    n = App.shape[0]
    if n == 0:
        return np.zeros(0), 0
    ncomp, lab = pressure_components(App)
    b = b.copy()
    for c in range(ncomp):
        m = lab == c
        b[m] -= b[m].mean()
    A = App.tolil()
    rhs = b.copy()
    for c in range(ncomp):
        i = np.nonzero(lab == c)[0][0]
        A.rows[i] = [i]
        A.data[i] = [1.0]
        rhs[i] = 0.0
    p = solve(A.tocsr(), rhs)
    for c in range(ncomp):
        m = lab == c
        p[m] -= p[m].mean()
    return p, ncomp


# ----------------------------------------------------------------------------
# The solver state and one time step (Section 2.2, steps 1-5)
# ----------------------------------------------------------------------------
class Oracle:
    """One deterministic run of the method on one mesh.
    Section 2.2: the fractional-step algorithm, one step at a time."""

    def __init__(self, mesh, props):
        """Base operators of Section 2.3 and the material data of Section 2.1."""
        self.g = g = Geometry(mesh["nodes"], mesh["cells"], mesh["faces"],
                              mesh["face_cells"], mesh["patch"])
        self.m = dict(props["material"])
        self.walls = list(props["walls"])
        self.props = props
        self.Lu, _ = velocity_diffusion(g)
        m = self.m
        # zones: 0 metal, 1 mold (conduction only: no flow, no latent heat);
        # the mold material and the metal-mold interface coefficient h come
        # from props["mold"] = dict(rho, cp, k, h, T_init)
        zone = mesh.get("cell_zone")
        self.metal = np.ones(g.Nc, bool) if zone is None else (np.asarray(zone) == 0)
        mold = props.get("mold")
        if mold is None:
            self.metal[:] = True
        self.mold = mold
        rho_c = np.where(self.metal, m["rho"], mold["rho"] if mold else m["rho"])
        cp_c = np.where(self.metal, m["cp"], mold["cp"] if mold else m["cp"])
        self.rcp = rho_c * cp_c
        self.rL = np.where(self.metal, m["rho"] * m["latent"], 0.0)
        q = np.maximum(g.neigh, 0)
        self.interface = g.interior & (self.metal[g.owner] != self.metal[q])
        # k(T) of the metal: props["k_table"] = [(T, k), ...], piecewise
        # linear, constant outside; props["no_flow"]: natural convection off
        kt = props.get("k_table")
        self.k_table = None if not kt else (np.array([a for a, _ in kt], float), np.array([b for _, b in kt], float))
        self.no_flow = bool(props.get("no_flow", False))
        self.btype, self.bval, self.bh = wall_data(g, self.walls)
        self.Deta_p = (g.E31 @ g.Pavg).tocsr()
        self.Dzeta_p = (g.E42 @ g.Pavg).tocsr()
        self.T = np.where(self.metal, props["T_init"], mold["T_init"] if mold else props["T_init"])
        # conductive operator (k inside): sum over faces of the face flux
        self.LTk, self.lTk = self.conduction(self.T)
        self.scheil = scheil_law(m)
        self.fs = self.fs_of(self.T)
        # grain growth (Eq. 24-26): props["grain"] = dict(kp, D_s, r0)
        self.grain = props.get("grain")
        self.reset_grain()
        self.T_old = self.T.copy()
        self.u = np.zeros((g.Nc, 3))
        self.u_old = np.zeros((g.Nc, 3))
        self.F = np.zeros(g.Nf)
        self.F_old = np.zeros(g.Nf)
        self.p = np.zeros(g.Nc)
        self.time = 0.0
        self.nstep = 0
        self.t_liq = np.where(self.metal & (self.T <= m["T_liq"]), 0.0, -1.0)
        self.t_sol = np.where(self.metal & (self.T <= m["T_sol"]), 0.0, -1.0)
        self.stats = {}

    # -- helpers ---------------------------------------------------------------
    def k_metal(self, T):
        """Conductivity of the metal at temperatures T.
        k(T) of Section 3 (the validation ingot's table), piecewise linear between table points."""
        if self.k_table is None:
            return np.full(np.shape(T), float(self.m["k"]))
        return np.interp(T, self.k_table[0], self.k_table[1])

    def conduction(self, T):
        """Conductive operator (L T + l = sum over faces of the conductive
        flux) with the conductivities of the temperature field T (only read
        with a k(T) table).
        The conduction term of Eq. 4 (Eq. 11-12), with the mold of Section 4."""
        g, m, mold = self.g, self.m, self.mold
        metal = self.metal
        q = np.maximum(g.neigh, 0)
        k_mold = mold["k"] if mold else m["k"]
        if self.k_table is None:
            k_own = np.where(metal[g.owner], m["k"], k_mold)
            k_nei = np.where(metal[q], m["k"], k_mold)
            k_face = k_own
        else:
            To = T[g.owner]
            Tq = np.where(g.interior, T[q], np.where(self.btype == BC_DIRICHLET, self.bval, To))
            k_own = np.where(metal[g.owner], self.k_metal(To), k_mold)
            k_nei = np.where(metal[q], self.k_metal(T[q]), k_mold)
            k_face = np.where(metal[g.owner], self.k_metal(0.5 * (To + Tq)), k_mold)
        G_int = np.zeros(g.Nf)
        if self.interface.any():
            G_int = np.where(self.interface, g.Af / (g.d_own / k_own + 1.0 / mold["h"] + g.d_nei / k_nei), 0.0)
        conv = self.btype == BC_CONVECTIVE
        G_conv = np.where(conv, g.Af / (g.d_own / k_own + 1.0 / np.where(conv, self.bh, 1.0)), 0.0)
        return temperature_diffusion(g, self.walls, k_face=k_face, interface=self.interface, G_int=G_int,
                                     G_conv=G_conv)

    def reset_grain(self):
        """Initial grain radius of the growth law, Eq. 24-26."""
        r0 = self.grain["r0"] if self.grain else 0.0
        self.r2 = np.where(self.metal, r0 * r0, 0.0)

    def grain_radius(self):
        """Grain radius per cell (m); 0 in the mold.
        Eq. 24-26."""
        return np.sqrt(self.r2)

    def fs_of(self, T):
        """Solid fraction of every cell at temperatures T (0 in the mold).
        Eq. 5 / Eq. 21, or the linear law between solidus and liquidus."""
        m = self.m
        return np.where(self.metal, solid_fraction(T, m["T_sol"], m["T_liq"], self.scheil), 0.0)

    def conv(self, phi, F):
        """Conv(phi, F)_c = sum_f sigma F_f (phi_C1 + phi_C2)/2 (walls carry F = 0).
        The convection term of Eq. 6, discretised as in Section 2.3."""
        return self.g.Div @ (F * (self.g.Avg @ phi))

    def face_cases(self, lm):
        """Section 2.4.2: 0 wall, 1 no solid neighbour, 2 solid neighbour only,
        3 solid owner.  Returns (case, ppe_active)."""
        g = self.g
        own_ok = lm[g.owner] & np.where(g.interior, lm[np.maximum(g.neigh, 0)], False)
        case = np.where(g.interior, np.where(own_ok, 1, 3), 0)
        # LM cells with no flow face are removed from the pressure system
        flow = np.zeros(g.Nc, bool)
        f12 = case == 1
        flow[g.owner[f12]] = True
        flow[g.neigh[f12]] = True
        ppe = lm & flow
        nsolid = g.NB @ (~ppe).astype(np.float64)
        case = np.where((case == 1) & (nsolid > 0), 2, case)
        return case, ppe

    def smeared_rows(self, case, ppe):
        """Section 2.4.2, Eq. 15-16: on case-2 faces the deleted (solid)
        neighbours' coefficients are spread equally over the remaining ones."""
        g = self.g
        De = self.Deta_p.tolil(copy=True)
        Dz = self.Dzeta_p.tolil(copy=True)
        NB = g.NB
        for f in np.nonzero(case == 2)[0]:
            nbr = NB.indices[NB.indptr[f]:NB.indptr[f + 1]]
            keep = nbr[ppe[nbr]]
            gone = nbr[~ppe[nbr]]
            for D in (De, Dz):
                row = dict(zip(D.rows[f], D.data[f]))
                s = sum(row.get(j, 0.0) for j in gone)
                for j in gone:
                    row.pop(j, None)
                for j in keep:
                    row[j] = row.get(j, 0.0) + s / len(keep)
                cols = sorted(row)
                D.rows[f] = cols
                D.data[f] = [row[j] for j in cols]
        return De.tocsr(), Dz.tocsr()

    # -- the step ------------------------------------------------------------------
    def step(self, dt):
        """Section 2.2: tags, predictor (Eq. 6), pressure (Eq. 9), correction (Eq. 8, 17), energy (Eq. 4, 18-20)."""
        g, m = self.g, self.m
        rho, mu = m["rho"], m["mu"]
        T_n, fs_n = self.T, self.fs
        # 1. tags from the previous temperature (Section 2.4); mold cells are never LM
        lm = self.metal & (T_n > m["T_sol"])
        solid = ~lm
        u_n = self.u.copy(); u_n[solid] = 0.0
        u_o = self.u_old.copy(); u_o[solid] = 0.0
        blocked = ~(lm[g.owner] & np.where(g.interior, lm[np.maximum(g.neigh, 0)], False))
        F_n = np.where(blocked, 0.0, self.F)
        F_o = np.where(blocked, 0.0, self.F_old)

        act = np.nonzero(lm)[0]
        if self.no_flow:
            # natural convection off: no flow at all
            case, ppe = self.face_cases(lm)
            u_star = np.zeros((g.Nc, 3))
            u_new = np.zeros((g.Nc, 3))
            F_new = np.zeros(g.Nf)
            p = np.zeros(g.Nc)
            b_full = np.zeros(g.Nc)
            self.stats = dict(n_active=int(lm.sum()), n_ppe=0, ncomp=0, ppe_relres=0.0)
        else:
            u_star, u_new, F_new, p, case, ppe, b_full = self.flow_step(dt, lm, act, u_n, u_o, F_n, F_o, T_n, fs_n)

        # 5. energy with latent heat on all cells (Eq. 4, Eq. 18-20), with the
        # conductivities of T^n when k depends on T
        if self.k_table is not None:
            self.LTk, self.lTk = self.conduction(T_n)
        T_new, fs_new, e_its = self.energy(dt, T_n, fs_n, self.T_old, F_n, F_o)

        # 6. microstructure bookkeeping (Eq. 22-23 use the local cooling rate;
        # Eq. 24-26 grow the grains of the cells that are mushy)
        self.update_crossings(T_n, T_new, dt)
        if self.grain:
            gr = self.grain
            self.r2 = np.where(self.metal, grain_update(self.r2, fs_n, fs_new, dt, gr["kp"], gr["D_s"]), 0.0)

        self.stats.update(e_its=e_its, n_faces_case2=int((case == 2).sum()),
                          n_faces_case3=int((case == 3).sum()))
        self.T_old, self.T, self.fs = T_n, T_new, fs_new
        self.u_old, self.u = u_n, u_new
        self.F_old, self.F = F_n, F_new
        self.p = p
        self.u_star = u_star
        self.case, self.ppe, self.lm = case, ppe, lm
        self.b_ppe = b_full
        self.time += dt
        self.nstep += 1
        return self.stats

    def flow_step(self, dt, lm, act, u_n, u_o, F_n, F_o, T_n, fs_n):
        """Steps 2-4 of Section 2.2: momentum predictor, pressure Poisson
        equation and the flux / velocity correction on the LM cells."""
        g, m = self.g, self.m
        rho, mu = m["rho"], m["mu"]
        # 2. momentum predictor on LM cells, Eq. 6 with Section 2.4.1 row deletion
        Lu = self.Lu[act][:, act]
        V = g.V[act]
        D = darcy_coefficient(fs_n[act], m["darcy_C"], m["darcy_eps"])
        M = (sp.diags(rho * V / dt + D * V) - 0.5 * mu * Lu).tocsr()
        gvec = np.asarray(m["g"], dtype=np.float64)
        buoy = -rho * m["beta"] * (T_n[act] - m["T_ref"])[:, None] * gvec[None, :] * V[:, None]
        u_star = np.zeros((g.Nc, 3))
        for k in range(3):
            conv = 1.5 * self.conv(u_n[:, k], F_n) - 0.5 * self.conv(u_o[:, k], F_o)
            rhs = (rho * V / dt * u_n[act, k] - rho * conv[act]
                   + 0.5 * mu * (self.Lu @ u_n[:, k])[act] + buoy[:, k])
            u_star[act, k] = solve(M, rhs)

        # 3. pressure Poisson equation on the flowing LM cells (Eq. 9, Section 2.4.2)
        case, ppe = self.face_cases(lm)
        De, Dz = self.smeared_rows(case, ppe)
        Nrow = g.normal_derivative_rows(g.Dxi, De, Dz)           # A_f (n . grad p)_f^mod
        flow = (case == 1) | (case == 2)
        Mdiv = g.Div @ sp.diags(flow.astype(np.float64))
        App_full = (Mdiv @ Nrow / rho).tocsr()
        uf = g.Avg @ u_star                                        # u*_f, owner mean
        Fstar = g.Af * np.einsum("fi,fi->f", g.n, uf) * flow
        b_full = (g.Div @ Fstar) / dt
        pa = np.nonzero(ppe)[0]
        App = App_full[pa][:, pa]
        p_act, ncomp = solve_singular(App, b_full[pa])
        p = np.zeros(g.Nc)
        p[pa] = p_act
        resid = b_full[pa] - App @ p_act
        self.stats = dict(n_active=int(lm.sum()), n_ppe=int(ppe.sum()), ncomp=ncomp,
                          ppe_relres=float(np.linalg.norm(resid) / max(np.linalg.norm(b_full[pa]), 1e-300)))

        # 4. face flux and cell velocity correction (Eq. 8, Eq. 17)
        F_new = (Fstar - dt / rho * (Nrow @ p)) * flow
        dxi, deta, dzeta = g.Dxi @ p, De @ p, Dz @ p
        grad_f = np.einsum("fij,fj->fi", g.Jinv, np.stack([dxi, deta, dzeta], axis=1))
        cnt = np.abs(g.Div) @ flow.astype(np.float64)
        gsum = np.abs(g.Div) @ (grad_f * flow[:, None])
        grad_c = np.where(cnt[:, None] > 0, gsum / np.maximum(cnt, 1)[:, None], 0.0)
        u_new = np.zeros((g.Nc, 3))
        u_new[act] = u_star[act] - dt / rho * grad_c[act]

        return u_star, u_new, F_new, p, case, ppe, b_full

    def energy_residual(self, T, dt, T_n, fs_n, T_o, F_n, F_o):
        """R(T) of the discrete energy equation (all terms moved to the left).
        Eq. 4 in the discrete form of Eq. 18-20."""
        g, m = self.g, self.m
        rcp, rL = self.rcp, self.rL
        conv = 1.5 * self.conv(T_n, F_n) - 0.5 * self.conv(T_o, F_o)
        fs = self.fs_of(T)
        return (rcp * g.V / dt * (T - T_n) + rcp * conv
                - 0.5 * (self.LTk @ T + self.lTk) - 0.5 * (self.LTk @ T_n + self.lTk)
                - rL * g.V / dt * (fs - fs_n))

    def energy(self, dt, T_n, fs_n, T_o, F_n, F_o):
        """Section 2.4.4 iteration: S_p, S_c from the last iterate, solve,
        update fs with lambda = 1; stop when T and fs stop changing.  After 20
        passes without convergence the temperature is taken from the
        linearised enthalpy instead (same fixed point)."""
        g, m = self.g, self.m
        cp, L = m["cp"], m["latent"]
        rcp, rL, metal = self.rcp, self.rL, self.metal
        Ts, Tl = m["T_sol"], m["T_liq"]
        conv = 1.5 * self.conv(T_n, F_n) - 0.5 * self.conv(T_o, F_o)
        base = (rcp * g.V / dt * T_n - rcp * conv
                + 0.5 * (self.LTk @ T_n + self.lTk) + 0.5 * self.lTk)
        K = (-0.5 * self.LTk).tocsr()
        T, fs = T_n.copy(), fs_n.copy()
        tolT = self.props.get("oracle_tol_T", 1e-11)
        for it in range(1, 200):
            dfs = np.where(metal, solid_fraction_slope(T, Ts, Tl, self.scheil), 0.0)
            Sp = rL * g.V / dt * dfs
            Sc = rL * g.V / dt * (fs - fs_n - dfs * T)
            A = (K + sp.diags(rcp * g.V / dt - Sp)).tocsr()
            T_lin = solve(A, base + Sc)
            if it <= 20:
                T_next = T_lin
            else:
                H = cp * T_lin + L * (1.0 - fs - dfs * (T_lin - T))
                T_next = np.where(metal, temperature_from_enthalpy(H, cp, L, Ts, Tl, self.scheil), T_lin)
            fs_next = self.fs_of(T_next)
            dT = np.max(np.abs(T_next - T))
            dF = np.max(np.abs(fs_next - fs))
            T, fs = T_next, fs_next
            if dT <= tolT and dF <= 1e-12:
                break
        return T, fs, it

    def update_crossings(self, T_n, T_new, dt):
        """Crossing times behind Eq. 22 (local solidification time and cooling rate)."""
        m = self.m
        for which, Tc in (("t_liq", m["T_liq"]), ("t_sol", m["T_sol"])):
            arr = getattr(self, which)
            hit = self.metal & (arr < 0) & (T_n > Tc) & (T_new <= Tc)
            frac = (T_n - Tc) / np.where(hit, T_n - T_new, 1.0)
            arr[hit] = self.time + dt * frac[hit]

    def qoi(self):
        """Local solidification time, cooling rate, SDAS and yield strength
        per cell (NaN where the cell has not yet passed the solidus).
        Eq. 22-23."""
        m = self.m
        done = self.metal & (self.t_sol >= 0) & (self.t_liq >= 0)
        tf = np.where(done, self.t_sol - self.t_liq, np.nan)
        with np.errstate(divide="ignore", invalid="ignore"):
            cr = (m["T_liq"] - m["T_sol"]) / tf
            lam = sdas_um(cr)
            ys = yield_strength_mpa(lam)
        return dict(t_f=tf, cooling_rate=cr, sdas=lam, yield_strength=ys)

    def qoi_extremes(self):
        """The four outputs of Section 5 over the whole domain: total
        solidification time (the latest solidus crossing; NaN while a metal
        cell is above the solidus), maximum SDAS, minimum yield strength and
        maximum grain radius."""
        q = self.qoi()
        metal = self.metal
        done = metal & (self.t_sol >= 0)
        both = np.isfinite(q["sdas"]) & metal
        t_total = self.t_sol[metal].max() if done.sum() == metal.sum() else np.nan
        lam = q["sdas"][both].max() if both.any() else np.nan
        ys = q["yield_strength"][both].min() if both.any() else np.nan
        return np.array([t_total, lam, ys, self.grain_radius()[metal].max()])

    def run(self, dt, nsteps):
        """Repeated steps of Section 2.2."""
        for _ in range(nsteps):
            self.step(dt)
        return self


def temperature_from_enthalpy(H, cp, L, T_sol, T_liq, scheil=None):
    """Invert H(T) = cp T + L (1 - fs(T)), strictly increasing in T.  Linear
    fs: piecewise linear, inverted in closed form.  Eq. 21: closed form in
    the solid, liquid and smear pieces; bisection on the Gulliver-Scheil
    piece (200 halvings of [T_sol + T_eps, T_liq])."""
    H = np.asarray(H, dtype=np.float64)
    if scheil is None:
        H_sol = cp * T_sol
        H_liq = cp * T_liq + L
        T_mush = T_sol + (H - H_sol) / (H_liq - H_sol) * (T_liq - T_sol)
        return np.where(H <= H_sol, H / cp, np.where(H >= H_liq, (H - L) / cp, T_mush))
    kp, T_f, T_eps = scheil
    T1, T2 = T_sol - T_eps, T_sol + T_eps

    def enthalpy(T):
        """H(T) of Eq. 4-5."""
        return cp * T + L * (1.0 - solid_fraction(T, T_sol, T_liq, scheil))

    H1, H2, H3 = cp * T1, float(enthalpy(T2)), cp * T_liq + L
    lo = np.full(H.shape, T2)
    hi = np.full(H.shape, T_liq)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        below = enthalpy(mid) < H
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    T_sch = 0.5 * (lo + hi)
    T_smr = T1 + (H - H1) / (H2 - H1) * (T2 - T1)
    return np.where(H <= H1, H / cp, np.where(H >= H3, (H - L) / cp, np.where(H < H2, T_smr, T_sch)))
