"""Workload definitions: material data, wall conditions and seeded UQ inputs.

Plain data only (no finite-volume arithmetic).  The numbers are the synthetic
stand-ins for the paper's castings (Sections 3-5 use an Sn-Bi ingot, a clamp
and a pulley whose geometry and data are not available): an Al-like alloy in a
0.1 x 0.1 x 0.0125 m cavity.
"""
from __future__ import annotations

import numpy as np

from .mesh import box_mesh, casting_mesh

# wall types of a boundary patch
BC_ADIABATIC = 0      # no heat flux, no-slip
BC_DIRICHLET = 1      # fixed temperature, no-slip

AL_ALLOY = dict(
    rho=2700.0, k=150.0, cp=900.0, latent=3.9e5,
    T_sol=833.0, T_liq=913.0, mu=1.3e-3, beta=1e-4,
    T_ref=913.0, g=(0.0, -9.81, 0.0),
    darcy_C=1e8, darcy_eps=1e-3,
)

# the same alloy with the smeared Gulliver-Scheil solid fraction: partition
# coefficient and freezing temperature of an Al-Si-like alloy, smear width 2 K
AL_SI_SCHEIL = dict(AL_ALLOY, fs_model=1, kp=0.13, T_f=933.0, T_eps=2.0)

# The Al-Si alloy of the paper's UQ study (Section 5): freezing point of Al
# 660 C and eutectic (solidus) 577 C from the phase diagram; both lines
# straight, with the eutectic at 12.6 wt% Si and the largest solubility of
# Si in solid Al 1.65 wt% (textbook values of the Al-Si diagram, which the
# paper reads off a figure), so the liquidus slope is -83/12.6 K per wt%
# and kp, the ratio of the liquidus to the solidus slope, is 1.65/12.6.
# Density, heat capacity, conductivity and latent heat stay those of the
# cavity alloy; T_liq is the value at the mean composition of 10 wt%.
AL_SI_T_F = 933.15
AL_SI_SLOPE = (850.15 - 933.15) / 12.6
AL_SI_PAPER = dict(AL_ALLOY, T_sol=850.15, T_liq=AL_SI_T_F + AL_SI_SLOPE * 10.0, T_ref=AL_SI_T_F + AL_SI_SLOPE * 10.0,
                   fs_model=1, kp=1.65 / 12.6, T_f=AL_SI_T_F, T_eps=2.0)

CAVITY = (0.1, 0.1, 0.0125)


def cavity_walls(T_cold=700.0, T_hot=950.0):
    """x = 0 wall held cold, x = L wall held hot, the other four adiabatic."""
    return [(BC_DIRICHLET, T_cold), (BC_DIRICHLET, T_hot),
            (BC_ADIABATIC, 0.0), (BC_ADIABATIC, 0.0),
            (BC_ADIABATIC, 0.0), (BC_ADIABATIC, 0.0)]


def all_walls(T_wall):
    return [(BC_DIRICHLET, float(T_wall))] * 6


def props(material=None, walls=None, T_init=950.0, p_rtol=1e-8, precision=0, **tol):
    """Solver settings in the layout of ``fvs_props`` (see include/fvs.h)."""
    p = dict(material=dict(AL_ALLOY if material is None else material),
             walls=list(cavity_walls() if walls is None else walls),
             T_init=float(T_init), p_rtol=float(p_rtol), precision=int(precision),
             mom_rtol=1e-10, e_rtol=1e-10, e_tol_T=1e-8, max_e_iters=40)
    p.update(tol)
    return p


def config_small():
    """32x32x4 orthogonal cavity, dt 1e-3 s, 200 steps."""
    return dict(mesh=box_mesh(32, 32, 4, CAVITY), dt=1e-3, steps=200, props=props())


def config_jittered(n=128, steps=500, seed_jitter=1810, seed_perm=8572):
    """n^3 cavity, interior nodes jittered by +-0.2 cell widths, cells permuted."""
    return dict(mesh=box_mesh(n, n, n, CAVITY, jitter=0.2, jitter_seed=seed_jitter,
                              permute_seed=seed_perm),
                dt=1e-3, steps=steps, props=props())


def uq_inputs(n_samples, seed):
    """Stochastic inputs per sample: melt temperature ~ N(950, 10) K, wall
    temperature ~ U(650, 750) K, solute C0 ~ U(3, 5) wt%.  Returns [S, 3]."""
    rng = np.random.default_rng(seed)
    T_melt = rng.normal(950.0, 10.0, n_samples)
    T_wall = rng.uniform(650.0, 750.0, n_samples)
    C0 = rng.uniform(3.0, 5.0, n_samples)
    return np.stack([T_melt, T_wall, C0], axis=1)


def paper_uq_inputs(n_samples, seed):
    """The stochastic inputs of Section 5: initial melt temperature
    ~ N(1000, 10) K, wall temperature ~ N(500, 5) K, solute C0 ~ N(10, 0.2)
    wt%.  Returns [S, 3] in the order (T_melt, T_wall, C0)."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.normal(1000.0, 10.0, n_samples), rng.normal(500.0, 5.0, n_samples),
                     rng.normal(10.0, 0.2, n_samples)], axis=1)


def latin_hypercube_normal(means, sds, n, seed):
    """n Latin-hypercube samples of independent normal inputs: one point in
    each of n equal-probability strata of every marginal, the strata paired
    across inputs by random permutations.  Returns [n, len(means)]."""
    from scipy.stats import norm
    rng = np.random.default_rng(seed)
    d = len(means)
    U = (np.stack([rng.permutation(n) for _ in range(d)], axis=1) + rng.uniform(size=(n, d))) / n
    return np.asarray(means, dtype=np.float64) + np.asarray(sds, dtype=np.float64) * norm.ppf(U)


def paper_liquidus_of(C0):
    """Liquidus of the Al-Si line above: T_f + slope C0."""
    return AL_SI_T_F + AL_SI_SLOPE * np.asarray(C0)


def liquidus_of(C0):
    """Liquidus shifted linearly by -5 K per wt% about 913 K at 4 wt%."""
    return 913.0 - 5.0 * (np.asarray(C0) - 4.0)


# steel mold shell of the casting-like workload, its initial temperature and
# the metal-mold heat-transfer coefficient
STEEL_MOLD = dict(rho=7800.0, cp=500.0, k=30.0, h=2000.0, T_init=500.0)


def casting_props(precision=1, T_wall=500.0, **tol):
    """Casting in its mold: melt at 950 K, mold at 500 K, the mold's outer
    surface held at ``T_wall``; mixed precision by default."""
    return props(walls=all_walls(T_wall), T_init=950.0, precision=precision, mold=dict(STEEL_MOLD), **tol)


def config_casting(h=0.46e-3):
    """Plate 0.2 x 0.1 x 0.02 m with three 5 mm ribs and a 20 mm riser in a
    3 mm steel shell, voxels of side h (0.46 mm: about 4.4M metal and 2.1M
    mold cells), dt 1e-3 s."""
    return dict(mesh=casting_mesh(h), dt=1e-3, props=casting_props())
