"""Shared test helpers: seeded initial temperature fields with solid regions.

These only shape inputs (temperatures); the method's arithmetic lives in the
oracle and in the CUDA library.
"""
import numpy as np

from fvs_inputs import box_mesh, cases


def frozen_corner_field(mesh, T_hot=950.0, T_cold=800.0, frac=0.35, seed=0):
    """Temperatures with a solid block near x = 0 and a few scattered solid
    cells, so that every face case of the pressure system occurs."""
    ijk = mesh["cell_ijk"]
    nx, ny, nz = mesh["shape"]
    rng = np.random.default_rng(seed)
    T = np.full(len(ijk), T_hot) - rng.uniform(0.0, 20.0, len(ijk))
    block = (ijk[:, 0] < max(1, int(frac * nx))) & (ijk[:, 1] < max(1, int(0.7 * ny)))
    T[block] = T_cold
    # a lone solid cell inside the melt makes case-2 faces all around it
    lone = (ijk[:, 0] == nx - 2) & (ijk[:, 1] == ny // 2) & (ijk[:, 2] == nz // 2)
    T[lone] = T_cold
    return T


def mushy_field(mesh, seed=0):
    """Temperatures spread over liquid, mushy and solid (around the interval)."""
    rng = np.random.default_rng(seed)
    x = mesh["cell_ijk"][:, 0] / max(1, mesh["shape"][0] - 1)
    return 820.0 + 130.0 * x + rng.uniform(-5.0, 5.0, len(x))


def small_jittered_mesh(nx=8, ny=8, nz=4, seed=7, permute=True):
    return box_mesh(nx, ny, nz, cases.CAVITY, jitter=0.2, jitter_seed=seed,
                    permute_seed=(seed + 1 if permute else None))


def set_state(o, T, u=None):
    """Put an oracle into a given state (temperature, optional velocity)."""
    m = o.m
    metal = o.metal
    o.T = np.array(T, dtype=np.float64)
    o.T_old = o.T.copy()
    o.fs = o.fs_of(o.T)
    o.reset_grain()
    o.t_liq = np.where(metal & (o.T <= m["T_liq"]), 0.0, -1.0)
    o.t_sol = np.where(metal & (o.T <= m["T_sol"]), 0.0, -1.0)
    if u is not None:
        still = ~metal | (o.T <= m["T_sol"])
        o.u = np.array(u, dtype=np.float64)
        o.u_old = o.u.copy()
        o.u[still] = 0.0
        o.u_old[still] = 0.0
    return o
