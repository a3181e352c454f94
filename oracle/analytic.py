"""Closed-form references that pin the oracle (test infrastructure only).

* ``stefan_linear``: one-dimensional freezing of a semi-infinite melt with a
  linear solid fraction between solidus and liquidus (the energy equation,
  Eq. 4, with the linear form of Eq. 5).  The mushy zone then has the apparent
  heat capacity cp + L/(T_liq - T_sol), so the temperature is an error-function
  profile in each of the three regions, with fronts moving as sqrt(t); two
  transcendental conditions (heat-flux continuity at both fronts) fix the
  front constants.
* ``neumann_isothermal``: the classical Neumann solution for a pure
  substance, the limit T_liq - T_sol -> 0.
* ``conduction_series``: a slab with fixed end temperatures and a uniform
  initial temperature, no latent heat (Fourier sine series).
"""
from __future__ import annotations

import functools

import numpy as np
from scipy.optimize import brentq
from scipy.special import erf, erfc, erfcx


def stefan_linear(x, t, T_w, T_0, T_sol, T_liq, k, rho, cp, L):
    """Temperature at positions ``x`` and time ``t`` for the three-region
    similarity solution; returns (T, (X1, X2)) with X1 the solidus front and
    X2 the liquidus front.

    With eta = x / (2 sqrt(alpha t)), r^2 = 1 + L / (cp (T_liq - T_sol)) and
    fronts at eta = l1 < l2, the profile is T_w + (T_sol - T_w) erf(eta)/erf(l1)
    (solid), T_sol + B (erfc(r l1) - erfc(r eta)) (mushy) and
    T_0 - (T_0 - T_liq) erfc(eta)/erfc(l2) (liquid)."""
    alpha = k / (rho * cp)
    dT = T_liq - T_sol
    r = np.sqrt(1.0 + L / (cp * dT))
    ds = T_sol - T_w
    l1, l2, z1, z2 = _stefan_fronts(float(T_w), float(T_0), float(T_sol), float(T_liq),
                                    float(cp), float(L))
    eta = np.asarray(x, dtype=np.float64) / (2.0 * np.sqrt(alpha * t))

    def erfc_ratio(a, b):            # erfc(a) / erfc(b) without underflow
        return erfcx(a) / erfcx(b) * np.exp(b * b - a * a)

    with np.errstate(over="ignore", invalid="ignore"):
        mush = T_sol + dT * (1.0 - erfc_ratio(r * eta, z1)) / (1.0 - erfc_ratio(z2, z1))
        T = np.where(eta <= l1, T_w + ds * erf(eta) / erf(l1),
                     np.where(eta <= l2, mush,
                              T_0 - (T_0 - T_liq) * erfc_ratio(eta, l2)))
    s = 2.0 * np.sqrt(alpha * t)
    return T, (l1 * s, l2 * s)


@functools.lru_cache(maxsize=64)
def _stefan_fronts(T_w, T_0, T_sol, T_liq, cp, L):
    """Front constants (l1, l2) of ``stefan_linear`` and r l1, r l2.  Heat-flux
    continuity at l1 fixes B; T = T_liq at l2 then fixes l2; heat-flux continuity at l2 is
    the remaining equation for l1.  Scaled complementary error functions keep
    it accurate when the mushy interval is narrow (large r)."""
    dT = T_liq - T_sol
    r = np.sqrt(1.0 + L / (cp * dT))
    ds = T_sol - T_w

    def front2(l1):
        # erfc(r l2) = erfc(r l1) - dT / B = exp(-z1^2) * D
        z1 = r * l1
        Q = dT * r * erf(l1) * np.exp(l1 ** 2) / ds
        D = erfcx(z1) - Q
        if D <= 0.0:
            return None
        h = lambda z: np.log(erfcx(z)) - z * z + z1 * z1 - np.log(D)
        hi = z1 + 1.0
        while h(hi) > 0.0:
            hi = 2.0 * hi + 1.0
        z2 = z1 if h(z1) <= 0.0 else brentq(h, z1, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
        return z1, z2

    def flux_mismatch(l1):
        z = front2(l1)
        if z is None:
            return -np.inf
        z1, z2 = z
        l2 = z2 / r
        mushy = ds * np.exp(-l1 ** 2) / erf(l1) * np.exp(z1 * z1 - z2 * z2)
        liquid = (T_0 - T_liq) / erfcx(l2)
        return (mushy - liquid) / (T_liq - T_w)

    grid = np.geomspace(1e-9, 10.0, 4000)
    vals = np.array([flux_mismatch(v) for v in grid])
    j = int(np.argmax(vals < 0.0))
    lo, hi = grid[j - 1], grid[j]
    if not np.isfinite(vals[j]):
        # tighten the upper end onto the edge of the valid range
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if np.isfinite(flux_mismatch(mid)) and flux_mismatch(mid) < 0.0:
                hi = mid
                break
            if flux_mismatch(mid) > 0.0:
                lo = mid
            else:
                hi = mid
    l1 = brentq(flux_mismatch, lo, hi, xtol=1e-17, rtol=1e-15, maxiter=500)
    z1, z2 = front2(l1)
    return l1, z2 / r, z1, z2


def neumann_isothermal(x, t, T_w, T_0, T_m, k, rho, cp, L):
    """Classical two-region Neumann solution (pure substance melting at T_m)."""
    alpha = k / (rho * cp)
    St_s = cp * (T_m - T_w) / L
    St_l = cp * (T_0 - T_m) / L

    def f(lam):
        return (St_s * np.exp(-lam ** 2) / erf(lam)
                - St_l * np.exp(-lam ** 2) / erfc(lam) - lam * np.sqrt(np.pi))

    lam = brentq(f, 1e-6, 5.0, xtol=1e-15)
    eta = np.asarray(x) / (2.0 * np.sqrt(alpha * t))
    T = np.where(eta <= lam, T_w + (T_m - T_w) * erf(eta) / erf(lam),
                 T_0 - (T_0 - T_m) * erfc(eta) / erfc(lam))
    return T, lam * 2.0 * np.sqrt(alpha * t)


def conduction_series(x, t, ell, T_a, T_b, T_0, alpha, n_terms=4000):
    """T(x, t) on 0 < x < ell with T(0) = T_a, T(ell) = T_b, T(x, 0) = T_0."""
    x = np.asarray(x, dtype=np.float64)
    k = np.arange(1, n_terms + 1)
    sign = (-1.0) ** k
    b = 2.0 / (k * np.pi) * ((T_0 - T_a) * (1.0 - sign) + (T_b - T_a) * sign)
    decay = np.exp(-alpha * (k * np.pi / ell) ** 2 * t)
    return (T_a + (T_b - T_a) * x / ell
            + np.sin(np.outer(x, k) * np.pi / ell) @ (b * decay))
