"""Pins of the grain-growth model (Eq. 24-26) in the oracle.  CPU only."""
import numpy as np
import pytest
from scipy.integrate import quad

from fvs_inputs import box_mesh, cases
from oracle.fv import (Oracle, grain_lambda, grain_supersaturation, grain_update, scheil_law, solid_fraction)
from tests.helpers import set_state

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

KP = 0.13


def test_no_supersaturation_before_freezing_and_growth_with_fs():
    """At fs = 0 the liquid holds the nominal content: S = 0 and lambda_s = 0.
    Solute rejected by the growing solid raises C_l, so -S and lambda_s grow
    with fs; both are real and finite inside the mushy range."""
    assert grain_supersaturation(0.0, KP) == 0.0
    assert grain_lambda(0.0, KP) == 0.0
    fs = np.linspace(1e-6, 1.0 - 1e-6, 2001)
    S = grain_supersaturation(fs, KP)
    lam = grain_lambda(fs, KP)
    assert np.all(S < 0.0) and np.all(np.diff(S) < 0.0)
    assert np.all(np.isfinite(lam)) and np.all(lam > 0.0) and np.all(np.diff(lam) > 0.0)
    assert grain_lambda(1.0, KP) == 0.0 and grain_lambda(1.2, KP) == 0.0


def test_lambda_inverts_the_invariant_size_relation():
    """Eq. 25 is the positive root of lambda^2 + (S / sqrt(pi)) lambda + S = 0,
    i.e. S = -sqrt(pi) lambda^2 / (sqrt(pi) + lambda): mapping lambda back
    must return S (a slip in the 4 pi or in a sign fails this)."""
    fs = np.linspace(1e-4, 0.999, 500)
    S = grain_supersaturation(fs, KP)
    lam = grain_lambda(fs, KP)
    back = -np.sqrt(np.pi) * lam ** 2 / (np.sqrt(np.pi) + lam)
    np.testing.assert_allclose(back, S, rtol=1e-12)
    # small supersaturation: lambda_s -> sqrt(-S)
    s_small = grain_supersaturation(1e-9, KP)
    assert grain_lambda(1e-9, KP) == pytest.approx(np.sqrt(-s_small), rel=1e-3)


def test_supersaturation_from_the_liquidus_line():
    """With the Scheil law the interface liquid content can also be read off
    a straight liquidus, C_l / C_0 = (T - T_f)/(T_liq - T_f); Eq. 26 computed
    from that and from fs(T) agree."""
    m = cases.AL_SI_SCHEIL
    law = scheil_law(m)
    T = np.linspace(m["T_sol"] + m["T_eps"] + 0.5, m["T_liq"] - 0.5, 200)
    fs = solid_fraction(T, m["T_sol"], m["T_liq"], law)
    cl_over_c0 = (T - m["T_f"]) / (m["T_liq"] - m["T_f"])
    kp = m["kp"]
    S_line = 2.0 * (cl_over_c0 - 1.0) / (kp * cl_over_c0 - cl_over_c0)
    np.testing.assert_allclose(grain_supersaturation(fs, kp), S_line, rtol=1e-11)


def test_time_integration():
    """Eq. 24 as d(r^2)/dt = lambda_s^2 D_s: exact for a held fs
    (r^2 = r0^2 + lambda^2 D_s t), and second-order convergent to the
    quadrature of a linear fs(t) history."""
    D = 3e-9
    r2 = np.array([1e-12])
    for _ in range(100):
        r2 = grain_update(r2, 0.4, 0.4, 1e-3, KP, D)
    assert r2[0] == pytest.approx(1e-12 + grain_lambda(0.4, KP) ** 2 * D * 0.1, rel=1e-13)

    t_end = 0.5

    def fs_of_t(t):
        return 0.05 + 1.8 * t

    exact = D * quad(lambda t: grain_lambda(fs_of_t(t), KP) ** 2, 0.0, t_end, epsabs=0, epsrel=1e-13)[0]
    errs = []
    for n in (50, 100, 200):
        dt = t_end / n
        r2 = np.zeros(1)
        for k in range(n):
            r2 = grain_update(r2, fs_of_t(k * dt), fs_of_t((k + 1) * dt), dt, KP, D)
        errs.append(abs(r2[0] - exact) / exact)
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5 and errs[2] < 1e-4


def test_grains_grow_only_while_mushy():
    """A small cavity cooled on every wall for a few steps: grains stay at r0
    in cells that were never mushy, never shrink, and grow exactly by the
    trapezoidal step of Eq. 24 between the step's solid fractions."""
    m = box_mesh(6, 6, 2, cases.CAVITY)
    grain = dict(kp=KP, D_s=3e-9, r0=1e-6)
    o = Oracle(m, cases.props(walls=cases.all_walls(700.0), T_init=915.0, grain=grain))
    set_state(o, np.full(len(m["cells"]), 915.0))
    r2 = o.r2.copy()
    never = np.ones(len(r2), bool)
    for _ in range(20):
        fs0 = o.fs.copy()
        o.step(2e-3)
        np.testing.assert_allclose(o.r2, grain_update(r2, fs0, o.fs, 2e-3, KP, 3e-9), rtol=1e-15)
        assert np.all(o.r2 >= r2)
        never &= (fs0 <= 0.0) & (o.fs <= 0.0)
        r2 = o.r2.copy()
    assert (~never).any()
    np.testing.assert_allclose(o.grain_radius()[never], 1e-6, rtol=1e-15)
    assert np.all(o.grain_radius()[~never] > 1e-6)
