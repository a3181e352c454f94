"""Pins of the smeared Gulliver-Scheil solid fraction (Eq. 5, Eq. 21) and of
the energy step that uses it (Section 2.4.4).  CPU only."""
import numpy as np
import pytest

from fvs_inputs import box_mesh, cases
from oracle.fv import Oracle, scheil_law, solid_fraction, solid_fraction_slope, temperature_from_enthalpy
from tests.helpers import set_state

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

MAT = cases.AL_SI_SCHEIL
LAW = scheil_law(MAT)
TS, TL = MAT["T_sol"], MAT["T_liq"]
KP, TF, TE = LAW


def fs(T):
    return solid_fraction(T, TS, TL, LAW)


def test_scheil_from_solute_balance():
    """Gulliver-Scheil from the solute balance: with no diffusion in the
    solid the liquid holds C_l = C0 (1 - fs)^(kp - 1) (the relation the paper
    uses for grain growth), and on a straight liquidus T = T_f + m_l C_l with
    T_liq = T_f + m_l C0.  Reading fs back off the temperature that a given
    fs produces must return it (outside the smear band)."""
    C0 = 7.0
    m_l = (TL - TF) / C0
    for f in (0.0, 0.05, 0.3, 0.6, 0.8):
        C_l = C0 * (1.0 - f) ** (KP - 1.0)
        T = TF + m_l * C_l
        assert T >= TS + TE
        assert float(fs(T)) == pytest.approx(f, abs=1e-13)


def test_smear_band_and_limits():
    """Eq. 21: 0 above the liquidus, 1 below T_sol - T_eps, a straight line
    across [T_sol - T_eps, T_sol + T_eps] meeting the Scheil curve, and
    monotone in between; continuous at every kink."""
    T2 = TS + TE
    assert float(fs(TL + 1e-9)) == 0.0 and float(fs(TL)) == pytest.approx(0.0, abs=1e-15)
    assert float(fs(TS - TE)) == 1.0 and float(fs(700.0)) == 1.0
    for k in (TS - TE, TS + TE, TL):
        assert abs(float(fs(k - 1e-9)) - float(fs(k + 1e-9))) < 1e-9
    # straight line across the band: its midpoint is the mean of its ends
    assert float(fs(TS)) == pytest.approx(0.5 * (1.0 + float(fs(T2))), abs=1e-13)
    T = np.linspace(700.0, 1000.0, 30001)
    f = fs(T)
    assert f.min() >= 0.0 and f.max() <= 1.0
    assert np.all(np.diff(f) <= 1e-15)
    # the Scheil curve leaves a large jump at the solidus that the band closes
    assert 0.6 < float(fs(T2)) < 0.95


@pytest.mark.parametrize("law", [None, LAW])
def test_slope_is_the_derivative(law):
    """dfs/dT equals a central difference away from the kinks and the
    one-sided difference on the mushy-interior side at each kink."""
    T = np.concatenate([np.linspace(700.0, 1000.0, 3001)])
    kinks = [TL, TS - TE, TS + TE] if law else [TL, TS]
    T = T[np.min(np.abs(T[:, None] - np.array(kinks)[None, :]), axis=1) > 1e-3]
    h = 1e-5
    num = (solid_fraction(T + h, TS, TL, law) - solid_fraction(T - h, TS, TL, law)) / (2 * h)
    np.testing.assert_allclose(solid_fraction_slope(T, TS, TL, law), num, rtol=1e-6, atol=1e-9)
    # kinks: the side towards the mushy interior
    for k, side in ((TL, -1.0), (TS - TE, 1.0), (TS + TE, 1.0)) if law else ((TL, -1.0), (TS, 1.0)):
        one = (solid_fraction(k + side * h, TS, TL, law) - solid_fraction(k, TS, TL, law)) / (side * h)
        assert float(solid_fraction_slope(k, TS, TL, law)) == pytest.approx(float(one), rel=1e-4)


@pytest.mark.parametrize("law", [None, LAW])
def test_enthalpy_inversion_round_trip(law):
    """T -> H = cp T + L (1 - fs(T)) -> T across every piece of the law."""
    cp, L = MAT["cp"], MAT["latent"]
    T = np.concatenate([np.linspace(780.0, 980.0, 2001), [TS - TE, TS, TS + TE, TL]])
    H = cp * T + L * (1.0 - solid_fraction(T, TS, TL, law))
    np.testing.assert_allclose(temperature_from_enthalpy(H, cp, L, TS, TL, law), T, rtol=0, atol=1e-9)


@pytest.mark.parametrize("T0", [960.0, 912.0, 880.0, 840.0, 834.0])
def test_energy_single_cell_scheil(T0):
    """One cube with one fixed-temperature face: a step's energy equation is
    the scalar equation
    rho cp V (T - T0)/dt = k h (T_w - T) + k h (T_w - T0) + rho L V (fs(T) - fs(T0))/dt,
    increasing in T; its root found by bisection must be where the oracle's
    latent-heat loop lands."""
    h = 0.01
    m = box_mesh(1, 1, 1, (h, h, h))
    Tw = 700.0
    o = Oracle(m, cases.props(material=MAT, walls=[(1, Tw)] + [(0, 0.0)] * 5, oracle_tol_T=1e-12))
    set_state(o, [T0])
    dt = 0.05
    o.step(dt)
    rho, cp, k, L = MAT["rho"], MAT["cp"], MAT["k"], MAT["latent"]
    V = h ** 3
    f0 = float(fs(T0))

    def R(T):
        return (rho * cp * V * (T - T0) / dt - k * h * (Tw - T) - k * h * (Tw - T0)
                - rho * L * V * (float(fs(T)) - f0) / dt)

    lo, hi = 600.0, 1000.0
    assert R(lo) < 0 < R(hi)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if R(mid) < 0:
            lo = mid
        else:
            hi = mid
    assert o.T[0] == pytest.approx(0.5 * (lo + hi), abs=1e-9)
    assert o.fs[0] == pytest.approx(float(fs(o.T[0])), abs=1e-14)


def test_scheil_freezes_early_and_leaves_a_remainder_at_the_solidus():
    """Scheil with a small partition coefficient freezes most of the metal
    just below the liquidus (fs above the linear law's at the same
    temperature) and leaves a liquid remainder that the smear band freezes
    at the solidus; below the band both laws are fully solid."""
    T = np.array([890.0, 870.0, 850.0, 830.0])
    lin = solid_fraction(T, TS, TL)
    sch = fs(T)
    assert np.all(sch[:3] > lin[:3])
    assert sch[3] == lin[3] == 1.0
    assert float(fs(TL - 30.0)) > 0.5
    assert 1.0 - float(fs(TS + TE)) > 0.1
