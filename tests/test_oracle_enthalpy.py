"""Pins of the oracle's enthalpy relation (Eqs. 5 and 11).

E(T) = C T + Lc f_l(T) with a linear liquid fraction between solidus and
liquidus; T(E) is its exact inverse.  Checked at, between and beyond the
breakpoints, in the isothermal limit, for monotonicity and continuity.
"""
import numpy as np
import pytest

import oracle

C, LC, TS, TL = 262.5, 1.1375e5, 821.0, 913.0


def test_breakpoint_values():
    assert oracle.E_from_T(TS, C, LC, TS, TL) == pytest.approx(C * TS, rel=1e-15)
    assert oracle.E_from_T(TL, C, LC, TS, TL) == pytest.approx(C * TL + LC, rel=1e-15)
    mid = 0.5 * (TS + TL)
    assert oracle.E_from_T(mid, C, LC, TS, TL) == pytest.approx(C * mid + 0.5 * LC, rel=1e-15)
    assert oracle.liquid_fraction(TS - 1, TS, TL) == 0.0
    assert oracle.liquid_fraction(TL + 1, TS, TL) == 1.0
    assert oracle.liquid_fraction(TS + 0.25 * (TL - TS), TS, TL) == pytest.approx(0.25)


@pytest.mark.parametrize("T", [250.0, 600.0, TS, TS + 1e-9, 850.0, 900.0, TL - 1e-9,
                               TL, 950.0, 1400.0])
def test_round_trip(T):
    E = oracle.E_from_T(T, C, LC, TS, TL)
    assert oracle.T_from_E(E, C, LC, TS, TL) == pytest.approx(T, abs=1e-10)


def test_monotone_and_continuous():
    T = np.linspace(300, 1200, 20001)
    E = np.array([oracle.E_from_T(t, C, LC, TS, TL) for t in T])
    assert (np.diff(E) > 0).all()
    # the slope is C outside and C + Lc/(Tl-Ts) inside the mushy range
    dE = np.diff(E) / np.diff(T)
    mushy = (T[:-1] > TS + 0.1) & (T[1:] < TL - 0.1)
    np.testing.assert_allclose(dE[mushy], C + LC / (TL - TS), rtol=1e-6)
    solid = T[1:] < TS - 0.1
    np.testing.assert_allclose(dE[solid], C, rtol=1e-6)
    Eg = np.linspace(E[0], E[-1], 5001)
    Tg = np.array([oracle.T_from_E(e, C, LC, TS, TL) for e in Eg])
    assert (np.diff(Tg) >= 0).all()
    assert np.abs(np.diff(Tg)).max() < 1.0   # no jumps


def test_isothermal_limit():
    Tm = 933.0
    # enthalpy inside the latent plateau maps to the melting point
    for frac in (0.0, 0.1, 0.5, 0.9):
        E = C * Tm + frac * LC
        assert oracle.T_from_E(E, C, LC, Tm, Tm) == (Tm if frac > 0 else pytest.approx(Tm))
    assert oracle.T_from_E(C * 500.0, C, LC, Tm, Tm) == pytest.approx(500.0)
    assert oracle.T_from_E(C * 1000.0 + LC, C, LC, Tm, Tm) == pytest.approx(1000.0)
    assert oracle.E_from_T(1000.0, C, LC, Tm, Tm) == pytest.approx(C * 1000.0 + LC)
    assert oracle.E_from_T(500.0, C, LC, Tm, Tm) == pytest.approx(C * 500.0)


def test_no_phase_change():
    assert oracle.T_from_E(C * 777.0, C, 0.0, 0.0, 0.0) == pytest.approx(777.0)
    assert oracle.E_from_T(777.0, C, 0.0, 0.0, 0.0) == pytest.approx(C * 777.0)
