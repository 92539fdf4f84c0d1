"""Pins of the oracle's thermal-field emission (Sec. 2.3.1) against classical limits:
Murphy-Good Fowler-Nordheim (cold, moderate field), Richardson-Dushman-Schottky (hot, low
field), the Forbes approximation of the Schottky-Nordheim barrier function, the Nottingham
inversion, and the flat-surface limit of the curved barrier."""
import math

import numpy as np
import pytest

from oracle import constants as C
from oracle import emission as em

PHI = 4.5


def murphy_good(F, phi):
    """Murphy-Good FN current density [A/m^2] with Forbes' v(f), t(f) (first FN constants
    a = 1.541434e-6 A eV V^-2, b = 6.830890 eV^-3/2 V nm^-1; F in V/nm)."""
    a, b = 1.541434e-6, 6.830890
    f = 1.439964 * F / phi ** 2
    v = 1 - f + f / 6 * math.log(f)
    t = 1 + f / 9 - f / 18 * math.log(f)
    return a * F * F / (phi * t * t) * math.exp(-v * b * phi ** 1.5 / F) * 1e18


def richardson_schottky(F, T, phi):
    A_R = 4 * math.pi * C.M_E * C.E_CHARGE * C.K_B ** 2 / (2 * math.pi * C.HBAR) ** 3
    dphi = math.sqrt(C.E_CHARGE * F * 1e9 / (4 * math.pi * C.EPS0))     # Schottky lowering [eV]
    return A_R * T * T * math.exp(-(phi - dphi) / (C.K_B_EV * T))


@pytest.mark.slow
@pytest.mark.parametrize("F", [3.0, 4.0, 5.0])
def test_cold_field_emission_matches_murphy_good(F):
    J, PN = em.current_density_quad(F, 30.0, PHI, math.inf)
    assert abs(math.log10(J) - math.log10(murphy_good(F, PHI))) < 0.02
    assert PN > 0          # cold emission heats the surface (electrons leave below E_F)


@pytest.mark.slow
@pytest.mark.parametrize("T", [2500.0, 3000.0])
def test_thermionic_limit_matches_richardson_schottky(T):
    F = 0.1
    J, PN = em.current_density_quad(F, T, PHI, math.inf)
    rd = richardson_schottky(F, T, PHI)
    assert J >= rd * 0.999                       # tunnelling below the top only adds current
    assert math.log10(J) - math.log10(rd) < 0.05
    assert PN < 0          # hot emission cools the surface


def test_gamow_exponent_at_fermi_level_matches_forbes_v():
    # G(E_F) = b phi^{3/2} v(f) / F for the Schottky-Nordheim barrier (v to 0.33 % by Forbes)
    b = 6.830890
    for F in (2.0, 5.0, 8.0, 11.0):
        xm, Um = em.barrier_max(F, PHI, math.inf)
        G = em.gamow(0.0, F, PHI, math.inf, xm)
        f = 1.439964 * F / PHI ** 2
        v = 1 - f + f / 6 * math.log(f)
        assert G == pytest.approx(b * PHI ** 1.5 * v / F, rel=0.004)
        # SN barrier: top at phi - sqrt(4 Q F) reached at x = sqrt(Q/F)
        assert xm == pytest.approx(math.sqrt(C.Q_IMAGE_EVNM / F), rel=1e-10)
        assert Um == pytest.approx(PHI - math.sqrt(4 * C.Q_IMAGE_EVNM * F), rel=1e-12)


def test_nottingham_inner_closed_form_matches_definition():
    # relative agreement everywhere, including far above E_F where I(W) ~ -(kT)^2 (w+1) e^-w
    for kT in (0.02585, 0.3):
        for W in (-6.0, -1.0, -0.05, 0.0, 0.02, 0.7, 3.0, 6.0):
            assert em.nottingham_inner(W, kT) == pytest.approx(em.nottingham_inner_quad(W, kT), rel=1e-9)
    w = 60.0
    assert em._L(np.array([w]))[0] == pytest.approx(math.exp(-w) * (1 - math.exp(-w) / 4), rel=1e-12)


@pytest.mark.slow
def test_flat_limit_and_monotonicity():
    J_inf, _ = em.current_density_quad(8.0, 300.0, PHI, math.inf)
    J_big, _ = em.current_density_quad(8.0, 300.0, PHI, 1e6)
    assert J_big == pytest.approx(J_inf, rel=1e-5)
    J_small, _ = em.current_density_quad(8.0, 300.0, PHI, 5.0)
    assert J_small < J_inf                  # the curved barrier is wider at the same surface field
    Js = [em.current_density_quad(F, 1500.0, PHI, 10.0)[0] for F in (4.0, 6.0, 8.0)]
    assert Js[0] < Js[1] < Js[2]
    JT = [em.current_density_quad(6.0, T, PHI, 10.0)[0] for T in (500.0, 1500.0, 2500.0)]
    assert JT[0] < JT[1] < JT[2]


@pytest.mark.slow
def test_fixed_rule_matches_adaptive_quadrature():
    cases = [(8.0, 300.0, 4.5, math.inf), (10.0, 2000.0, 4.3, 5.0), (2.0, 3500.0, 4.8, 3.0),
             (13.0, 800.0, 4.1, 15.0), (1.2, 4000.0, 4.9, 1.0), (0.0609, 3300.0, 4.5, 2.0),
             (0.17, 3300.0, 4.5, 2.0), (1.955, 614.0, 4.37, 2.67), (0.1, 3000.0, 4.5, math.inf)]
    F, T, W, R = (np.array(c) for c in zip(*cases))
    J, PN = em.current_density_fixed(F, T, W, R)
    for r, c in enumerate(cases):
        Jq, Pq = em.current_density_quad(*c)
        assert J[r] == pytest.approx(Jq, rel=1e-7)
        assert PN[r] == pytest.approx(Pq, rel=1e-6, abs=1e-9 * abs(Jq))


def test_no_emission_without_pulling_field():
    assert em.current_density_quad(0.0, 300.0, PHI, 5.0) == (0.0, 0.0)
    J, P = em.current_density_fixed(np.array([-1.0, 0.0]), 300.0, PHI, np.array([5.0, np.inf]))
    assert np.all(J == 0) and np.all(P == 0)
