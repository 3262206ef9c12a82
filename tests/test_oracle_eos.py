"""Pins of the oracle's equation of state (Enskog-Vlasov closure and Eq. gamma).

Each check compares against something other than the oracle's own formula:
an independent quadrature, a textbook limit, finite differences of a
definition, or the virial series of hard spheres.
"""
import math

import numpy as np
import pytest

import oracle
import oracle.eos as E

CASES = [(E.CS, 1.0, 4.0), (E.CS, 0.1, 4.0), (E.VDW, 9 / 392, 2 / 21)]


@pytest.mark.parametrize("eos,a,b", CASES)
def test_critical_point_is_inflection(eos, a, b):
    """dp/drho = d2p/drho2 = 0 at (rho_c, RT_c), by central differences of p."""
    rc, Tc = E.critical_point(eos, a, b)
    h = 1e-4 * rc
    p = lambda r: float(E.pressure(eos, a, b, Tc, r))
    d1 = (p(rc + h) - p(rc - h)) / (2 * h)
    d2 = (p(rc + h) - 2 * p(rc) + p(rc - h)) / h**2
    scale = Tc  # dp/drho ~ RT
    assert abs(d1) < 1e-7 * scale
    assert abs(d2) * rc < 1e-5 * scale


def test_vdw_critical_point_closed_form():
    """van der Waals: rho_c = 1/(3b), RT_c = 8a/(27b)."""
    rc, Tc = E.critical_point(E.VDW, 9 / 392, 2 / 21)
    assert rc == pytest.approx(3.5, rel=1e-15)
    assert Tc == pytest.approx(1 / 14, rel=1e-14)


@pytest.mark.parametrize("eos,a,b", CASES)
@pytest.mark.parametrize("tr", [0.7, 0.8, 0.85, 0.9, 0.97])
def test_maxwell_equal_area(eos, a, b, tr):
    """Newton's coexistence satisfies the equal-area rule int p dv = p_sat (v_v - v_l),
    evaluated by an independent Simpson quadrature, and equal pressures."""
    rc, Tc = E.critical_point(eos, a, b)
    rv, rl = E.maxwell(eos, a, b, tr * Tc)
    assert rv < rc < rl
    psat = float(E.pressure(eos, a, b, tr * Tc, rl))
    assert float(E.pressure(eos, a, b, tr * Tc, rv)) == pytest.approx(psat, rel=1e-10, abs=1e-16)
    resid = E.equal_area_residual(eos, a, b, tr * Tc, rv, rl)
    assert abs(resid) < 1e-9 * max(abs(psat), tr * Tc * rc * 1e-3)


def test_vdw_near_critical_scaling():
    """van der Waals close to T_c: (rho_l - rho_v)/rho_c -> 4 sqrt(1 - T/T_c)."""
    a, b = 9 / 392, 2 / 21
    rc, Tc = E.critical_point(E.VDW, a, b)
    for eps in (1e-3, 1e-4):
        rv, rl = E.maxwell(E.VDW, a, b, (1 - eps) * Tc)
        ratio = (rl - rv) / rc / (4 * math.sqrt(eps))
        assert ratio == pytest.approx(1.0, abs=2 * math.sqrt(eps))


def test_cs_virial_series():
    """Carnahan-Starling Z(eta) = 1 + 4 eta + 10 eta^2 + 18 eta^3 + ... (hard-sphere
    virial series), read through the oracle's P0/(rho RT)."""
    b = 4.0
    etas = np.linspace(1e-4, 2e-3, 12)
    Z = np.array([oracle.eos_state(E.CS, b, eta * 4 / b, 1.0)[1] for eta in etas])  # theta0 / RT
    coef = np.polyfit(etas, Z - 1.0, 3)[::-1]
    assert coef[0] == pytest.approx(0.0, abs=1e-9)
    assert coef[1] == pytest.approx(4.0, rel=1e-6)
    assert coef[2] == pytest.approx(10.0, rel=1e-3)


def test_vdw_form_is_papers():
    """P_E = rho RT/(1 - b rho), the form of the Enskog pressure the paper writes."""
    b, rho, RT = 0.1, 3.0, 0.07
    P0, th, _ = oracle.eos_state(E.VDW, b, rho, RT)
    assert P0 == pytest.approx(rho * RT / (1 - b * rho), rel=1e-15)
    assert th == pytest.approx(P0 / rho, rel=1e-15)


@pytest.mark.parametrize("eos,b,rho", [(E.CS, 4.0, 0.03), (E.CS, 4.0, 0.3), (E.VDW, 2 / 21, 1.0),
                                       (E.VDW, 2 / 21, 6.5)])
def test_gamma0_from_definition(eos, b, rho):
    """gamma0 = (dlnP0/dlnrho)_T + 2/3 (P_E/(rho RT)) (dlnP0/dlnT)_rho  (Eq. gamma),
    evaluated by central differences of the oracle's P0(rho, T) with P0 = P_E."""
    RT = 0.05
    h = 1e-5
    lnP = lambda r, t: math.log(oracle.eos_state(eos, b, r, t)[0])
    dlr = (lnP(rho * math.exp(h), RT) - lnP(rho * math.exp(-h), RT)) / (2 * h)
    dlt = (lnP(rho, RT * math.exp(h)) - lnP(rho, RT * math.exp(-h))) / (2 * h)
    PE, _, g0 = oracle.eos_state(eos, b, rho, RT, thermal=1)
    assert g0 == pytest.approx(dlr + 2 / 3 * PE / (rho * RT) * dlt, rel=1e-8)
    # Temperature frozen: only the isothermal part remains.
    assert oracle.eos_state(eos, b, rho, RT, thermal=0)[2] == pytest.approx(dlr, rel=1e-8)


def test_ideal_gas_gamma():
    """b = 0: Z = 1 and gamma0 = 5/3 (monatomic ideal gas), so Phi' vanishes."""
    for eos in (E.VDW, E.CS):
        P0, th, g0 = oracle.eos_state(eos, 0.0, 1.3, 0.2)
        assert th == pytest.approx(0.2, rel=1e-15)
        assert g0 == pytest.approx(5 / 3, rel=1e-15)


def test_interface_width_and_tension_scale():
    """Square-gradient interface: width ~ sqrt(kappa), sigma ~ sqrt(kappa)."""
    eos, a, b = E.CS, 1.0, 4.0
    _, Tc = E.critical_point(eos, a, b)
    w1, s1 = E.interface(eos, a, b, 0.8 * Tc, 1.0)
    w4, s4 = E.interface(eos, a, b, 0.8 * Tc, 4.0)
    assert w4 / w1 == pytest.approx(2.0, rel=1e-6)
    assert s4 / s1 == pytest.approx(2.0, rel=1e-6)


@pytest.mark.parametrize("eos,a,b", CASES)
def test_free_energy_chemical_potential_and_pressure_are_consistent(eos, a, b):
    """Helmholtz free-energy density f(rho) at fixed T: mu = df/drho and dp/drho =
    rho dmu/drho (central differences), and the Euler relation p = rho mu - f; checked
    over vapour, spinodal and liquid densities at T/Tc = 0.8."""
    rc, Tc = E.critical_point(eos, a, b)
    RT = 0.8 * Tc
    for rho in (0.05 * rc, 0.5 * rc, rc, 1.8 * rc, 2.4 * rc):
        h = 1e-5 * rho
        f = lambda r: float(E.free_energy(eos, a, b, RT, r))
        mu = lambda r: float(E.chem_potential(eos, a, b, RT, r))
        p = float(E.pressure(eos, a, b, RT, rho))
        assert (f(rho + h) - f(rho - h)) / (2 * h) == pytest.approx(mu(rho), rel=1e-8, abs=1e-10 * RT)
        assert rho * (mu(rho + h) - mu(rho - h)) / (2 * h) == pytest.approx(
            float(E.dp_drho(eos, a, b, RT, rho)), rel=1e-6, abs=1e-9 * RT)
        assert rho * mu(rho) - f(rho) == pytest.approx(p, rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("eos,a,b", CASES)
def test_grand_excess_vanishes_at_coexistence_and_is_positive_between(eos, a, b):
    _, Tc = E.critical_point(eos, a, b)
    RT = 0.8 * Tc
    rv, rl = E.maxwell(eos, a, b, RT)
    om = E.grand_excess(eos, a, b, RT, np.array([rv, rl]), rv, rl)
    scale = float(E.pressure(eos, a, b, RT, rl))
    assert np.all(np.abs(om) <= 1e-10 * max(scale, RT * rl))
    mid = np.linspace(rv, rl, 101)[1:-1]
    assert np.all(E.grand_excess(eos, a, b, RT, mid, rv, rl) > 0)


def test_interface_on_a_quartic_well_matches_the_tanh_closed_forms(monkeypatch):
    """Square-gradient theory on a double well omega = A (rho - rv)^2 (rl - rho)^2 has the
    profile rho = mid + (rl - rv)/2 tanh(x / xi), xi = sqrt(2 kappa / A) / (rl - rv), so
    the 10-90 % width is 2 xi artanh(0.8) and sigma = (rl - rv)^3 sqrt(2 kappa A) / 6.
    The oracle's interface() is run with its coexistence and excess grand potential
    replaced by this well, and must reproduce both closed forms."""
    rv, rl, A, kappa = 0.2, 1.4, 3.0, 0.7
    monkeypatch.setattr(E, "maxwell", lambda *args, **kw: (rv, rl))
    monkeypatch.setattr(E, "grand_excess",
                        lambda eos, a, b, RT, rho, v, l: A * (np.asarray(rho) - v) ** 2 * (l - np.asarray(rho)) ** 2)
    width, sigma = E.interface(E.CS, 0.1, 4.0, 0.01, kappa)
    xi = np.sqrt(2.0 * kappa / A) / (rl - rv)
    assert width == pytest.approx(2.0 * xi * np.arctanh(0.8), rel=2e-5)
    assert sigma == pytest.approx((rl - rv) ** 3 * np.sqrt(2.0 * kappa * A) / 6.0, rel=1e-8)
