"""Equation-of-state thermodynamics for the oracle (test infrastructure only).

The fluid of the Enskog-Vlasov model has the pressure
    p(rho, T) = P_E(rho, T) + P_V(rho),   P_V = -a rho^2,
with the Enskog pressure P_E either in the van der Waals form the paper uses,
P_E = rho RT / (1 - b rho), or with the Carnahan-Starling contact value,
P_E = rho RT (1 + eta + eta^2 - eta^3)/(1 - eta)^3, eta = b rho / 4.
(Section "Enskog-Vlasov closure", Eqs. EVforce1 and Ework, and the Vlasov
pressure P_V = -a rho^2 stated beside them.)

Here: the critical point, liquid-vapour coexistence by the Maxwell
construction (equal pressure and equal chemical potential, the line of the
paper's Fig. 1), and the planar square-gradient interface (profile width and
surface tension) that the capillarity coefficient kappa gives.
"""
from __future__ import annotations

import math

import numpy as np

VDW, CS = 0, 1


def Z(eos: int, b: float, rho):
    """Compressibility factor P_E / (rho R T)."""
    rho = np.asarray(rho, dtype=np.float64)
    if eos == VDW:
        return 1.0 / (1.0 - b * rho)
    eta = b * rho / 4.0
    return (1.0 + eta + eta**2 - eta**3) / (1.0 - eta) ** 3


def pressure(eos: int, a: float, b: float, RT: float, rho):
    """p = P_E + P_V = rho RT Z(rho) - a rho^2."""
    rho = np.asarray(rho, dtype=np.float64)
    return rho * RT * Z(eos, b, rho) - a * rho**2


def dp_drho(eos: int, a: float, b: float, RT: float, rho):
    rho = np.asarray(rho, dtype=np.float64)
    if eos == VDW:
        return RT / (1.0 - b * rho) ** 2 - 2.0 * a * rho
    eta = b * rho / 4.0
    return RT * (1 + 4 * eta + 4 * eta**2 - 4 * eta**3 + eta**4) / (1 - eta) ** 4 - 2.0 * a * rho


def chem_potential(eos: int, a: float, b: float, RT: float, rho):
    """mu = d(free energy density)/d rho, up to a T-dependent constant."""
    rho = np.asarray(rho, dtype=np.float64)
    if eos == VDW:
        return RT * (np.log(rho / (1.0 - b * rho)) + b * rho / (1.0 - b * rho)) - 2.0 * a * rho
    eta = b * rho / 4.0
    return RT * (np.log(rho) + (8 * eta - 9 * eta**2 + 3 * eta**3) / (1 - eta) ** 3) - 2.0 * a * rho


def free_energy(eos: int, a: float, b: float, RT: float, rho):
    """Helmholtz free energy density, consistent with chem_potential and pressure
    (p = rho mu - f)."""
    rho = np.asarray(rho, dtype=np.float64)
    if eos == VDW:
        return rho * RT * (np.log(rho / (1.0 - b * rho)) - 1.0) - a * rho**2
    eta = b * rho / 4.0
    return rho * RT * (np.log(rho) - 1.0 + (4 * eta - 3 * eta**2) / (1 - eta) ** 2) - a * rho**2


def critical_point(eos: int, a: float, b: float):
    """(rho_c, RT_c): dp/drho = d2p/drho2 = 0."""
    if eos == VDW:
        return 1.0 / (3.0 * b), 8.0 * a / (27.0 * b)
    # With y(eta) = eta Z(eta): RT y'(eta) = 8 a eta / b and RT y''(eta) = 8 a / b,
    # hence y'(eta_c) = eta_c y''(eta_c).
    def y1(e):
        return (1 + 4 * e + 4 * e**2 - 4 * e**3 + e**4) / (1 - e) ** 4

    def y2(e):
        return (4 + 8 * e - 12 * e**2 + 4 * e**3) / (1 - e) ** 4 + 4 * (1 + 4 * e + 4 * e**2 - 4 * e**3 + e**4) / (1 - e) ** 5

    lo, hi = 0.01, 0.4
    g = lambda e: y1(e) - e * y2(e)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if g(lo) * g(mid) <= 0:
            hi = mid
        else:
            lo = mid
    eta_c = 0.5 * (lo + hi)
    return 4.0 * eta_c / b, 8.0 * a / (b * y2(eta_c))


def spinodal(eos: int, a: float, b: float, RT: float):
    """(rho_s1 < rho_s2) where dp/drho = 0 below the critical temperature."""
    rho_c, _ = critical_point(eos, a, b)
    rmax = (1.0 / b) if eos == VDW else (4.0 / b)

    def root(lo, hi):
        flo = dp_drho(eos, a, b, RT, lo)
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            fm = dp_drho(eos, a, b, RT, mid)
            if flo * fm <= 0:
                hi = mid
            else:
                lo, flo = mid, fm
        return 0.5 * (lo + hi)

    return root(1e-9 * rho_c, rho_c), root(rho_c, rmax * (1 - 1e-9))


def maxwell(eos: int, a: float, b: float, RT: float, tol: float = 1e-14):
    """Coexisting (rho_v, rho_l) at temperature RT < RT_c by Newton iteration on
    p(rho_v) = p(rho_l) and mu(rho_v) = mu(rho_l)."""
    s1, s2 = spinodal(eos, a, b, RT)
    # Initial guess: a bracketing bisection on the pressure level.
    def densities_at(P):
        # vapour root in (0, s1), liquid root in (s2, rmax)
        def bis(lo, hi, up):
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                val = pressure(eos, a, b, RT, mid) - P
                if (val > 0) == up:
                    hi = mid
                else:
                    lo = mid
            return 0.5 * (lo + hi)

        rmax = (1.0 / b) if eos == VDW else (4.0 / b)
        rv = bis(1e-12, s1, True)
        rl = bis(s2, rmax * (1 - 1e-12), True)
        return rv, rl

    Plo = max(pressure(eos, a, b, RT, s2), 1e-300)
    Phi = pressure(eos, a, b, RT, s1)
    for _ in range(200):          # bisection on the pressure level: equal mu
        P = 0.5 * (Plo + Phi)
        rv, rl = densities_at(P)
        d = chem_potential(eos, a, b, RT, rl) - chem_potential(eos, a, b, RT, rv)
        if d < 0:             # liquid more stable: pressure above saturation
            Phi = P
        else:
            Plo = P
        if Phi - Plo < 1e-15 * abs(Phi):
            break
    rv, rl = densities_at(0.5 * (Plo + Phi))
    for _ in range(50):           # Newton polish
        F1 = pressure(eos, a, b, RT, rl) - pressure(eos, a, b, RT, rv)
        F2 = chem_potential(eos, a, b, RT, rl) - chem_potential(eos, a, b, RT, rv)
        pl, pv = dp_drho(eos, a, b, RT, rl), dp_drho(eos, a, b, RT, rv)
        J = np.array([[-pv, pl], [-pv / rv, pl / rl]])
        dx = np.linalg.solve(J, -np.array([F1, F2]))
        rv, rl = rv + dx[0], rl + dx[1]
        if abs(dx[0]) < tol * rv and abs(dx[1]) < tol * rl:
            break
    return float(rv), float(rl)


def equal_area_residual(eos: int, a: float, b: float, RT: float, rv: float, rl: float, n: int = 20001):
    """(1/(v_v - v_l)) int_{v_l}^{v_v} p dv - p_sat, v = 1/rho, by Simpson quadrature.
    Zero at the Maxwell construction."""
    v = np.linspace(1.0 / rl, 1.0 / rv, n)
    pv = pressure(eos, a, b, RT, 1.0 / v)
    h = v[1] - v[0]
    integral = h / 3.0 * (pv[0] + pv[-1] + 4.0 * pv[1:-1:2].sum() + 2.0 * pv[2:-1:2].sum())
    psat = float(pressure(eos, a, b, RT, rl))
    return integral / (v[-1] - v[0]) - psat


def grand_excess(eos: int, a: float, b: float, RT: float, rho, rv: float, rl: float):
    """omega(rho) = f(rho) - mu_sat rho + p_sat >= 0 between the coexisting densities."""
    mu = float(chem_potential(eos, a, b, RT, rv))
    ps = float(pressure(eos, a, b, RT, rv))
    return free_energy(eos, a, b, RT, rho) - mu * np.asarray(rho) + ps


def interface(eos: int, a: float, b: float, RT: float, kappa: float, n: int = 200001):
    """Planar square-gradient interface: kappa/2 (d rho/dx)^2 = omega(rho).
    Returns (width_10_90, sigma) with sigma = int sqrt(2 kappa omega) d rho."""
    rv, rl = maxwell(eos, a, b, RT)
    rho = np.linspace(rv, rl, n)[1:-1]
    om = np.maximum(grand_excess(eos, a, b, RT, rho, rv, rl), 0.0)
    grad = np.sqrt(2.0 * om / kappa)                    # |d rho / dx|
    sigma = float(np.trapezoid(kappa * grad, rho))
    r10 = rv + 0.1 * (rl - rv)
    r90 = rv + 0.9 * (rl - rv)
    m = (rho >= r10) & (rho <= r90)
    width = float(np.trapezoid(1.0 / grad[m], rho[m]))
    return width, sigma


def kappa_for_width(eos: int, a: float, b: float, RT: float, width: float = 4.0):
    """kappa giving a 10-90 % interface width `width` (width scales as sqrt(kappa))."""
    w1, _ = interface(eos, a, b, RT, 1.0)
    return (width / w1) ** 2
