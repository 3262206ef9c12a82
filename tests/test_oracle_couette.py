"""The supersonic thermal Couette flow of the paper's validation (the channel between a
static and a moving wall, u = 0, T = T_w at x = 0 and u = (0, U_w), T = T_w at x = L_x,
Ma = 1.2 at the moving wall; the paper's Fig. 2) on the oracle, against the steady
solution of the Navier-Stokes-Fourier equations the model recovers (Eqs. momentum_balance,
LB_energy_balance with mu = tau P0 (Eq. viscosity) and k = 5/2 R mu).

The paper does not state its wall scheme; the oracle reads it as diffusely reflecting
wall nodes (oracle/evlbm_oracle.c, "Walls"): the columns x = 0 and x = nx - 1 absorb the
populations that stream into them and re-emit the wall equilibrium with the same mass.

Steady solution (derived here; the paper prints none).  With u_x = 0 the x-momentum
balance makes p = P_E - a rho^2 uniform; the shear stress S = mu u_y' and the total
energy flux -k T' - mu u_y u_y' are uniform.  With k = 5/2 R mu the two combine to
    T(u_y) = T_w + u_y (U_w - u_y) / (5 R),
whatever the variation of mu = tau P_E(rho, T) across the channel, and then
    x(u_y) = L int_0^{u_y} mu du / int_0^{U_w} mu du,
with rho(u_y) from p(rho, T(u_y)) = p.  For an ideal gas (a = b = 0) mu is uniform:
u_y = U_w x/L and T = T_w + U_w^2/(5R) (x/L)(1 - x/L).

Pins: every fluid node's u_y within 1e-3 U_w of x(u_y), rho within 1e-3, T within 1 % of
the viscous heating U_w^2/(20 R) of T(u_y); p uniform within 1e-3; the fluid mass plus
the mass in transit into the walls (returned by them one step later) constant to rounding
once the walls have emitted their first populations; the Mach number at the moving wall
above 1.  Van der Waals and Carnahan-Starling dense gases and an ideal gas.  A viscous heating or heat
conduction that were off by a factor (e.g. the energy populations relaxing the heat flux
at another rate, or a wall that leaks mass) moves T(u_y) by far more than 1 %: with an
equilibrium wall at the density of the adjacent node instead of the mass-conserving one,
the channel loses 3 % of its mass every 20000 steps and T'' falls to 0.6 of -2/5 u_y'^2.
"""
import math

import numpy as np
import pytest

import oracle
import oracle.eos as E

scipy_optimize = pytest.importorskip("scipy.optimize")

NX, TAU, RTW, MA, STEPS = 66, 0.5, 0.2, 1.2, 100000


def fluid_mass(o):
    """Mass of the fluid nodes plus the mass streaming into the wall nodes at the next step
    (the post-collision populations of the nodes next to the walls that move toward them),
    which the walls return one step later."""
    c, _ = oracle.lattice(9)
    f = o.f.reshape(9, NX)
    return o.macro()[0][1:-1].sum() + f[c[:, 0] == -1, 1].sum() + f[c[:, 0] == 1, NX - 2].sum()


def couette(eos, b, a, rho0=1.0):
    """Steady Couette flow of the fluid (eos, b, a) from rest at rho0, T_w."""
    P0, _, g0 = oracle.eos_state(eos, b, rho0, RTW)
    c = math.sqrt(g0 * P0 / rho0 - 2 * a * rho0)          # adiabatic sound speed of p = P_E - a rho^2
    Uw = MA * c
    p = oracle.Params(Q=9, nx=NX, ny=1, eos=eos, a=a, b=b, kappa=0.0, tau=TAU, thermal=1,
                      walls=((0, 0, 0), (0, Uw, 0), RTW))
    u = np.zeros((2, NX))
    u[1, -1] = Uw
    o = oracle.State(p, np.full(NX, rho0), u, np.full(NX, RTW))
    o.step(1)
    m1 = fluid_mass(o)
    o.step(STEPS - 1)
    rho, uu, T, _ = o.macro()
    return Uw, rho, uu[1], T, m1, fluid_mass(o)


def steady_solution(eos, b, a, Uw, pbar):
    """(u_y, rho) at the nodes x = 0..NX-1 from the quadrature of the steady equations."""
    Tof = lambda v: RTW + v * (Uw - v) / 5.0
    rmax = 1e3 if b == 0 else (0.999 / b if eos == E.VDW else 3.0 / b)
    rho_of = lambda v: scipy_optimize.brentq(lambda x: E.pressure(eos, a, b, Tof(v), x) - pbar, 1e-9, rmax)
    vs = np.linspace(0.0, Uw, 4001)
    mu = np.array([TAU * float(E.pressure(eos, 0.0, b, Tof(v), rho_of(v))) for v in vs])      # tau P_E
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (mu[1:] + mu[:-1]) * np.diff(vs))])
    u_an = np.interp(np.arange(NX), (NX - 1) * cum / cum[-1], vs)
    return u_an, np.array([rho_of(v) for v in u_an]), Tof


@pytest.mark.parametrize("eos,b,a", [(E.VDW, 0.1, 0.05), (E.CS, 0.2, 0.05), (E.VDW, 0.0, 0.0)])
def test_supersonic_thermal_couette(eos, b, a):
    Uw, rho, uy, T, m1, m2 = couette(eos, b, a)
    fl = slice(1, NX - 1)
    assert np.isfinite(rho).all() and np.isfinite(T).all()
    assert abs(m2 / m1 - 1.0) < 1e-12                                 # mass-conserving walls
    pr = E.pressure(eos, a, b, T, rho)
    pbar = float(pr[fl].mean())
    assert (pr[fl].max() - pr[fl].min()) / pbar < 1e-3                # uniform pressure
    u_an, rho_an, Tof = steady_solution(eos, b, a, Uw, pbar)
    assert np.abs(uy - u_an)[fl].max() < 1e-3 * Uw
    assert (np.abs(rho - rho_an) / rho_an)[fl].max() < 1e-3
    heat = Uw**2 / 20.0                                               # T(U_w/2) - T_w
    assert np.abs(T - Tof(uy))[fl].max() < 0.01 * heat
    assert T[NX // 2] - RTW == pytest.approx(heat, rel=0.02)
    # supersonic at the moving wall: Mach number of the fluid next to it
    n = NX - 2
    P0, _, g0 = oracle.eos_state(eos, b, rho[n], T[n])
    assert uy[n] / math.sqrt(g0 * P0 / rho[n] - 2 * a * rho[n]) > 1.1
    if a == 0.0 and b == 0.0:
        # ideal gas: the closed form
        x = np.arange(NX) / (NX - 1)
        assert np.abs(uy - Uw * x)[fl].max() < 1e-3 * Uw
        assert np.abs(T - (RTW + Uw**2 / 5.0 * x * (1 - x)))[fl].max() < 0.01 * heat
