"""Pins of the oracle's time step (Eq. pre_LBM with Eqs. beta, u_shift, T_shift,
EVforce1, P0E, feq, f_star, correction_u/gamma/q, geq, gstar, g_corr).

The checks reduce the step to textbook cases (plain BGK, Navier-Stokes-Fourier
acoustics), invariants (conservation), an exact lattice identity (D2Q9 is the
c_z-marginal of D3Q27) and analytic derivatives (force stencils).
"""
import math

import numpy as np
import pytest

import oracle
import oracle.eos as E
from paper_2508_00577_gb300 import inputs

CS_A, CS_B = 0.1, 4.0


def cs_state(tr):
    rc, Tc = E.critical_point(E.CS, CS_A, CS_B)
    RT = tr * Tc
    rv, rl = E.maxwell(E.CS, CS_A, CS_B, RT)
    kappa = E.kappa_for_width(E.CS, CS_A, CS_B, RT, 4.0)
    return RT, rv, rl, kappa


def droplet_oracle(nx=48, ny=40, tr=0.8, thermal=1, force_form=0, tau=0.3, Q=9, nz=1):
    RT, rv, rl, kappa = cs_state(tr)
    p = oracle.Params(Q=Q, nx=nx, ny=ny, nz=nz, eos=E.CS, a=CS_A, b=CS_B, kappa=kappa, tau=tau,
                      thermal=thermal, force_form=force_form)
    rho, u, T = inputs.droplet(nx, ny, 10.0, rv, rl, RT)
    if nz > 1:
        rho, T = np.tile(rho, nz), np.tile(T, nz)
        u = np.concatenate([np.tile(u, (1, nz)), np.zeros((1, nx * ny * nz))]) if Q == 27 else np.tile(u, (1, nz))
    return oracle.State(p, rho, u, T)


@pytest.mark.parametrize("thermal,tr", [(0, 0.9), (1, 0.8)])
def test_mass_and_momentum_conserved(thermal, tr):
    """Mass is conserved to rounding; with the divergence-form force sum_x F = 0,
    so the raw momentum stays at rounding level (collision adds dt F per node)."""
    s = droplet_oracle(thermal=thermal, tr=tr)
    t0 = s.totals()
    s.step(300)
    t1 = s.totals()
    assert abs(t1[0] - t0[0]) / t0[0] < 1e-13
    assert abs(t1[1]) < 1e-13 * t0[0] and abs(t1[2]) < 1e-13 * t0[0]


def test_literal_force_form_moves_momentum_by_sum_F():
    """Literal force: the total raw momentum changes by exactly sum_x F each step."""
    s = droplet_oracle(force_form=1)
    s.step(50)
    t0 = s.totals()
    _, _, _, F = s.macro()
    s.step(1)
    t1 = s.totals()
    scale = np.abs(F).sum()
    assert abs((t1[1] - t0[1]) - F[0].sum()) < 1e-12 * scale
    assert abs((t1[2] - t0[2]) - F[1].sum()) < 1e-12 * scale


def test_energy_changes_by_work_of_force():
    """rho E = Gamma + dt/2 u.F and g* carries E* = E + lambda u.F/rho, so one step
    changes sum g by exactly dt sum_x u.F."""
    s = droplet_oracle(thermal=1)
    s.step(40)
    g0 = s.totals()[4]
    _, u, _, F = s.macro()
    work = float((u * F).sum())
    s.step(1)
    g1 = s.totals()[4]
    assert abs(work) > 1e-9 * abs(g0)
    assert g1 - g0 == pytest.approx(work, rel=1e-7)


@pytest.mark.parametrize("thermal", [0, 1])
def test_d2q9_is_marginal_of_d3q27(thermal):
    """On z-invariant fields the c_z-sums of the D3Q27 populations evolve exactly as
    D2Q9 (weights, Psi and the force stencils all marginalise)."""
    nx, ny, nz = 24, 20, 3
    s2 = droplet_oracle(nx, ny, thermal=thermal, tr=0.9)
    s3 = droplet_oracle(nx, ny, thermal=thermal, Q=27, nz=nz, tr=0.9)
    for _ in range(3):
        s2.step(10)
        s3.step(10)
        N = nx * ny
        for h2, h3 in ((s2.f, s3.f), (s2.g, s3.g)) if thermal else ((s2.f, s3.f),):
            m = h3.reshape(3, 9, nz, N).sum(axis=0)          # sum over c_z
            for z in range(nz):
                np.testing.assert_allclose(m[:, z], h2, rtol=1e-10, atol=1e-17)


def _bgk_reference(f, omega, theta, steps):
    """Independent plain BGK on D2Q9 with the product-form equilibrium at fixed theta:
    pull streaming, rho = sum f, u = sum c f / rho, f += omega (f^eq - f)."""
    c = [(i % 3 - 1, i // 3 - 1) for i in range(9)]
    for _ in range(steps):
        f = np.stack([np.roll(np.roll(f[i], c[i][1], axis=0), c[i][0], axis=1) for i in range(9)])
        rho = f.sum(0)
        ux = sum(c[i][0] * f[i] for i in range(9)) / rho
        uy = sum(c[i][1] * f[i] for i in range(9)) / rho
        psi = lambda ci, v: 1 - theta - v * v if ci == 0 else 0.5 * (theta + v * v + ci * v)
        feq = np.stack([rho * psi(c[i][0], ux) * psi(c[i][1], uy) for i in range(9)])
        f = f + omega * (feq - f)
    return f


def test_reduces_to_plain_bgk():
    """a = b = kappa = 0, theta0 = RT = 1/3, frozen temperature, shear flow: F = 0,
    Phi = Phi' = 0, f* = f^eq and the step is plain BGK with omega = 2 beta."""
    nx, ny, tau = 8, 32, 0.3
    p = oracle.Params(Q=9, nx=nx, ny=ny, eos=E.VDW, a=0.0, b=0.0, kappa=0.0, tau=tau, thermal=0)
    rho, u, T = inputs.shear_wave(nx, ny, 1.0, 1.0 / 3.0, U=0.05)
    s = oracle.State(p, rho, u, T)
    f0 = s.f.reshape(9, ny, nx).copy()
    s.step(30)
    ref = _bgk_reference(f0, 2.0 / (2.0 * tau + 1.0), 1.0 / 3.0, 30)
    np.testing.assert_allclose(s.f.reshape(9, ny, nx), ref, rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("RT", [1.0 / 3.0, 0.2])
@pytest.mark.parametrize("tau", [0.3, 1.0])
def test_shear_wave_viscosity(RT, tau):
    """Ideal gas, thermal: a shear wave decays at nu = mu/rho = tau P0/rho (Eq. viscosity,
    1/(2 beta) - 1/2 = tau/dt), within 1 % at L = 64."""
    L = 64
    p = oracle.Params(Q=9, nx=1, ny=L, eos=E.VDW, a=0.0, b=0.0, kappa=0.0, tau=tau, thermal=1)
    rho, u, T = inputs.shear_wave(1, L, 1.0, RT, U=1e-4)
    s = oracle.State(p, rho, u, T)
    k = 2 * math.pi / L
    y = np.arange(L)
    amps = []
    for _ in range(300):
        _, uu, _, _ = s.macro()
        amps.append(2.0 / L * np.sum(uu[0] * np.sin(k * y)))
        s.step(1)
    t = np.arange(len(amps))
    nu = -np.polyfit(t[20:], np.log(np.abs(amps[20:])), 1)[0] / k**2
    assert nu == pytest.approx(tau * RT, rel=0.01)


@pytest.mark.parametrize("RT,tau", [(0.2, 0.3), (1.0 / 3.0, 0.5)])
def test_sound_wave_speed_and_attenuation(RT, tau):
    """Ideal monatomic gas with Pr = 1 (k = 5/2 R mu, Eq. LB_energy_balance) and zero bulk
    viscosity: adiabatic sound speed c^2 = 5/3 RT and amplitude decay rate nu k^2
    ((4/3) nu + (gamma - 1) nu over 2).  Pins the energy populations and the Phi', q'
    corrections (a wrong Fourier-flux or bulk correction changes the decay rate)."""
    L, A = 128, 1e-4
    p = oracle.Params(Q=9, nx=L, ny=1, eos=E.VDW, a=0.0, b=0.0, kappa=0.0, tau=tau, thermal=1)
    x = np.arange(L, dtype=float)
    k = 2 * math.pi / L
    rho = 1.0 + A * np.cos(k * x)
    T = RT * (1.0 + (2.0 / 3.0) * A * np.cos(k * x))       # adiabatic: dT/T = (gamma-1) drho/rho
    s = oracle.State(p, rho, np.zeros((2, L)), T)
    cs = math.sqrt(5.0 / 3.0 * RT)
    energy, rhohat = [], []
    for _ in range(1500):
        r, uu, _, _ = s.macro()
        rh = 2.0 / L * np.sum((r - 1.0) * np.cos(k * x))
        uh = 2.0 / L * np.sum(uu[0] * np.sin(k * x))
        energy.append(rh**2 + (uh / cs) ** 2)
        rhohat.append(rh)
        s.step(1)
    t = np.arange(len(energy))
    alpha = -0.5 * np.polyfit(t[100:], np.log(energy[100:]), 1)[0]
    assert alpha == pytest.approx(tau * RT * k**2, rel=0.05)
    rh = np.array(rhohat)
    zc = np.where(np.diff(np.sign(rh)) != 0)[0]
    period = 2.0 * np.mean(np.diff(zc))
    assert 2 * math.pi / period / k == pytest.approx(cs, rel=0.01)


@pytest.mark.parametrize("form", [0, 1])
def test_force_stencil_second_order(form):
    """F = grad(a rho^2) + kappa rho grad(lap rho) (Enskog gauge, Eqs. EVforce1, P0E) from
    the discrete stencils converges to the analytic force at second order."""
    a, kappa = 0.3, 0.7
    errs = []
    for L in (64, 128):
        p = oracle.Params(Q=9, nx=L, ny=L, eos=E.CS, a=a, b=4.0, kappa=kappa, tau=0.5, force_form=form)
        k = 2 * math.pi / L
        y, x = np.mgrid[0:L, 0:L].astype(float)
        rho = 0.2 + 0.02 * np.sin(k * x) + 0.01 * np.cos(2 * k * y) + 0.005 * np.sin(k * (x + y))
        F = oracle.force(p, rho.ravel()).reshape(2, L, L)
        # analytic derivatives
        rx = 0.02 * k * np.cos(k * x) + 0.005 * k * np.cos(k * (x + y))
        ry = -0.02 * k * np.sin(2 * k * y) + 0.005 * k * np.cos(k * (x + y))
        lap = -0.02 * k**2 * np.sin(k * x) - 0.04 * k**2 * np.cos(2 * k * y) - 0.01 * k**2 * np.sin(k * (x + y))
        lapx = -0.02 * k**3 * np.cos(k * x) - 0.01 * k**3 * np.cos(k * (x + y))
        lapy = 0.08 * k**3 * np.sin(2 * k * y) - 0.01 * k**3 * np.cos(k * (x + y))
        Fx = 2 * a * rho * rx + kappa * rho * lapx
        Fy = 2 * a * rho * ry + kappa * rho * lapy
        errs.append(max(np.abs(F[0] - Fx).max(), np.abs(F[1] - Fy).max()) / np.abs(Fx).max())
    assert errs[1] < 0.02
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.15)


def test_force_forms_agree_on_smooth_fields():
    """Divergence and literal forms differ only by discretisation error."""
    L = 64
    k = 2 * math.pi / L
    y, x = np.mgrid[0:L, 0:L].astype(float)
    rho = (0.2 + 0.02 * np.sin(k * x) * np.cos(k * y)).ravel()
    F = [oracle.force(oracle.Params(Q=9, nx=L, ny=L, a=0.3, b=4.0, kappa=0.7, force_form=ff), rho)
         for ff in (0, 1)]
    assert np.abs(F[0] - F[1]).max() < 0.01 * np.abs(F[0]).max()


def test_isothermal_state_holds_temperature():
    """thermal = 0 keeps the frozen temperature field exactly."""
    s = droplet_oracle(thermal=0, tr=0.9)
    T0 = s.T_iso.copy()
    s.step(20)
    _, _, T, _ = s.macro()
    np.testing.assert_array_equal(T, T0)


def test_step_is_deterministic_and_composes():
    """n steps at once equal n single steps (bit for bit)."""
    a = droplet_oracle()
    b = droplet_oracle()
    a.step(7)
    for _ in range(7):
        b.step(1)
    np.testing.assert_array_equal(a.f, b.f)
    np.testing.assert_array_equal(a.g, b.g)


def _dense_gas(b, rho0, RT0):
    """Carnahan-Starling hard-sphere gas (a = kappa = 0, so F = 0 and P0 = P_E = rho RT Z):
    Z, rho Z'/Z, c_v = 3/2 R and c_p = c_v + R Z^2/(Z + rho Z')  (R = 1)."""
    P0, th, g0 = oracle.eos_state(E.CS, b, rho0, RT0)
    Z = th / RT0
    eta = b * rho0 / 4
    dlnZ = eta * (4 + 4 * eta - 2 * eta**2) / ((1 - eta) * (1 + eta + eta**2 - eta**3))
    return P0, Z, dlnZ, 1.5, 1.5 + Z / (1 + dlnZ)


@pytest.mark.parametrize("tau", [0.2, 0.5])
def test_dense_gas_heat_conduction(tau):
    """Entropy mode of a dense gas (P0 = P_E != rho RT, so the Fourier-flux correction
    q' of Eq. correction_q is active) decays at k_th/(rho c_p) k^2 with k_th = 5/2 R mu
    and mu = tau P0 (Eqs. viscosity, LB_energy_balance)."""
    b, rho0, RT0, L, A = 4.0, 0.2, 0.05, 64, 1e-4
    P0, Z, dlnZ, cv, cp = _dense_gas(b, rho0, RT0)
    p = oracle.Params(Q=9, nx=L, ny=1, eos=E.CS, a=0.0, b=b, kappa=0.0, tau=tau, thermal=1)
    x = np.arange(L, dtype=float)
    k = 2 * math.pi / L
    dT = A * RT0 * np.cos(k * x)
    drho = -(rho0 * Z) * dT / (RT0 * Z * (1 + dlnZ))       # isobaric: dP = 0
    s = oracle.State(p, rho0 + drho, np.zeros((2, L)), RT0 + dT)
    amps = []
    for _ in range(2500):
        r, _, T, _ = s.macro()
        ds = 1.5 * (T - RT0) / RT0 - Z * (r - rho0) / rho0   # entropy per mass / R
        amps.append(2.0 / L * np.sum(ds * np.cos(k * x)))
        s.step(1)
    t = np.arange(len(amps))
    rate = -np.polyfit(t[200:], np.log(np.abs(amps[200:])), 1)[0]
    assert rate == pytest.approx(2.5 * tau * P0 / (rho0 * cp) * k**2, rel=0.01)


def test_dense_gas_sound():
    """Sound in a dense gas: c^2 = gamma0 P0/rho (gamma0 of Eq. gamma is the adiabatic
    exponent of P = rho RT Z with c_v = 3/2 R) and zero bulk viscosity (Phi', Eq.
    correction_gamma): amplitude decay (k^2/2)[(4/3) nu + (k_th/rho)(1/c_v - 1/c_p)]."""
    b, rho0, RT0, L, A, tau = 4.0, 0.2, 0.05, 128, 1e-4, 0.3
    P0, Z, dlnZ, cv, cp = _dense_gas(b, rho0, RT0)
    g0 = oracle.eos_state(E.CS, b, rho0, RT0)[2]
    p = oracle.Params(Q=9, nx=L, ny=1, eos=E.CS, a=0.0, b=b, kappa=0.0, tau=tau, thermal=1)
    x = np.arange(L, dtype=float)
    k = 2 * math.pi / L
    drho = A * rho0 * np.cos(k * x)
    T = RT0 * (1.0 + (2.0 / 3.0) * Z * drho / rho0)          # isentropic
    s = oracle.State(p, rho0 + drho, np.zeros((2, L)), T)
    cs = math.sqrt(g0 * P0 / rho0)
    energy, rhohat = [], []
    for _ in range(1500):
        r, uu, _, _ = s.macro()
        rh = 2.0 / L * np.sum((r - rho0) * np.cos(k * x)) / rho0
        uh = 2.0 / L * np.sum(uu[0] * np.sin(k * x))
        energy.append(rh**2 + (uh / cs) ** 2)
        rhohat.append(rh)
        s.step(1)
    t = np.arange(len(energy))
    alpha = -0.5 * np.polyfit(t[100:], np.log(energy[100:]), 1)[0]
    nu = tau * P0 / rho0
    want = 0.5 * k**2 * (4.0 / 3.0 * nu + 2.5 * tau * P0 / rho0 * (1 / cv - 1 / cp))
    assert alpha == pytest.approx(want, rel=0.05)
    rh = np.array(rhohat)
    zc = np.where(np.diff(np.sign(rh)) != 0)[0]
    assert 2 * math.pi / (2.0 * np.mean(np.diff(zc))) / k == pytest.approx(cs, rel=0.01)


@pytest.mark.parametrize("Q", [9, 27])
@pytest.mark.parametrize("thermal", [1, 0])
@pytest.mark.parametrize("u0", [(0.0, 0.0, 0.0), (0.03, -0.02, 0.01)])
def test_uniform_state_is_a_fixed_point(Q, thermal, u0):
    """A uniform state (liquid density of the non-ideal fluid, at rest or moving) has
    no gradients: F = 0 (Eq. EVforce1), Phi = Phi' = q' = 0, so f* = f^eq, g* = g^eq and
    the collision of Eq. pre_LBM leaves the equilibria unchanged; streaming moves equal
    values.  The populations stay at their initial values to rounding, and the
    macroscopic fields are returned unchanged."""
    RT, rv, rl, kappa = cs_state(0.8)
    nx, ny, nz = 6, 5, (4 if Q == 27 else 1)
    N = nx * ny * nz
    D = 2 if Q == 9 else 3
    p = oracle.Params(Q=Q, nx=nx, ny=ny, nz=nz, eos=E.CS, a=CS_A, b=CS_B, kappa=kappa, tau=0.3, thermal=thermal)
    u = np.array([np.full(N, u0[a]) for a in range(D)])
    s = oracle.State(p, np.full(N, rl), u, np.full(N, RT))
    f0, g0 = s.f.copy(), s.g.copy()
    s.step(10)
    assert np.max(np.abs(s.f - f0)) <= 1e-14 * np.max(np.abs(f0))
    if thermal:
        assert np.max(np.abs(s.g - g0)) <= 1e-14 * np.max(np.abs(g0))
    rho, uu, T, F = s.macro()
    assert np.allclose(rho, rl, rtol=1e-14) and np.allclose(T, RT, rtol=1e-13)
    assert np.allclose(uu, u, atol=1e-15) and np.all(np.abs(F) <= 1e-15)


def _perm_fields(rho, u, T, n, D, op):
    """Apply an axis permutation or reflection of the cubic (square) lattice to fields
    stored [z][y][x]: op = 'xy' swaps x and y, 'xz' swaps x and z, 'rx' reflects x."""
    shp = (n, n, n) if D == 3 else (1, n, n)

    def f3(a):
        a = a.reshape(shp)
        if op == "xy":
            a = np.swapaxes(a, 1, 2)
        elif op == "xz":
            a = np.swapaxes(a, 0, 2)
        else:
            a = np.roll(a[:, :, ::-1], 1, axis=2)              # x -> -x (mod n)
        return np.ascontiguousarray(a).reshape(-1)

    uu = [f3(u[a]) for a in range(D)]
    if op == "xy":
        uu[0], uu[1] = uu[1], uu[0]
    elif op == "xz":
        uu[0], uu[2] = uu[2], uu[0]
    else:
        uu[0] = -uu[0]
    return f3(rho), np.array(uu), f3(T)


@pytest.mark.parametrize("Q,op", [(9, "xy"), (9, "rx"), (27, "xy"), (27, "xz"), (27, "rx")])
def test_step_commutes_with_the_lattice_symmetries(Q, op):
    """The velocity sets, stencils and equilibria are invariant under the permutations
    and reflections of the axes, so stepping a transformed state gives the transformed
    result (to rounding): an index or sign slip on one axis breaks this."""
    RT, rv, rl, kappa = cs_state(0.85)
    n = 6 if Q == 27 else 10
    D = 3 if Q == 27 else 2
    N = n ** D
    s1, s2 = E.spinodal(E.CS, CS_A, CS_B, RT)
    rho = inputs.spinodal_noise(n, n, n if D == 3 else 1, 0.5 * (s1 + s2), RT, amplitude=0.05, D=D)[0]
    r = np.random.default_rng(3)
    u = 0.01 * r.standard_normal((D, N))
    T = RT * (1.0 + 0.02 * r.standard_normal(N))
    p = oracle.Params(Q=Q, nx=n, ny=n, nz=n if D == 3 else 1, eos=E.CS, a=CS_A, b=CS_B, kappa=kappa, tau=0.3)
    a = oracle.State(p, rho, u, T)
    a.step(5)
    ra, ua, Ta, _ = a.macro()
    b = oracle.State(p, *_perm_fields(rho, u, T, n, D, op))
    b.step(5)
    rb, ub, Tb, _ = b.macro()
    pr, pu, pT = _perm_fields(ra, ua, Ta, n, D, op)
    assert np.max(np.abs(rb - pr) / pr) <= 1e-12
    assert np.max(np.abs(Tb - pT) / pT) <= 1e-12
    assert np.max(np.abs(ub - pu)) <= 1e-13
