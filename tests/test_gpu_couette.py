"""The supersonic thermal Couette flow (the paper's Fig. 2 set-up) on the GPU, through the C
ABI (lbm_set_walls), against the oracle run with the same diffusely reflecting wall nodes
(tests/test_oracle_couette.py states the reading and the steady solution):
* FP64 stage kernels: populations bit-identical to the oracle (D2Q9 and D3Q27);
* fused FP32 D2Q9 kernel: rho and T within 1e-5, u within 1e-6 of the oracle after 50
  steps, one launch per step;
  (these two start from a density perturbed along y, so that every stencil direction
  takes part, and run at Ma = 0.6: from an impulsive start at Ma = 1.2 such a perturbed
  channel diverges within 100 steps, in the oracle as on the GPU; the paper's flow is
  uniform along the walls);
* the steady state after 100000 steps of the fused FP32 kernel at Ma = 1.2: the profiles
  of the oracle pin (u_y within 1e-3 U_w of the steady solution, rho within 1e-3, T within
  1 % of the viscous heating of T(u_y) = T_w + u_y (U_w - u_y)/5) and within 1e-4 of the
  oracle's own steady state;
* argument checks of lbm_set_walls.
"""
import math

import numpy as np
import pytest

import oracle
import oracle.eos as E
import paper_2508_00577_gb300 as ev

import test_oracle_couette as C

pytestmark = pytest.mark.gpu


def setup(Q, nx, ny, nz, eos, b, a, precision, Ma=0.6):
    P0, _, g0 = oracle.eos_state(eos, b, 1.0, C.RTW)
    Uw = Ma * math.sqrt(g0 * P0 - 2 * a)
    D = 2 if Q == 9 else 3
    N = nx * ny * nz
    # a small y-dependent perturbation so that the y stencils matter
    y = np.repeat(np.arange(ny), nx)
    y = np.tile(y, nz)
    x = np.tile(np.arange(nx), ny * nz)
    rho = 1.0 + 0.01 * np.sin(2 * np.pi * y / ny) * np.sin(np.pi * x / (nx - 1))
    u = np.zeros((D, N))
    u[1, x == nx - 1] = Uw
    T = np.full(N, C.RTW)
    walls = ((0, 0, 0), (0, Uw, 0), C.RTW)
    o = oracle.State(oracle.Params(Q=Q, nx=nx, ny=ny, nz=nz, eos=eos, a=a, b=b, kappa=0.0, tau=C.TAU,
                                   thermal=1, walls=walls), rho, u, T)
    p = ev.lbm_params.make(lattice=ev.LBM_D2Q9 if Q == 9 else ev.LBM_D3Q27, nx=nx, ny=ny, nz=nz, eos=eos, a=a,
                           b=b, kappa=0.0, tau=C.TAU, thermal=1, precision=precision)
    g = ev.Lattice(p, rho, u, T)
    ev.lbm_set_walls(g.ctx, 1, walls[0], walls[1], C.RTW)
    return o, g, Uw


@pytest.mark.parametrize("Q,dims,eos,b,a", [(9, (40, 6, 1), E.VDW, 0.1, 0.05), (9, (33, 5, 2), E.CS, 0.2, 0.05),
                                            (27, (14, 5, 3), E.VDW, 0.1, 0.05)])
def test_walls_fp64_bitexact(Q, dims, eos, b, a):
    o, g, _ = setup(Q, *dims, eos, b, a, ev.LBM_FP64)
    with g:
        assert ev.lbm_launches_per_step(g.ctx) == 5
        for n in (1, 30, 170):
            o.step(n)
            g.step(n)
            f, gg = g.populations()
            assert np.array_equal(f, o.f) and np.array_equal(gg, o.g), n


@pytest.mark.parametrize("eos,b,a", [(E.VDW, 0.1, 0.05), (E.CS, 0.2, 0.05)])
def test_walls_fused_fp32_parity(eos, b, a):
    o, g, _ = setup(9, 130, 70, 1, eos, b, a, ev.LBM_FP32)
    with g:
        assert ev.lbm_launches_per_step(g.ctx) == 1
        o.step(50)
        g.step(50)
        ro, uo, To, _ = o.macro()
        rg, ug, Tg, _ = g.moments()
    er = float(np.max(np.abs(rg - ro) / ro))
    eT = float(np.max(np.abs(Tg - To) / To))
    eu = float(np.max(np.abs(ug - uo)))
    assert er <= 1e-5 and eT <= 1e-5 and eu <= 1e-6, (er, eT, eu)


def test_supersonic_couette_steady_state_fused_fp32():
    eos, b, a = E.VDW, 0.1, 0.05
    nx = C.NX
    P0, _, g0 = oracle.eos_state(eos, b, 1.0, C.RTW)
    Uw = C.MA * math.sqrt(g0 * P0 - 2 * a)
    u = np.zeros((2, nx))
    u[1, -1] = Uw
    p = ev.lbm_params.make(nx=nx, ny=1, eos=eos, a=a, b=b, kappa=0.0, tau=C.TAU, thermal=1,
                           precision=ev.LBM_FP32)
    with ev.Lattice(p, np.ones(nx), u, np.full(nx, C.RTW)) as g:
        ev.lbm_set_walls(g.ctx, 1, (0, 0, 0), (0, Uw, 0), C.RTW)
        g.step(C.STEPS)
        rho, uu, T, _ = g.moments()
    uy = uu[1]
    fl = slice(1, nx - 1)
    pr = E.pressure(eos, a, b, T, rho)
    pbar = float(pr[fl].mean())
    assert (pr[fl].max() - pr[fl].min()) / pbar < 1e-3
    u_an, rho_an, Tof = C.steady_solution(eos, b, a, Uw, pbar)
    heat = Uw**2 / 20.0
    assert np.abs(uy - u_an)[fl].max() < 1e-3 * Uw
    assert (np.abs(rho - rho_an) / rho_an)[fl].max() < 1e-3
    assert np.abs(T - Tof(uy))[fl].max() < 0.01 * heat
    # and the oracle's own steady state
    _, orho, ouy, oT, _, _ = C.couette(eos, b, a)
    assert np.abs(uy - ouy)[fl].max() < 1e-4 * Uw
    assert (np.abs(rho - orho) / orho)[fl].max() < 1e-4
    assert np.abs(T - oT)[fl].max() < 1e-4 * C.RTW


def test_set_walls_argument_checks():
    p = ev.lbm_params.make(nx=16, ny=8, kappa=0.0, precision=ev.LBM_FP32)
    f = (np.full(128, 0.1), np.zeros((2, 128)), np.full(128, 0.01))
    with ev.Lattice(p, *f) as g:
        for args in [((0.1, 0, 0), (0, 0, 0), 0.01), ((0, 0, 0), (0, 0, 0.1), 0.01), ((0, 0, 0), (0, 0, 0), 0.0)]:
            with pytest.raises(ev.LBMError) as e:
                ev.lbm_set_walls(g.ctx, 1, *args)
            assert e.value.code == ev.LBM_EINVAL
        ev.lbm_set_walls(g.ctx, 1, (0, 0, 0), (0, 0.01, 0), 0.01)
        ev.lbm_set_walls(g.ctx, 0)
    pk = ev.lbm_params.make(nx=16, ny=8, kappa=0.1, precision=ev.LBM_FP32)
    with ev.Lattice(pk, *f) as g:
        with pytest.raises(ev.LBMError):
            ev.lbm_set_walls(g.ctx, 1, (0, 0, 0), (0, 0.01, 0), 0.01)       # kappa != 0
    p16 = ev.lbm_params.make(nx=16, ny=8, kappa=0.0, precision=ev.LBM_BF16_DEV)
    with ev.Lattice(p16, *f) as g:
        with pytest.raises(ev.LBMError):
            ev.lbm_set_walls(g.ctx, 1, (0, 0, 0), (0, 0.01, 0), 0.01)       # 16-bit storage
