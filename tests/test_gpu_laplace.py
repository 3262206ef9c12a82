"""The Laplace-law droplets of the oracle pin (tests/test_oracle_laplace.py) on the fused
FP32 D2Q9 kernel, through the C ABI.

Isothermal Carnahan-Starling fluid at T/Tc = 0.9, 12-node interfaces, bare tau = 3,
droplets of radius 36 and 48 in periodic boxes of 2R + 40 nodes, 6000 steps.  The GPU
run is compared with the FP64 oracle's run of the same droplets:
* element by element after 50 steps: rho and T within 1e-5 relative, u within 1e-6 (as
  the other FP32 parity tests); FP32 storage rounds every population once per step, and
  at tau = 3 the sound waves that carry that rounding are damped slowly (2.3e-5 in rho
  after 200 steps, 1.7e-3 after 6000, measured), so after the 6000 steps 5e-3 is asked;
* the time-averaged pressure jump (second half of the run, sampled every 10 steps)
  within 1 % of the oracle's, and its ratio to the flat-slab tension of the oracle within
  5 %, as the oracle pin requires of the oracle itself.
"""
import numpy as np
import pytest

import oracle
import oracle.eos as E
import paper_2508_00577_gb300 as ev
from paper_2508_00577_gb300 import inputs

import test_oracle_laplace as L

pytestmark = pytest.mark.gpu

WIDTH, TAU, MARGIN, STEPS, EVERY = 12.0, 3.0, 40, 6000, 10


def jump(rho, n, RT):
    c = n // 2
    rin = rho[c - 2:c + 2, c - 2:c + 2].mean()
    rout = rho[0:2, :].mean()
    Re = np.sqrt((rho.sum() - rout * n * n) / (rin - rout) / np.pi)
    return L.pressure(RT, rin) - L.pressure(RT, rout), Re


@pytest.mark.parametrize("R", [36, 48])
def test_laplace_droplet_fused_fp32(R):
    RT, rv, rl, kappa, sigma = L.thermo(WIDTH)
    _, _, sig_m = L.flat_slab(WIDTH, TAU)
    n = 2 * R + MARGIN
    fields = inputs.droplet(n, n, float(R), rv, rl, RT, width=WIDTH)
    o = oracle.State(oracle.Params(Q=9, nx=n, ny=n, eos=E.CS, a=L.A, b=L.B, kappa=kappa, tau=TAU, thermal=0),
                     *fields)
    p = ev.lbm_params.make(nx=n, ny=n, eos=ev.LBM_EOS_CS, a=L.A, b=L.B, kappa=kappa, tau=TAU, thermal=0,
                           precision=ev.LBM_FP32)
    acc_o, acc_g = [], []
    with ev.Lattice(p, *fields) as g:
        assert ev.lbm_launches_per_step(g.ctx) == 1
        for k in range(STEPS // EVERY):
            o.step(EVERY)
            g.step(EVERY)
            ro, uo, To, _ = o.macro()
            rg, ug, Tg, _ = g.moments()
            if (k + 1) * EVERY in (50, STEPS):
                er = float(np.max(np.abs(rg - ro) / ro))
                eT = float(np.max(np.abs(Tg - To) / To))
                eu = float(np.max(np.abs(ug.reshape(uo.shape) - uo)))
                tol = 1e-5 if (k + 1) * EVERY == 50 else 5e-3
                assert er <= tol and eT <= tol and eu <= 0.1 * tol, ((k + 1) * EVERY, er, eT, eu)
            if k >= STEPS // EVERY // 2:
                acc_o.append(jump(ro.reshape(n, n), n, RT))
                acc_g.append(jump(rg.reshape(n, n), n, RT))
    dpo, Reo = np.mean(np.array(acc_o), axis=0)
    dpg, Reg = np.mean(np.array(acc_g), axis=0)
    print(f"\nR {R}: oracle dp R/sigma_model {dpo * Reo / sig_m:.4f}, GPU {dpg * Reg / sig_m:.4f}")
    assert abs(dpg / dpo - 1.0) <= 0.01
    assert abs(Reg / Reo - 1.0) <= 1e-3
    assert abs(dpg * Reg / sig_m - 1.0) <= 0.05
