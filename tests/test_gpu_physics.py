"""The static-droplet Laplace sweep at full size (9 x 1024^2 D2Q9 thermal FP32 layers,
T/Tc in {0.7, 0.8, 0.9} x R in {64, 128, 256}, 20000 steps).  Reported per layer: whether
it stayed finite, the pressure jump p_in - p_out, spurious currents and temperatures;
per temperature the fitted slope of dp against 1/R next to the square-gradient tension.
Asserted: the T/Tc >= 0.8 layers stay finite.  At 4-node interfaces the thermal
model's spurious currents (a few 1e-2) and drop/vapour temperature differences give
pressure differences larger than the Laplace jump sigma/R, so dp is reported, not
checked against 1/R; the currents shrink as the interface widens (width 8: 6e-3).
Run with -s."""
import numpy as np
import pytest

import oracle.eos as E
import paper_2508_00577_gb300 as ev
from paper_2508_00577_gb300 import inputs

pytestmark = pytest.mark.gpu

A, B, KAPPA, TAU = 0.1, 4.0, 0.116, 0.3
TRS = (0.7, 0.8, 0.9)
RADII = (64.0, 128.0, 256.0)


def test_laplace_sweep_full_size():
    n, steps = 1024, 20000
    _, Tc = E.critical_point(E.CS, A, B)
    cases = []
    for tr in TRS:
        rv, rl = E.maxwell(E.CS, A, B, tr * Tc)
        for R in RADII:
            cases.append((R, rv, rl, tr * Tc))
    rho, u, T = inputs.droplet_stack(n, n, cases)
    p = ev.lbm_params.make(nx=n, ny=n, nz=len(cases), eos=ev.LBM_EOS_CS, a=A, b=B, kappa=KAPPA, tau=TAU,
                           precision=ev.LBM_FP32)
    with ev.Lattice(p, rho, u, T) as g:
        ev.lbm_autotune(g.ctx, 2)
        g.step(steps)
        r, uu, TT, _ = g.moments()
    L = len(cases)
    r = r.reshape(L, n, n)
    TT = TT.reshape(L, n, n)
    uu = uu.reshape(2, L, n, n)
    finite = [bool(np.isfinite(r[k]).all() and np.isfinite(TT[k]).all()) for k in range(L)]
    c = n // 2
    print("\nT/Tc   R    finite rho_in    rho_out   dp          max|u|    T_in/Tc  T_out/Tc")
    for k, tr in enumerate(TRS):
        dps, invR = [], []
        for m, R in enumerate(RADII):
            idx = 3 * k + m
            if not finite[idx]:
                print(f"{tr:4.2f} {R:5.0f} no")
                continue
            sl_in = (idx, slice(c - 3, c + 3), slice(c - 3, c + 3))
            sl_out = (idx, slice(0, 6), slice(0, 6))
            p_in = E.pressure(E.CS, A, B, TT[sl_in], r[sl_in]).mean()
            p_out = E.pressure(E.CS, A, B, TT[sl_out], r[sl_out]).mean()
            dps.append(p_in - p_out)
            invR.append(1.0 / R)
            umax = float(np.abs(uu[:, idx]).max())
            print(f"{tr:4.2f} {R:5.0f} yes {r[sl_in].mean():9.5f} {r[sl_out].mean():9.5f} {p_in - p_out: .3e} "
                  f"{umax:.2e} {TT[sl_in].mean() / Tc:7.4f} {TT[sl_out].mean() / Tc:7.4f}")
        if len(dps) == 3:
            slope = np.polyfit(invR, dps, 1)[0]
            _, sigma = E.interface(E.CS, A, B, tr * Tc, KAPPA)
            print(f"  T/Tc={tr}: fitted dp-vs-1/R slope {slope:.3e}, square-gradient sigma {sigma:.3e}")
        if tr >= 0.8:
            assert len(dps) == 3, f"T/Tc={tr} layers went non-finite"


def test_flat_slab_coexistence_curve_on_gpu():
    """The paper's Fig. 1 setting on the fused FP32 kernel (isothermal van der Waals slabs,
    a = 9/392/16, b = 2/21, 8-node interfaces, 8000 steps): the coexistence densities
    agree with the FP64 oracle's run of the same slab to 1e-4 and, like the oracle's,
    with the Maxwell construction -- liquid within 1 %, vapour below it by at most 30 %
    (tests/test_oracle_coexistence.py pins the oracle).  Prints the curve."""
    import oracle
    a, b = 9 / 392 / 16, 2 / 21
    _, Tc = E.critical_point(E.VDW, a, b)
    print("\nT/Tc  rho_l (Maxwell)  rho_v (Maxwell)")
    for tr in (0.7, 0.8, 0.9, 0.95):
        RT = tr * Tc
        rv, rl = E.maxwell(E.VDW, a, b, RT)
        kappa = E.kappa_for_width(E.VDW, a, b, RT, 8.0)
        f = inputs.slab(384, 4, rv, rl, RT, thickness=192.0, width=8.0)
        p = ev.lbm_params.make(nx=384, ny=4, eos=ev.LBM_EOS_VDW, a=a, b=b, kappa=kappa, tau=0.3, thermal=0,
                               precision=ev.LBM_FP32)
        with ev.Lattice(p, *f) as g:
            g.step(8000)
            rho = g.moments()[0]
        o = oracle.State(oracle.Params(Q=9, nx=384, ny=4, eos=E.VDW, a=a, b=b, kappa=kappa, tau=0.3, thermal=0), *f)
        o.step(8000)
        ro = o.macro()[0]
        print(f"{tr:.2f}  {rho.max():.5f} ({rl:.5f})  {rho.min():.5f} ({rv:.5f})")
        assert abs(rho.max() / ro.max() - 1) <= 1e-4 and abs(rho.min() / ro.min() - 1) <= 1e-4
        assert abs(rho.max() / rl - 1) <= 0.01
        assert -0.30 <= rho.min() / rv - 1 <= 0.0
