"""Flat-interface coexistence of the oracle's isothermal step against the Maxwell
equal-area construction of the same equation of state (the paper's Fig. 1 setting: the
van der Waals form of P_E, Eq. P0E with the attraction -a rho^2; T frozen, Sec. 5).

The method reaches the Maxwell densities in the limit of a resolved interface: the
liquid branch within 1 %, the vapour branch below it by an amount that shrinks as the
interface widens (a discretisation error of the split between the lattice pressure
P_E and the force).  a = 9/392/16, b = 2/21 (R T_c = 0.0045): with a four to sixteen
times larger a the liquid's lattice sound speed approaches one lattice unit per step
below T/Tc = 0.8 and the slab diverges."""
import numpy as np
import pytest

import oracle
import oracle.eos as E
from paper_2508_00577_gb300 import inputs

A, B = 9 / 392 / 16, 2 / 21


def slab_coexistence(tr, width, nx=384, steps=8000):
    _, Tc = E.critical_point(E.VDW, A, B)
    RT = tr * Tc
    rv, rl = E.maxwell(E.VDW, A, B, RT)
    kappa = E.kappa_for_width(E.VDW, A, B, RT, width)
    f = inputs.slab(nx, 4, rv, rl, RT, thickness=nx / 2, width=width)
    o = oracle.State(oracle.Params(Q=9, nx=nx, ny=4, eos=E.VDW, a=A, b=B, kappa=kappa, tau=0.3, thermal=0), *f)
    o.step(steps)
    rho = o.macro()[0]
    assert np.isfinite(rho).all()
    return rho.max() / rl - 1.0, rho.min() / rv - 1.0


@pytest.mark.parametrize("tr", [0.7, 0.8, 0.9, 0.95])
def test_flat_slab_coexistence_vdw(tr):
    liq, vap = slab_coexistence(tr, 8.0)
    assert abs(liq) <= 0.01
    assert -0.30 <= vap <= 0.0


def test_coexistence_converges_with_interface_width():
    errs = [slab_coexistence(0.9, w) for w in (4.0, 8.0, 12.0)]
    vap = [abs(v) for _, v in errs]
    assert vap[0] > vap[1] > vap[2]
    assert vap[2] <= 0.05
    assert all(abs(l) <= 0.005 for l, _ in errs)
