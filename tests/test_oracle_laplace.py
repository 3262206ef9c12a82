"""Capillarity of the oracle's step: the Laplace law for droplets and the tension of a
flat interface against the square-gradient theory of the model's capillary term.

The Vlasov force of the Enskog-Vlasov closure carries the capillary term
kappa rho grad(lap rho) (beside Eq. EVforce1).  In the continuum it is the divergence
of the Korteweg stress, whose planar interface has the square-gradient tension
sigma = int kappa (d rho/dx)^2 dx = int sqrt(2 kappa omega(rho)) d rho
(oracle/eos.interface), and a droplet of radius R in 2-D holds the pressure jump
p(rho_in) - p(rho_out) = sigma / R (Laplace), p = P_E - a rho^2.

Two pins, on the whole discrete step (force, shifted velocity, equilibria and
collision acting together), isothermal Carnahan-Starling fluid at T/Tc = 0.9:
* A flat slab relaxes to mechanical equilibrium (equal bulk pressures) and its
  profile's tension kappa sum_x (D_x rho)^2 per interface approaches sigma as the
  interface widens: the error falls monotonically with the width and is below 5 %
  at a 12-node interface.
* Droplets of radius 36 and 48 at a 12-node interface hold a pressure jump whose
  slope against 1/R (fitted through the origin, with the equimolar radius of the
  relaxed droplet) equals the tension of the flat slab of the same run parameters
  within 5 %, as does each jump; the slope is within 8 % of the square-gradient
  sigma (the flat interface's own discretisation error at this width is ~5 %).  The bulk pressures are taken at the
  droplet centre and at the two lattice rows farthest from it, time-averaged over the
  second half of the run (the relaxation launches sound waves that the viscosity damps
  only slowly; tau = 3 damps them faster and leaves the equilibrium unchanged to within
  the stated bounds).

A planted error in the capillary stress fails both: without the -1/2 kappa |grad rho|^2
term of the Korteweg stress the slab tension at a 12-node interface falls from 0.951 sigma
to 0.893 sigma (measured), outside the first pin's 5 % and the second pin's 8 %.
"""
import numpy as np
import pytest

import oracle
import oracle.eos as E
from paper_2508_00577_gb300 import inputs

A, B, TR = 0.1, 4.0, 0.9


def thermo(width):
    _, Tc = E.critical_point(E.CS, A, B)
    RT = TR * Tc
    rv, rl = E.maxwell(E.CS, A, B, RT)
    kappa = E.kappa_for_width(E.CS, A, B, RT, width)
    sigma = E.interface(E.CS, A, B, RT, kappa)[1]
    return RT, rv, rl, kappa, sigma


def pressure(RT, rho):
    return float(E.pressure(E.CS, A, B, RT, rho))


def flat_slab(width, tau, steps=16000):
    """Relaxed 1-D slab (nx x 1 lattice, two interfaces).  Returns (rho_liquid,
    rho_vapour, tension per interface kappa sum_x (central difference of rho)^2)."""
    RT, rv, rl, kappa, _ = thermo(width)
    n = int(12 * width) + 48
    f = inputs.slab(n, 1, rv, rl, RT, thickness=n / 2, width=width)
    o = oracle.State(oracle.Params(Q=9, nx=n, ny=1, eos=E.CS, a=A, b=B, kappa=kappa, tau=tau, thermal=0), *f)
    o.step(steps)
    rho = o.macro()[0]
    assert np.isfinite(rho).all()
    d = 0.5 * (np.roll(rho, -1) - np.roll(rho, 1))
    return rho[n // 2], rho[0], 0.5 * kappa * float(np.sum(d * d))


def test_flat_interface_tension_converges_to_square_gradient():
    errs = []
    for width in (4.0, 6.0, 8.0, 12.0, 16.0):
        RT, rv, rl, kappa, sigma = thermo(width)
        rho_l, rho_v, sig_m = flat_slab(width, tau=1.0)
        # mechanical equilibrium of the two bulk phases: equal pressures, to within the
        # pressure jump of a droplet of radius 50 (the slab still rings with sound waves)
        assert abs(pressure(RT, rho_l) - pressure(RT, rho_v)) <= sigma / 50.0, width
        errs.append(abs(sig_m / sigma - 1.0))
    assert all(e1 > e2 for e1, e2 in zip(errs, errs[1:])), errs
    assert errs[0] > 0.2                      # a 4-node interface is far from resolved
    assert errs[3] <= 0.05 and errs[4] <= 0.03, errs


def relaxed_droplet(R, width, tau, rv, rl, RT, kappa, steps=6000, margin=32, every=10):
    """Time-averaged (p(rho_centre) - p(rho_far), equimolar radius) of a droplet."""
    n = 2 * R + margin
    f = inputs.droplet(n, n, float(R), rv, rl, RT, width=width)
    o = oracle.State(oracle.Params(Q=9, nx=n, ny=n, eos=E.CS, a=A, b=B, kappa=kappa, tau=tau, thermal=0), *f)
    c = n // 2
    acc = []
    for k in range(steps // every):
        o.step(every)
        if k >= steps // every // 2:
            rho = o.macro()[0].reshape(n, n)
            rin = rho[c - 2:c + 2, c - 2:c + 2].mean()
            rout = rho[0:2, :].mean()
            Re = np.sqrt((rho.sum() - rout * n * n) / (rin - rout) / np.pi)
            acc.append((pressure(RT, rin) - pressure(RT, rout), Re))
    assert np.isfinite(np.array(acc)).all()
    return tuple(np.mean(np.array(acc), axis=0))


def test_laplace_law_droplets():
    width, tau = 12.0, 3.0
    RT, rv, rl, kappa, sigma = thermo(width)
    _, _, sig_m = flat_slab(width, tau)
    jumps = [relaxed_droplet(R, width, tau, rv, rl, RT, kappa, margin=40) for R in (36, 48)]
    dp = np.array([j[0] for j in jumps])
    Re = np.array([j[1] for j in jumps])
    ratios = dp * Re / sig_m
    slope = float(np.sum(dp / Re) / np.sum(1.0 / Re**2))
    print(f"\nLaplace: sigma_model/sigma {sig_m / sigma:.4f}, dp R/sigma_model {ratios}, "
          f"slope/sigma_model {slope / sig_m:.4f}, slope/sigma {slope / sigma:.4f}")
    assert np.all(np.abs(ratios - 1.0) <= 0.05), ratios
    assert abs(slope / sig_m - 1.0) <= 0.05
    # and the square-gradient tension itself, within the flat-interface discretisation
    # error of a 12-node interface (about 5 %, first pin)
    assert abs(slope / sigma - 1.0) <= 0.08
