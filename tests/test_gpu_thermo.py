"""The library's thermodynamic set-up helpers against the FP64 oracle's EOS module:
spinodal densities (host bisection in the library), the planar square-gradient
interface (width and tension; the library integrates mu - mu_sat on a grid, the
oracle the free energy) and the kappa that gives a target width.  These set up the
benchmark workloads, which may not call the oracle."""
import pytest

import oracle.eos as E
import paper_2508_00577_gb300 as ev

pytestmark = pytest.mark.gpu

CASES = [(E.CS, 0.1, 4.0), (E.VDW, 9 / 392, 2 / 21), (E.VDW, 9 / 392 / 16, 2 / 21)]


@pytest.mark.parametrize("eos,a,b", CASES)
@pytest.mark.parametrize("tr", [0.6, 0.7, 0.85, 0.95])
def test_spinodal_interface_and_kappa_match_oracle(eos, a, b, tr):
    _, Tc = E.critical_point(eos, a, b)
    RT = tr * Tc
    s = ev.lbm_spinodal(eos, a, b, RT)
    so = E.spinodal(eos, a, b, RT)
    assert s[0] == pytest.approx(so[0], rel=1e-12) and s[1] == pytest.approx(so[1], rel=1e-12)
    # The oracle's 10-90 % band is the set of its 2e5 grid points inside it, so its width
    # can miss up to one cell at each end: 2 / (0.8 * 2e5) = 1.25e-5 relative (the
    # library's grid has nodes on both band edges).  kappa ~ width^-2 doubles that.
    w, sigma = ev.lbm_interface(eos, a, b, RT, 0.5)
    wo, sigmao = E.interface(eos, a, b, RT, 0.5)
    assert w == pytest.approx(wo, rel=2e-5)
    assert sigma == pytest.approx(sigmao, rel=1e-6)
    assert ev.lbm_kappa_for_width(eos, a, b, RT, 4.0) == pytest.approx(E.kappa_for_width(eos, a, b, RT, 4.0),
                                                                       rel=4e-5)


def test_thermo_helpers_reject_bad_input():
    _, Tc = E.critical_point(E.CS, 0.1, 4.0)
    for call in (lambda: ev.lbm_spinodal(E.CS, 0.1, 4.0, 1.01 * Tc),
                 lambda: ev.lbm_interface(E.CS, 0.1, 4.0, 0.8 * Tc, 0.0),
                 lambda: ev.lbm_interface(E.CS, 0.1, 4.0, 1.2 * Tc, 1.0)):
        with pytest.raises(ev.LBMError) as e:
            call()
        assert e.value.code == ev.LBM_EINVAL
