"""The oracle's critical points against stored textbook and published values
(tests/golden/critical_constants.txt): the van der Waals closed forms and the
tabulated critical point of the Carnahan-Starling closure with van der Waals
attraction.  The Enskog pressure plus the mean-field attraction is the paper's
construction (Eq. EVforce1 with P0 = P_E); the numbers are not the oracle's."""
import pathlib

import pytest

import oracle.eos as E

GOLDEN = pathlib.Path(__file__).parent / "golden" / "critical_constants.txt"
EOS = {"vdw": E.VDW, "cs": E.CS}


def rows():
    out = []
    for line in GOLDEN.read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            name, *vals = line.split()
            out.append((name, *map(float, vals)))
    return out


@pytest.mark.parametrize("name,brc,bTc,pc,Zc,tol", rows())
@pytest.mark.parametrize("a,b", [(1.0, 4.0), (0.1, 4.0), (9 / 392, 2 / 21)])
def test_critical_constants_match_literature(name, brc, bTc, pc, Zc, tol, a, b):
    eos = EOS[name]
    rc, Tc = E.critical_point(eos, a, b)
    p = float(E.pressure(eos, a, b, Tc, rc))
    assert b * rc == pytest.approx(brc, rel=tol)
    assert b * Tc / a == pytest.approx(bTc, rel=tol)
    assert b * b * p / a == pytest.approx(pc, rel=tol)
    assert p / (rc * Tc) == pytest.approx(Zc, rel=tol)


def test_cs_critical_point_high_precision():
    """The critical point of the CS closure solved independently at 30 digits (sympy's
    Newton on dp/deta = d2p/deta2 = 0 of the symbolic pressure) agrees with the
    oracle's bisection to 1e-13."""
    sp = pytest.importorskip("sympy")
    eta, t = sp.symbols("eta t", positive=True)
    p = 4 * eta * t * (1 + eta + eta**2 - eta**3) / (1 - eta) ** 3 - 16 * eta**2   # a = b = 1
    e_c, t_c = sp.nsolve([sp.diff(p, eta), sp.diff(p, eta, 2)], [eta, t], [0.13, 0.38], prec=30)
    rc, Tc = E.critical_point(E.CS, 1.0, 1.0)
    assert rc == pytest.approx(4 * float(e_c), rel=1e-13)
    assert Tc == pytest.approx(float(t_c), rel=1e-13)
