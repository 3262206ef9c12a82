"""Pins of the oracle's lattice equilibria (Eqs. phi, feq, f_star, geq) and of the
nonlinear idempotent operator K_lambda (Eqs. K, def_ustar, lim_projection).
"""
import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(7)


def moments(Q, f):
    c, _ = oracle.lattice(Q)
    return c, f


@pytest.mark.parametrize("Q", [9, 27])
def test_weights_are_rest_equilibrium(Q):
    """f^eq(rho=1, u=0, theta0=1/3) gives the lattice weights 4/9, 1/9, 1/36 (D2Q9)
    and 8/27, 2/27, 1/54, 1/216 (D3Q27)."""
    c, w = oracle.lattice(Q)
    f = oracle.feq(Q, 1.0, np.zeros(3), 1.0 / 3.0)
    ref = {9: {0: 4 / 9, 1: 1 / 9, 2: 1 / 36}, 27: {0: 8 / 27, 1: 2 / 27, 2: 1 / 54, 3: 1 / 216}}[Q]
    for i in range(Q):
        assert f[i] == pytest.approx(ref[int(np.abs(c[i]).sum())], rel=1e-15)
        assert w[i] == pytest.approx(f[i], rel=1e-15)


@pytest.mark.parametrize("Q", [9, 27])
def test_feq_moments(Q):
    """The product form reproduces the moments 1, c_a, c_a c_b of the local
    Maxwellian with pressure P0: sum f = rho, sum c f = rho u,
    sum c_a c_b f = P0 delta_ab + rho u_a u_b."""
    c, _ = oracle.lattice(Q)
    D = 2 if Q == 9 else 3
    for _ in range(20):
        rho = RNG.uniform(0.01, 3.0)
        u = RNG.uniform(-0.2, 0.2, D)
        th = RNG.uniform(0.05, 0.6)
        f = oracle.feq(Q, rho, u, th)
        assert f.sum() == pytest.approx(rho, rel=1e-14)
        for a in range(D):
            assert (c[:, a] * f).sum() == pytest.approx(rho * u[a], rel=1e-12, abs=1e-15)
            for b in range(D):
                want = rho * th * (a == b) + rho * u[a] * u[b]
                assert (c[:, a] * c[:, b] * f).sum() == pytest.approx(want, rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("Q", [9, 27])
def test_geq_moments(Q):
    """sum g^eq = rho E and sum c_a g^eq = u_a (rho E + P0) (enthalpy flux),
    E = 3/2 RT + u^2/2."""
    c, _ = oracle.lattice(Q)
    D = 2 if Q == 9 else 3
    for _ in range(20):
        rho = RNG.uniform(0.01, 3.0)
        u = RNG.uniform(-0.2, 0.2, D)
        RT = RNG.uniform(0.01, 0.4)
        th = RT * RNG.uniform(1.0, 4.0)
        g = oracle.geq(Q, rho, u, th, RT)
        E = 1.5 * RT + 0.5 * (u**2).sum()
        assert g.sum() == pytest.approx(rho * E, rel=1e-13)
        for a in range(D):
            assert (c[:, a] * g).sum() == pytest.approx(u[a] * (rho * E + rho * th), rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("Q", [9, 27])
def test_geq_equals_operator_definition(Q):
    """g^eq_i = rho prod_a Psi_ia(O_a, O_a^2) E(u, RT) with O_a A = theta0 dA/du_a + u_a A
    (Eq. geq), expanded symbolically by sympy, equals the oracle on every population."""
    sp = pytest.importorskip("sympy")
    D = 2 if Q == 9 else 3
    us = sp.symbols("u0:%d" % D)
    th, RT, rho = sp.symbols("theta RT rho")
    E = sp.Rational(3, 2) * RT + sum(v**2 for v in us) / 2
    O = lambda a, A: th * sp.diff(A, us[a]) + us[a] * A
    c, _ = oracle.lattice(Q)
    exprs = []
    for i in range(Q):
        A = E
        for a in range(D):
            ci = int(c[i, a])
            # Psi(xi, zeta) = 1 - c^2 + 1/2[(3c^2 - 2) zeta + c xi] with xi -> O, zeta -> O^2.
            OA = O(a, A)
            OOA = O(a, OA)
            A = (1 - ci**2) * A + sp.Rational(1, 2) * ((3 * ci**2 - 2) * OOA + ci * OA)
        exprs.append(sp.lambdify((rho, th, RT) + us, rho * A, "math"))
    for _ in range(5):
        rv, tv, RTv = RNG.uniform(0.1, 2), RNG.uniform(0.05, 0.5), RNG.uniform(0.02, 0.3)
        uv = RNG.uniform(-0.3, 0.3, D)
        g = oracle.geq(Q, rv, uv, tv, RTv)
        want = np.array([e(rv, tv, RTv, *uv) for e in exprs])
        np.testing.assert_allclose(g, want, rtol=1e-12, atol=1e-15)


def _K(Q, J, rho, u, RT, lam):
    """K_lambda(J) of Eq. (K) on the lattice with the ideal gauge (P0 = rho RT) and
    no Phi correction: [f^eq(u*, RT*) - f^eq(u, RT)] / lambda, with
    u* = u + lambda F/rho, RT* = RT + 2 lambda Q~/(3 rho) - lambda^2 F.F/(3 rho^2) (Eq. def_ustar),
    F = sum c J, Q~ = sum |c - u|^2/2 J (Eqs. defF, defQ).  The 3 of Eq. (def_ustar)
    counts the translational degrees of freedom; a lattice resolving D of them
    (D2Q9 on its own) uses D in its place."""
    c, _ = oracle.lattice(Q)
    D = 2 if Q == 9 else 3
    cc = c[:, :D].astype(float)
    F = cc.T @ J
    Qt = 0.5 * (((cc - u) ** 2).sum(1) * J).sum()
    us = u + lam * F / rho
    RTs = RT + 2 * lam * Qt / (D * rho) - lam**2 * (F @ F) / (D * rho**2)
    return (oracle.feq(Q, rho, us, RTs) - oracle.feq(Q, rho, u, RT)) / lam


@pytest.mark.parametrize("Q", [9, 27])
def test_K_idempotent_and_orthogonal(Q):
    """K(K(J)) = K(J) and K(J - K(J)) = 0, the properties stated after Eq. (def_ustar)."""
    D = 2 if Q == 9 else 3
    for _ in range(10):
        rho = RNG.uniform(0.5, 2.0)
        u = RNG.uniform(-0.1, 0.1, D)
        RT = RNG.uniform(0.2, 0.4)
        J = RNG.normal(0.0, 0.01, Q)
        lam = RNG.uniform(0.1, 1.0)
        KJ = _K(Q, J, rho, u, RT, lam)
        np.testing.assert_allclose(_K(Q, KJ, rho, u, RT, lam), KJ, rtol=1e-10, atol=1e-14)
        np.testing.assert_allclose(_K(Q, J - KJ, rho, u, RT, lam), 0.0, atol=1e-13)


@pytest.mark.parametrize("Q", [9, 27])
def test_K_linear_projection_limit(Q):
    """lambda -> 0: K -> rho^-1 df^eq/du . F + 2/(3 rho) df^eq/d(RT) Q~ (Eq. lim_projection),
    with an O(lambda) error."""
    D = 2 if Q == 9 else 3
    c, _ = oracle.lattice(Q)
    cc = c[:, :D].astype(float)
    rho, RT = 1.3, 0.3
    u = np.array([0.05, -0.03, 0.02][:D])
    J = RNG.normal(0.0, 0.01, Q)
    F = cc.T @ J
    Qt = 0.5 * (((cc - u) ** 2).sum(1) * J).sum()
    h = 1e-6
    K0 = np.zeros(Q)
    for a in range(D):
        e = np.zeros(D); e[a] = h
        K0 += (oracle.feq(Q, rho, u + e, RT) - oracle.feq(Q, rho, u - e, RT)) / (2 * h) * F[a] / rho
    K0 += (oracle.feq(Q, rho, u, RT + h) - oracle.feq(Q, rho, u, RT - h)) / (2 * h) * 2 * Qt / (D * rho)
    errs = [np.abs(_K(Q, J, rho, u, RT, lam) - K0).max() for lam in (1e-2, 5e-3)]
    assert errs[0] < 1e-3 * np.abs(K0).max() * 10
    assert errs[0] / errs[1] == pytest.approx(2.0, rel=0.05)
