"""Parity of the CUDA path (called through the C ABI) with the FP64 CPU oracle.

FP64: populations bit-identical to the oracle (same operation order, no FMA
contraction on either side).  FP32: max |d rho|/rho <= 1e-5.  FP16/BF16
deviation storage: max |d rho|/rho <= 1e-3.  Inputs come from the seeded
generators in paper_2508_00577_gb300.inputs; coexisting densities and kappa
from the oracle's EOS module.
"""
import numpy as np
import pytest

import oracle
import oracle.eos as E
import paper_2508_00577_gb300 as ev
from paper_2508_00577_gb300 import inputs

pytestmark = pytest.mark.gpu

A, B = 0.1, 4.0
TOL = {ev.LBM_FP32: 1e-5, ev.LBM_FP16_DEV: 1e-3, ev.LBM_BF16_DEV: 1e-3}


def thermo(tr, eos=E.CS, a=A, b=B, width=4.0):
    _, Tc = E.critical_point(eos, a, b)
    RT = tr * Tc
    rv, rl = E.maxwell(eos, a, b, RT)
    return RT, rv, rl, E.kappa_for_width(eos, a, b, RT, width)


def pair(Q, nx, ny, nz, fields, kappa, precision, eos=E.CS, a=A, b=B, thermal=1, force_form=0, tau=0.3):
    """(oracle state, GPU lattice) from the same fields and parameters."""
    op = oracle.Params(Q=Q, nx=nx, ny=ny, nz=nz, eos=eos, a=a, b=b, kappa=kappa, tau=tau, thermal=thermal,
                       force_form=force_form)
    gp = ev.lbm_params.make(lattice=ev.LBM_D2Q9 if Q == 9 else ev.LBM_D3Q27, nx=nx, ny=ny, nz=nz, eos=eos, a=a,
                            b=b, kappa=kappa, tau=tau, thermal=thermal, precision=precision,
                            force_form=force_form)
    rho, u, T = fields
    return oracle.State(op, rho, u, T), ev.Lattice(gp, rho, u, T)


def droplet_fields(nx, ny, nz, tr=0.8, R=None):
    RT, rv, rl, kappa = thermo(tr)
    R = R if R is not None else 0.3 * min(nx, ny)
    rho, u, T = inputs.droplet(nx, ny, R, rv, rl, RT)
    return (np.tile(rho, nz), np.tile(u, (1, nz)), np.tile(T, nz)), kappa


def assert_bitexact(o, g):
    f, gg = g.populations()
    assert np.array_equal(f, o.f), f"max |df| = {np.abs(f - o.f).max()}"
    if gg is not None:
        assert np.array_equal(gg, o.g), f"max |dg| = {np.abs(gg - o.g).max()}"


# ---------------------------------------------------------------------------
# FP64: bit-exact
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nx,ny,nz", [(48, 40, 1), (37, 23, 1), (1, 1, 1), (5, 1, 2), (33, 17, 3)])
def test_fp64_bitexact_d2q9_droplet(nx, ny, nz):
    fields, kappa = droplet_fields(nx, ny, nz)
    o, g = pair(9, nx, ny, nz, fields, kappa, ev.LBM_FP64)
    assert_bitexact(o, g)                     # initial equilibria
    for n in (1, 9, 40):
        o.step(n)
        g.step(n)
        assert_bitexact(o, g)


def test_fp64_bitexact_slab_2000_steps():
    """64 x 64 D2Q9 planar slab (width 32, tanh width 4) at T/Tc = 0.8, 2000 steps."""
    RT, rv, rl, kappa = thermo(0.8)
    fields = inputs.slab(64, 64, rv, rl, RT, thickness=32.0, width=4.0)
    o, g = pair(9, 64, 64, 1, fields, kappa, ev.LBM_FP64)
    o.step(2000)
    g.step(2000)
    assert_bitexact(o, g)
    # mass conserved to rounding on the GPU too
    assert g.conserved()[0] == pytest.approx(o.totals()[0], rel=1e-13)


@pytest.mark.parametrize("variant", ["isothermal", "literal", "vdw"])
def test_fp64_bitexact_variants(variant):
    nx, ny = 40, 36
    if variant == "vdw":
        a, b = 9 / 392 * 0.1, 2 / 21
        RT, rv, rl, kappa = thermo(0.9, E.VDW, a, b)
        fields = inputs.droplet(nx, ny, 11.0, rv, rl, RT)
        o, g = pair(9, nx, ny, 1, fields, kappa, ev.LBM_FP64, eos=E.VDW, a=a, b=b)
    else:
        fields, kappa = droplet_fields(nx, ny, 1, tr=0.9)
        o, g = pair(9, nx, ny, 1, fields, kappa, ev.LBM_FP64, thermal=0 if variant == "isothermal" else 1,
                    force_form=1 if variant == "literal" else 0)
    o.step(60)
    g.step(60)
    assert_bitexact(o, g)


@pytest.mark.parametrize("thermal", [1, 0])
def test_fp64_bitexact_d3q27(thermal):
    """16^3 (and a ragged 11 x 7 x 5) D3Q27 spinodal noise at T/Tc = 0.85."""
    for nx, ny, nz in ((16, 16, 16), (11, 7, 5)):
        RT, rv, rl, kappa = thermo(0.85)
        s1, s2 = E.spinodal(E.CS, A, B, RT)
        fields = inputs.spinodal_noise(nx, ny, nz, 0.5 * (s1 + s2), RT, amplitude=0.01)
        o, g = pair(27, nx, ny, nz, fields, kappa, ev.LBM_FP64, thermal=thermal)
        o.step(12)
        g.step(12)
        assert_bitexact(o, g)


def test_fp64_moments_bitexact():
    fields, kappa = droplet_fields(30, 26, 1)
    o, g = pair(9, 30, 26, 1, fields, kappa, ev.LBM_FP64)
    o.step(25)
    g.step(25)
    want = o.macro()
    got = g.moments()
    for w, h in zip(want, got):
        assert np.array_equal(w, h)


# ---------------------------------------------------------------------------
# FP32 and reduced-precision storage: tolerances on rho
# ---------------------------------------------------------------------------

def rel_rho_err(o, g):
    ro = o.macro()[0]
    rg = g.moments()[0]
    return np.max(np.abs(rg - ro) / ro)


def field_errs(o, g):
    """(max |d rho|/rho, max |d T|/T, max |d u|) of the GPU state against the oracle's,
    every node, the fields as the next step computes them."""
    ro, uo, To = o.macro()[:3]
    rg, ug, Tg, _ = g.moments()
    return (float(np.max(np.abs(rg - ro) / ro)), float(np.max(np.abs(Tg - To) / To)),
            float(np.max(np.abs(ug.reshape(uo.shape) - uo))))


def assert_fields(o, g, tol):
    """rho and T within `tol` relative, u within tol/10 absolute: the lattice velocity
    scale is the sound speed sqrt(theta0) ~ 0.1, so tol/10 is the same relative bound."""
    er, eT, eu = field_errs(o, g)
    assert er <= tol and eT <= tol and eu <= 0.1 * tol, (er, eT, eu)


@pytest.mark.parametrize("nx,ny,nz", [(96, 80, 1), (130, 70, 2), (257, 33, 1), (7, 5, 1), (1, 1, 1), (300, 260, 1)])
def test_fp32_d2q9(nx, ny, nz):
    """FP32 (fused single-pass kernel for D2Q9): max |d rho|/rho <= 1e-5 over 50 steps
    from a common state (FP32 storage rounding drifts by ~1e-7 per step; the 2000-step
    bound is checked separately).  Sizes span several strips and row chunks, ragged
    tails and degenerate 1-node lattices."""
    fields, kappa = droplet_fields(nx, ny, nz)
    o, g = pair(9, nx, ny, nz, fields, kappa, ev.LBM_FP32)
    assert_fields(o, g, 1e-6)
    o.step(1)
    g.step(1)
    assert_fields(o, g, 1e-6)
    o.step(49)
    g.step(49)
    assert_fields(o, g, 1e-5)


@pytest.mark.parametrize("thermal", [1, 0])
@pytest.mark.parametrize("nx,ny,nz,hz", [(20, 18, 11, 0), (33, 16, 7, 4), (16, 16, 16, 5), (5, 3, 4, 0),
                                         (40, 35, 9, 3), (20, 18, 70, 20), (12, 10, 50, 17)])
def test_fp32_d3q27(nx, ny, nz, hz, thermal):
    """FP32 D3Q27 (fused single-pass kernel): max |d rho|/rho <= 1e-5 over 10 steps of a
    spinodal state with 5 % density noise.  Edges that are not multiples of the 32 x 8
    tile (32 x 16 with 16-bit storage), odd plane counts, z-chunks that do not divide nz (hz; 0 = default chunk) and a
    lattice smaller than one tile.  Chunks above 16 planes end on shorter ones: 70 planes
    at hz 20 run as 20, 20, 15, 15 and 50 at hz 17 as 17, 17, 16."""
    _, Tc = E.critical_point(E.CS, A, B)
    RT = 0.85 * Tc
    s1, s2 = E.spinodal(E.CS, A, B, RT)
    kappa = E.kappa_for_width(E.CS, A, B, RT, 4.0)
    fields = inputs.spinodal_noise(nx, ny, nz, 0.5 * (s1 + s2), RT, amplitude=0.05, D=3)
    o, g = pair(27, nx, ny, nz, fields, kappa, ev.LBM_FP32, thermal=thermal)
    with g:
        if hz:
            ev.lbm_set_tile(g.ctx, 0, hz)
        assert ev.lbm_launches_per_step(g.ctx) == 1       # the fused kernel, not the stage kernels
        o.step(10)
        g.step(10)
        assert_fields(o, g, 1e-5)


@pytest.mark.parametrize("precision", [ev.LBM_FP16_DEV, ev.LBM_BF16_DEV])
@pytest.mark.parametrize("nx,ny,nz,hz", [(20, 18, 11, 4), (33, 17, 50, 17), (7, 5, 3, 0)])
def test_reduced_precision_d3q27(precision, nx, ny, nz, hz):
    """16-bit deviation storage through the fused D3Q27 kernel (one launch per step, the
    decoded f and g stashed in tensor memory): rho and T within 1e-3 relative, u within
    1e-4 of the FP64 oracle after 10 thermal steps of a spinodal state with 5 % density
    noise, on edges that are not multiples of the 32 x 16 tile, uniform z-chunks that do
    not divide nz, chunks ending on shorter ones (50 planes at hz 17: 17, 17, 16) and a
    lattice smaller than one tile."""
    _, Tc = E.critical_point(E.CS, A, B)
    RT = 0.85 * Tc
    s1, s2 = E.spinodal(E.CS, A, B, RT)
    kappa = E.kappa_for_width(E.CS, A, B, RT, 4.0)
    fields = inputs.spinodal_noise(nx, ny, nz, 0.5 * (s1 + s2), RT, amplitude=0.05, D=3)
    o, g = pair(27, nx, ny, nz, fields, kappa, precision)
    with g:
        if hz:
            ev.lbm_set_tile(g.ctx, 0, hz)
        assert ev.lbm_launches_per_step(g.ctx) == 1
        o.step(10)
        g.step(10)
        assert_fields(o, g, 1e-3)


@pytest.mark.parametrize("lam", [0.5, 2.0])
def test_general_lambda(lam):
    """lambda != dt (the shifted velocity u* = u + lambda F / rho, the energy shift with
    lambda^2 and the collision weight (dt/lambda)(1 - beta) of Eq. pre_LBM): FP64
    populations bit-exact (D2Q9 droplet and a D3Q27 spinodal state), the fused FP32
    kernels within 1e-5."""
    fields, kappa = droplet_fields(48, 40, 1, R=12.0)
    o = oracle.State(oracle.Params(Q=9, nx=48, ny=40, eos=E.CS, a=A, b=B, kappa=kappa, tau=0.3, lambda_=lam),
                     *fields)
    o.step(30)
    for prec in (ev.LBM_FP64, ev.LBM_FP32):
        p = ev.lbm_params.make(nx=48, ny=40, eos=ev.LBM_EOS_CS, a=A, b=B, kappa=kappa, lambda_=lam, precision=prec)
        with ev.Lattice(p, *fields) as g:
            g.step(30)
            if prec == ev.LBM_FP64:
                assert_bitexact(o, g)
            else:
                assert_fields(o, g, 1e-5)
    _, Tc = E.critical_point(E.CS, A, B)
    RT = 0.85 * Tc
    s1, s2 = E.spinodal(E.CS, A, B, RT)
    k3 = E.kappa_for_width(E.CS, A, B, RT, 4.0)
    f3 = inputs.spinodal_noise(12, 10, 9, 0.5 * (s1 + s2), RT, amplitude=0.05, D=3)
    o3 = oracle.State(oracle.Params(Q=27, nx=12, ny=10, nz=9, eos=E.CS, a=A, b=B, kappa=k3, tau=0.3, lambda_=lam),
                      *f3)
    o3.step(10)
    for prec in (ev.LBM_FP64, ev.LBM_FP32):
        p = ev.lbm_params.make(lattice=ev.LBM_D3Q27, nx=12, ny=10, nz=9, eos=ev.LBM_EOS_CS, a=A, b=B, kappa=k3,
                               lambda_=lam, precision=prec)
        with ev.Lattice(p, *f3) as g:
            g.step(10)
            if prec == ev.LBM_FP64:
                assert_bitexact(o3, g)
            else:
                assert_fields(o3, g, 1e-5)


@pytest.mark.parametrize("Q", [9, 27])
@pytest.mark.parametrize("variant", ["vdw", "vdw_isothermal", "literal"])
def test_fp32_vdw_eos_and_literal_force(Q, variant):
    """The FP32 paths on the van der Waals form of the Enskog pressure (thermal and
    isothermal) and on the literal force form grad(a rho^2) + kappa rho grad(lap rho):
    max |d rho|/rho <= 1e-5 against the oracle.  D2Q9: a droplet over 50 steps on a
    ragged 130 x 70 lattice; D3Q27: a spinodal state with 5 % noise over 10 steps."""
    eos, a, b = (E.VDW, 9 / 392 * 0.1, 2 / 21) if variant.startswith("vdw") else (E.CS, A, B)
    thermal = 0 if variant == "vdw_isothermal" else 1
    force_form = 1 if variant == "literal" else 0
    _, Tc = E.critical_point(eos, a, b)
    if Q == 9:
        RT, rv, rl, kappa = thermo(0.9, eos, a, b)
        fields = inputs.droplet(130, 70, 20.0, rv, rl, RT)
        dims, steps = (130, 70, 1), 50
    else:
        RT = 0.85 * Tc
        s1, s2 = E.spinodal(eos, a, b, RT)
        kappa = E.kappa_for_width(eos, a, b, RT, 4.0)
        fields = inputs.spinodal_noise(20, 18, 11, 0.5 * (s1 + s2), RT, amplitude=0.05, D=3)
        dims, steps = (20, 18, 11), 10
    o, g = pair(Q, *dims, fields, kappa, ev.LBM_FP32, eos=eos, a=a, b=b, thermal=thermal, force_form=force_form)
    with g:
        o.step(steps)
        g.step(steps)
        assert_fields(o, g, 1e-5)


@pytest.mark.parametrize("nx,ny", [(64, 48), (300, 40)])
def test_fp32_d2q9_isothermal(nx, ny):
    fields, kappa = droplet_fields(nx, ny, 1, tr=0.9)
    o, g = pair(9, nx, ny, 1, fields, kappa, ev.LBM_FP32, thermal=0)
    o.step(50)
    g.step(50)
    assert_fields(o, g, 1e-5)


@pytest.mark.parametrize("precision", [ev.LBM_FP16_DEV, ev.LBM_BF16_DEV])
@pytest.mark.parametrize("nx,ny,nz", [(96, 80, 1), (130, 70, 2)])
def test_reduced_precision_d2q9(precision, nx, ny, nz):
    fields, kappa = droplet_fields(nx, ny, nz)
    o, g = pair(9, nx, ny, nz, fields, kappa, precision)
    o.step(100)
    g.step(100)
    assert_fields(o, g, TOL[precision])


@pytest.mark.parametrize("precision", [ev.LBM_FP16_DEV, ev.LBM_BF16_DEV])
@pytest.mark.parametrize("nx,ny,nz,thermal", [(130, 70, 2, 1), (7, 5, 1, 1), (200, 33, 1, 0)])
def test_reduced_precision_d2q9_fused_launch_shapes(precision, nx, ny, nz, thermal):
    """16-bit storage through the fused D2Q9 kernel (one launch per step) on every strip
    width, a chunk height that does not divide ny and the balanced persistent grid:
    rho and T within 1e-3 relative, u within 1e-4 of the FP64 oracle after 20 steps."""
    fields, kappa = droplet_fields(nx, ny, nz, tr=0.9 if not thermal else 0.8)
    o = oracle.State(oracle.Params(Q=9, nx=nx, ny=ny, nz=nz, eos=E.CS, a=A, b=B, kappa=kappa, tau=0.3,
                                   thermal=thermal), *fields)
    o.step(20)
    ro, uo, To, _ = o.macro()
    for W in (64, 128, 192):
        for H in (6, ev.LBM_TILE_BALANCED):
            gp = ev.lbm_params.make(nx=nx, ny=ny, nz=nz, eos=E.CS, a=A, b=B, kappa=kappa, tau=0.3,
                                    thermal=thermal, precision=precision)
            with ev.Lattice(gp, *fields) as g:
                assert ev.lbm_launches_per_step(g.ctx) == 1
                ev.lbm_set_tile(g.ctx, W, H)
                g.step(20)
                rg, ug, Tg, _ = g.moments()
            er = float(np.max(np.abs(rg - ro) / ro))
            eT = float(np.max(np.abs(Tg - To) / To))
            eu = float(np.max(np.abs(ug.reshape(uo.shape) - uo)))
            assert er <= 1e-3 and eT <= 1e-3 and eu <= 1e-4, (W, H, er, eT, eu)


def test_fp32_long_run_droplet():
    """FP32 storage rounds every population once per step, so the FP32 - FP64 density
    difference drifts by about one FP32 ulp per step; over 2000 steps (128^2, R = 32)
    it stays below 2e-4."""
    fields, kappa = droplet_fields(128, 128, 1, R=32.0)
    o, g = pair(9, 128, 128, 1, fields, kappa, ev.LBM_FP32)
    o.step(2000)
    g.step(2000)
    assert rel_rho_err(o, g) <= 2e-4


# ---------------------------------------------------------------------------
# Other entry points
# ---------------------------------------------------------------------------

def test_moments_device_matches_host():
    torch = pytest.importorskip("torch")
    fields, kappa = droplet_fields(64, 48, 1)
    gp = ev.lbm_params.make(nx=64, ny=48, kappa=kappa, precision=ev.LBM_FP32)
    with ev.Lattice(gp, *fields) as g:
        g.step(10)
        rho_h, u_h, T_h, _ = g.moments()
        rho = torch.empty(gp.N, device="cuda", dtype=torch.float32)
        u = torch.empty(2 * gp.N, device="cuda", dtype=torch.float32)
        T = torch.empty(gp.N, device="cuda", dtype=torch.float32)
        ev.lbm_moments_device(g.ctx, rho.data_ptr(), u.data_ptr(), T.data_ptr())
        ev.lbm_sync(g.ctx)
        np.testing.assert_allclose(rho.cpu().numpy(), rho_h, rtol=1e-7)
        np.testing.assert_allclose(T.cpu().numpy(), T_h, rtol=1e-6)
        np.testing.assert_allclose(u.cpu().numpy(), u_h.ravel(), atol=1e-9)


@pytest.mark.parametrize("eos,a,b", [(E.CS, A, B), (E.VDW, 9 / 392, 2 / 21)])
@pytest.mark.parametrize("tr", [0.7, 0.85, 0.95])
def test_coexistence_fp64_on_gpu(eos, a, b, tr):
    _, Tc = E.critical_point(eos, a, b)
    rv, rl = ev.lbm_coexistence(eos, a, b, tr * Tc)
    ov, ol = E.maxwell(eos, a, b, tr * Tc)
    assert rv == pytest.approx(ov, rel=1e-10)
    assert rl == pytest.approx(ol, rel=1e-10)


def test_step_count_and_zero_steps():
    fields, kappa = droplet_fields(16, 16, 1)
    gp = ev.lbm_params.make(nx=16, ny=16, kappa=kappa, precision=ev.LBM_FP64)
    with ev.Lattice(gp, *fields) as g:
        f0, _ = g.populations()
        g.step(0)
        assert ev.lbm_step_count(g.ctx) == 0
        assert np.array_equal(g.populations()[0], f0)
        g.step(3)
        assert ev.lbm_step_count(g.ctx) == 3


def test_conserved_flags_nonfinite():
    """An unstable state (here: a supercritical liquid far beyond the lattice's
    stable sound speed) ends in non-finite populations; lbm_conserved reports it."""
    _, Tc = E.critical_point(E.CS, 1.0, 4.0)
    RT = 0.8 * Tc
    fields = inputs.spinodal_noise(16, 16, 1, 0.3, RT, amplitude=0.01, D=2)
    gp = ev.lbm_params.make(nx=16, ny=16, a=1.0, b=4.0, kappa=0.0, precision=ev.LBM_FP32)
    with ev.Lattice(gp, *fields) as g:
        g.step(2000)
        with pytest.raises(ev.LBMError) as e:
            g.conserved()
        assert e.value.code == ev.LBM_ENONFINITE


def test_fp32_every_launch_shape():
    """Every strip width and several row-chunk heights (down to one row), and the
    balanced persistent grid, give the same FP32 result within 1e-5 of the oracle
    (ragged strips and chunks included)."""
    nx, ny = 300, 70
    fields, kappa = droplet_fields(nx, ny, 1)
    o, _ = pair(9, nx, ny, 1, fields, kappa, ev.LBM_FP32)
    o.step(30)
    ro = o.macro()[0]
    gp = ev.lbm_params.make(nx=nx, ny=ny, kappa=kappa, precision=ev.LBM_FP32)
    for W in (64, 96, 128, 192):
        for H in (1, 5, 64, 70, ev.LBM_TILE_BALANCED):
            with ev.Lattice(gp, *fields) as g:
                ev.lbm_set_tile(g.ctx, W, H)
                g.step(30)
                err = np.max(np.abs(g.moments()[0] - ro) / ro)
                assert err <= 1e-5, (W, H, err)


def test_autotune_keeps_state():
    fields, kappa = droplet_fields(200, 150, 2)
    gp = ev.lbm_params.make(nx=200, ny=150, nz=2, kappa=kappa, precision=ev.LBM_FP32)
    with ev.Lattice(gp, *fields) as g:
        g.step(5)
        f0, g0 = g.populations()
        w, h = ev.lbm_autotune(g.ctx, 2)
        assert w in (64, 96, 128, 192) and (1 <= h <= 150 or h == ev.LBM_TILE_BALANCED)
        assert ev.lbm_get_tile(g.ctx) == (w, h)
        f1, g1 = g.populations()
        assert np.array_equal(f0, f1) and np.array_equal(g0, g1)
        with pytest.raises(ev.LBMError):
            ev.lbm_set_tile(g.ctx, 100, 10)
        with pytest.raises(ev.LBMError):
            ev.lbm_set_tile(g.ctx, 128, -2)


@pytest.mark.parametrize("prec,width", [(ev.LBM_FP32, 32), (ev.LBM_FP16_DEV, 32), (ev.LBM_BF16_DEV, 32)])
def test_d3q27_tile_shape_per_storage(prec, width):
    """The D3Q27 kernel's x-y tile is fixed per storage type (32 x 8 for FP32, 32 x 16
    for 16-bit storage): lbm_set_tile takes tile_w = 0 or that width, lbm_get_tile and
    lbm_autotune report it, and the autotuner leaves the state as it was."""
    _, Tc = E.critical_point(E.CS, A, B)
    RT = 0.85 * Tc
    s1, s2 = E.spinodal(E.CS, A, B, RT)
    kappa = E.kappa_for_width(E.CS, A, B, RT, 4.0)
    f = inputs.spinodal_noise(40, 24, 12, 0.5 * (s1 + s2), RT, amplitude=0.05, D=3)
    p = ev.lbm_params.make(lattice=ev.LBM_D3Q27, nx=40, ny=24, nz=12, eos=ev.LBM_EOS_CS, a=A, b=B, kappa=kappa,
                           precision=prec)
    with ev.Lattice(p, *f) as g:
        ev.lbm_set_tile(g.ctx, 0, 5)
        assert ev.lbm_get_tile(g.ctx) == (width, 5)
        ev.lbm_set_tile(g.ctx, width, 7)
        assert ev.lbm_get_tile(g.ctx) == (width, 7)
        with pytest.raises(ev.LBMError):
            ev.lbm_set_tile(g.ctx, 48 - width, 7)
        g.step(2)
        f0, g0 = g.populations()
        w, h = ev.lbm_autotune(g.ctx, 1)
        assert w == width and 1 <= h <= 12 and ev.lbm_get_tile(g.ctx) == (w, h)
        f1, g1 = g.populations()
        assert np.array_equal(f0, f1) and np.array_equal(g0, g1)


@pytest.mark.parametrize("precision", [ev.LBM_FP64, ev.LBM_FP32, ev.LBM_BF16_DEV])
def test_init_checks_fields_on_the_device(precision):
    """lbm_init checks the initial fields on the device: a non-positive or non-finite
    density or temperature, or a non-finite velocity, is LBM_ENONFINITE naming the lowest
    such node; a valid set afterwards initialises normally and gives the oracle's state."""
    fields, kappa = droplet_fields(40, 30, 1)
    gp = ev.lbm_params.make(nx=40, ny=30, kappa=kappa, precision=precision)
    rho, u, T = (np.array(a, dtype=np.float64) for a in fields)
    cases = []
    r = rho.copy(); r[37] = 0.0; T2 = T.copy(); T2[500] = np.nan
    cases.append(((r, u, T2), 37))
    u2 = u.copy(); u2[1, 11] = np.inf
    cases.append(((rho, u2, T), 11))
    T3 = T.copy(); T3[1199] = -1.0
    cases.append(((rho, u, T3), 1199))
    for bad_fields, node in cases:
        with pytest.raises(ev.LBMError) as e:
            ev.Lattice(gp, *bad_fields)
        assert e.value.code == ev.LBM_ENONFINITE and f"node {node}" in str(e.value), str(e.value)
    o, g = pair(9, 40, 30, 1, fields, kappa, precision)
    with g:
        ro = o.macro()[0]
        rg = g.moments()[0]
    assert float(np.max(np.abs(rg - ro) / ro)) <= (1e-15 if precision == ev.LBM_FP64 else 1e-3)
