"""Parity at the workloads' full sizes, in the launch configurations the benchmark times.

* Droplet Laplace sweep, 9 x 1024^2 D2Q9 thermal FP32, autotuned fused-kernel tile:
  every node's density, velocity and temperature after 10 steps against the FP64
  oracle run of the same 9 layers (FP32 bound 1e-5 relative on rho and T; on u,
  1e-5 of the lattice velocity scale, the sound speed sqrt(theta0) ~ 0.1: 1e-6).
* Batched ensemble, 512 uneven droplet-pair domains (64..512)^2 in one persistent
  launch with the autotuned tile: five sampled domains after 20 steps against the
  oracle run of each domain alone (same bounds), one of them a coalescing pair at the
  cold end (T/Tc 0.701, gap 2.3); and the full 5000 steps of the workload, after which
  all but the nine domains the method itself does not hold stay finite (one of those,
  on its own, diverges in the FP64 oracle as on the GPU).
* 3-D spinodal decomposition, 256^3 D3Q27 thermal: 2 steps in FP32 (bound 1e-5)
  and with FP16 / BF16 deviation storage (bound 1e-3) against the oracle.
* Surrogate U-Net at batch 32 x 256^2: one output pixel depends on the whole domain,
  so the oracle cannot produce samples one by one; properties that hold at any size
  are checked instead -- periodic translation equivariance by 8 pixels (the pooling
  stride product) and independence of the batch order.

All inputs are built from the oracle's own EOS routines (oracle/eos.py)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench
import oracle
import oracle.eos as E
import paper_2508_00577_gb300 as ev
from paper_2508_00577_gb300 import inputs
from paper_2508_00577_gb300 import surrogate as S

pytestmark = pytest.mark.gpu


def compare(o_rho, o_u, o_T, g_rho, g_u, g_T, tol):
    er = float(np.max(np.abs(g_rho - o_rho) / o_rho))
    eT = float(np.max(np.abs(g_T - o_T) / o_T))
    eu = float(np.max(np.abs(g_u - o_u)))
    return er, eT, eu


def test_sweep_full_size_in_bench_launch_shape():
    (rho, u, T), nz = bench.workload_fields(E.maxwell, E.critical_point)
    n = bench.NX
    p = ev.lbm_params.make(nx=n, ny=n, nz=nz, eos=ev.LBM_EOS_CS, a=bench.A, b=bench.B, kappa=bench.KAPPA,
                           tau=bench.TAU, precision=ev.LBM_FP32)
    with ev.Lattice(p, rho, u, T) as g:
        tile = ev.lbm_autotune(g.ctx, 1)
    steps = 10
    o = oracle.State(oracle.Params(Q=9, nx=n, ny=n, nz=nz, eos=E.CS, a=bench.A, b=bench.B, kappa=bench.KAPPA,
                                   tau=bench.TAU), rho, u, T)
    o.step(steps)
    orho, ou, oT = o.macro()[:3]
    # The autotuned shape, and both shapes the autotuner chooses between on this workload
    # (128-column strips in 256-row chunks, or the balanced persistent grid).
    for shape in dict.fromkeys([tuple(tile), (128, 256), (128, ev.LBM_TILE_BALANCED)]):
        with ev.Lattice(p, rho, u, T) as g:
            ev.lbm_set_tile(g.ctx, *shape)
            g.step(steps)
            gr, gu, gT, _ = g.moments()
        er, eT, eu = compare(orho, ou, oT, gr, gu, gT, 1e-5)
        print(f"\nsweep 9 x 1024^2, tile {shape}: max rel rho {er:.2e}, T {eT:.2e}, max abs u {eu:.2e}")
        assert er <= 1e-5 and eT <= 1e-5 and eu <= 1e-6, shape


def test_ensemble_full_size_sampled_domains():
    _, Tc = E.critical_point(E.CS, bench.A, bench.B)
    doms = inputs.ensemble_domains(512)
    fields, sizes = [], []
    for dm in doms:
        rv, rl = E.maxwell(E.CS, bench.A, bench.B, dm["tr"] * Tc)
        fields.append(inputs.two_droplets(dm["nx"], dm["ny"], dm["r1"], dm["r2"], dm["gap"], rv, rl, dm["tr"] * Tc))
        sizes.append((dm["nx"], dm["ny"]))
    params = ev.lbm_params.make(eos=ev.LBM_EOS_CS, a=bench.A, b=bench.B, kappa=bench.ENSEMBLE_KAPPA, tau=bench.TAU,
                                precision=ev.LBM_FP32)
    steps = 20
    bt = ev.Batch(params, sizes, [f[0] for f in fields], [f[1] for f in fields], [f[2] for f in fields])
    try:
        bt.autotune(1)          # probes on the live state and restores it (tests/test_gpu_batch.py)
        bt.step(steps)
        for d in (0, 34, 137, 300, 511):
            nx, ny = sizes[d]
            rho, u, T = fields[d]
            o = oracle.State(oracle.Params(Q=9, nx=nx, ny=ny, eos=E.CS, a=bench.A, b=bench.B,
                                           kappa=bench.ENSEMBLE_KAPPA, tau=bench.TAU), rho, u, T)
            o.step(steps)
            orho, ou, oT = o.macro()[:3]
            gr, gu, gT = bt.moments(d)
            er, eT, eu = compare(orho, ou, oT, gr, gu.reshape(2, -1), gT, 1e-5)
            assert er <= 1e-5 and eT <= 1e-5 and eu <= 1e-6, (d, sizes[d], er, eT, eu)
    finally:
        bt.close()


def test_ensemble_full_length_finite_domains():
    """The ensemble workload over its full 5000 steps in one persistent launch: at least
    503 of the 512 domains finite.  Domain 390 (80 x 128, T/Tc 0.703, radii 19.7 and 10,
    gap 3.3) is one the method does not hold: its temperature minimum falls from 0.006 to
    zero within 80 steps and the state diverges near step 90 in the FP64 oracle; run alone
    for 30 steps the GPU matches the oracle, and both have diverged by step 200."""
    _, Tc = E.critical_point(E.CS, bench.A, bench.B)
    doms = inputs.ensemble_domains(512)
    fields, sizes = [], []
    for dm in doms:
        rv, rl = E.maxwell(E.CS, bench.A, bench.B, dm["tr"] * Tc)
        fields.append(inputs.two_droplets(dm["nx"], dm["ny"], dm["r1"], dm["r2"], dm["gap"], rv, rl, dm["tr"] * Tc))
        sizes.append((dm["nx"], dm["ny"]))
    params = ev.lbm_params.make(eos=ev.LBM_EOS_CS, a=bench.A, b=bench.B, kappa=bench.ENSEMBLE_KAPPA, tau=bench.TAU,
                                precision=ev.LBM_FP32)
    bt = ev.Batch(params, sizes, [f[0] for f in fields], [f[1] for f in fields], [f[2] for f in fields])
    try:
        bt.set_tile(128, 256)
        bt.step(bench.ENSEMBLE_STEPS)
        finite = [bool(np.isfinite(bt.moments(d)[0]).all()) for d in range(len(sizes))]
    finally:
        bt.close()
    print(f"\nensemble, {bench.ENSEMBLE_STEPS} steps: {sum(finite)}/512 domains finite; "
          f"non-finite: {[d for d, ok in enumerate(finite) if not ok]}")
    assert sum(finite) >= 503
    assert not finite[390]
    d = 390
    nx, ny = sizes[d]
    p1 = ev.lbm_params.make(nx=nx, ny=ny, eos=ev.LBM_EOS_CS, a=bench.A, b=bench.B, kappa=bench.ENSEMBLE_KAPPA,
                            tau=bench.TAU, precision=ev.LBM_FP32)
    o = oracle.State(oracle.Params(Q=9, nx=nx, ny=ny, eos=E.CS, a=bench.A, b=bench.B, kappa=bench.ENSEMBLE_KAPPA,
                                   tau=bench.TAU), *fields[d])
    with ev.Lattice(p1, *fields[d]) as g:
        o.step(30)
        g.step(30)
        orho, gr = o.macro()[0], g.moments()[0]
        assert np.isfinite(orho).all() and float(np.max(np.abs(gr - orho) / orho)) <= 1e-5
        o.step(170)
        g.step(170)
        assert not np.isfinite(o.macro()[0]).all() and not np.isfinite(g.moments()[0]).all()


N3, STEPS3 = 256, 2


@pytest.fixture(scope="module")
def spinodal3d():
    """Fields, kappa and the FP64 oracle's density after STEPS3 steps (computed once)."""
    _, Tc = E.critical_point(E.CS, bench.A, bench.B)
    RT = 0.85 * Tc
    s1, s2 = E.spinodal(E.CS, bench.A, bench.B, RT)
    kappa = E.kappa_for_width(E.CS, bench.A, bench.B, RT, 4.0)
    fields = inputs.spinodal_noise(N3, N3, N3, 0.5 * (s1 + s2), RT, amplitude=0.01)
    o = oracle.State(oracle.Params(Q=27, nx=N3, ny=N3, nz=N3, eos=E.CS, a=bench.A, b=bench.B, kappa=kappa,
                                   tau=bench.TAU), *fields)
    o.step(STEPS3)
    orho = o.macro()[0]
    del o
    return fields, kappa, orho


@pytest.mark.parametrize("prec,tol", [(ev.LBM_FP32, 1e-5), (ev.LBM_FP16_DEV, 1e-3), (ev.LBM_BF16_DEV, 1e-3)])
def test_spinodal3d_full_size(spinodal3d, prec, tol):
    fields, kappa, orho = spinodal3d
    n, steps = N3, STEPS3
    p = ev.lbm_params.make(lattice=ev.LBM_D3Q27, nx=n, ny=n, nz=n, eos=ev.LBM_EOS_CS, a=bench.A, b=bench.B,
                           kappa=kappa, tau=bench.TAU, precision=prec)
    with ev.Lattice(p, *fields) as g:
        g.step(steps)
        gr = g.moments()[0]
    err = float(np.max(np.abs(gr - orho) / orho))
    print(f"\n256^3 D3Q27, precision {prec}: max rel rho {err:.2e}")
    assert err <= tol


def test_surrogate_full_size_equivariance_and_batch_independence():
    n, B = 256, 32
    r = np.random.default_rng(3)
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    samples = []
    for b in range(B):
        k = r.integers(1, 4, size=(4, 2))
        ph = r.random((4, 2)) * 2 * np.pi
        samples.append(np.stack([np.sin(2 * np.pi * k[c, 0] * yy / n + ph[c, 0]) *
                                 np.cos(2 * np.pi * k[c, 1] * xx / n + ph[c, 1]) for c in range(4)]))
    base = np.stack(samples, 1)                                   # [4][B][n][n]
    scale = np.array([0.05, 0.004, 0.004, 0.0005])[:, None, None, None]
    mean = np.array([0.1, 0.0, 0.0, 0.0075])[:, None, None, None]
    x = (mean + scale * base).astype(np.float32)

    def run(m, fields):
        d = torch.tensor(fields.reshape(4, -1), device="cuda").contiguous()
        out = torch.empty_like(d)
        torch.cuda.synchronize()
        m.infer(d.data_ptr(), out.data_ptr(), B)
        torch.cuda.synchronize()
        return out.cpu().numpy().reshape(4, B, n, n)

    with S.Surrogate(n, n, seed=7) as m:
        m.set_norm(mean.ravel(), scale.ravel(), np.array([0.002, 0.001, 0.001, 8e-5]))
        y0 = run(m, x)
        ys = run(m, np.roll(x, shift=(8, 16), axis=(2, 3)))
        perm = r.permutation(B)
        yp = run(m, x[:, perm])
    assert np.isfinite(y0).all()
    # The same arithmetic on shifted data: exact up to the shift.
    np.testing.assert_array_equal(np.roll(y0, shift=(8, 16), axis=(2, 3)), ys)
    np.testing.assert_array_equal(y0[:, perm], yp)
