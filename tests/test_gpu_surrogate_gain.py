"""What the trained surrogate gains over the lattice Boltzmann method alone.

Trained with the project's own kernels on lattice Boltzmann trajectories of
droplet-pair domains (256^2, 50-step windows), evaluated on held-out domains:

* accuracy: on a held-out validation batch the network's loss (mean squared
  error of the normalised increment) must be below 0.25 -- predicting no change
  (persistence) scores about 1 -- and its one-window density error must be below
  half of persistence's;
* cost: one surrogate window (inference of the batch) must take less time than the
  50 lattice Boltzmann steps it replaces, on the same batch.

The long-horizon rollout error is reported (run with -s), not asserted: after
100 autoregressive windows the surrogate alone drifts far beyond 1e-2."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2508_00577_gb300 as ev
from paper_2508_00577_gb300 import inputs
from paper_2508_00577_gb300 import surrogate as S

pytestmark = pytest.mark.gpu

A, B, KAPPA, TAU = 0.1, 4.0, 0.2, 0.3
N1, STEPS, WIN = 256, 50, 40
dev = "cuda"


def trajectories(doms, Tc):
    nd, Mb = len(doms), N1 * N1
    N = nd * Mb
    rho, T = [], []
    for dm in doms:
        rv, rl = ev.lbm_coexistence(1, A, B, dm["tr"] * Tc)
        r, _, t = inputs.two_droplets(N1, N1, dm["r1"], dm["r2"], dm["gap"], rv, rl, dm["tr"] * Tc)
        rho.append(r)
        T.append(t)
    rho, T = np.concatenate(rho), np.concatenate(T)
    p = ev.lbm_params.make(nx=N1, ny=N1, nz=nd, eos=ev.LBM_EOS_CS, a=A, b=B, kappa=KAPPA, tau=TAU,
                           precision=ev.LBM_FP32)
    snaps = torch.empty((WIN + 1, 4, N), device=dev)
    with ev.Lattice(p, rho, np.zeros((2, N)), T) as g:
        for w in range(WIN + 1):
            if w:
                g.step(STEPS)
            base = snaps.data_ptr() + w * 16 * N
            ev.lbm_moments_device(g.ctx, base, base + 4 * N, base + 12 * N)
        ev.lbm_sync(g.ctx)
        # Time one lattice Boltzmann window of this batch.
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.step(STEPS)
        ev.lbm_sync(g.ctx)
        t_lb = time.perf_counter() - t0
    torch.cuda.synchronize()
    return snaps.reshape(WIN + 1, 4, nd, Mb), t_lb


def test_surrogate_beats_persistence_and_is_cheaper_than_lb():
    _, Tc = ev.lbm_critical_point(1, A, B)
    train, _ = trajectories(inputs.ensemble_domains(32, seed=11, side_min=N1, side_max=N1), Tc)
    test, t_lb = trajectories(inputs.ensemble_domains(16, seed=12, side_min=N1, side_max=N1), Tc)
    x, y = train[:-1], train[1:]
    mean = x.mean(dim=(0, 2, 3)).cpu().numpy()
    scale = x.std(dim=(0, 2, 3)).cpu().numpy()
    oscale = (y - x).std(dim=(0, 2, 3)).cpu().numpy()
    bs, steps = 16, 1500

    def batch(v, w, d):
        w = torch.as_tensor(w, device=dev)
        d = torch.as_tensor(d, device=dev)
        return (v[w, :, d, :].permute(1, 0, 2).reshape(4, -1).contiguous(),
                v[w + 1, :, d, :].permute(1, 0, 2).reshape(4, -1).contiguous())

    rng = np.random.default_rng(0)
    vx, vy = batch(test, np.arange(0, WIN, WIN // bs)[:bs], np.arange(bs))
    with S.Surrogate(N1, N1, seed=3) as m:
        m.set_norm(mean, scale, oscale)
        for it in range(steps):
            xb, yb = batch(train, rng.integers(0, WIN, bs), rng.integers(0, 32, bs))
            torch.cuda.synchronize()
            lr = 3e-4 * min(1.0, (it + 1) / 200) * 0.5 * (1 + np.cos(np.pi * it / steps))
            m.train_step(xb.data_ptr(), yb.data_ptr(), bs, float(lr), want_loss=False)
        val = m.forward_backward(vx.data_ptr(), vy.data_ptr(), bs)
        pred = torch.empty_like(vx)
        m.infer(vx.data_ptr(), pred.data_ptr(), bs)
        torch.cuda.synchronize()
        err = float((pred[0] - vy[0]).norm() / vy[0].norm())
        pers = float((vx[0] - vy[0]).norm() / vy[0].norm())
        # Cost of one window: inference of the 16 test domains vs 50 lattice Boltzmann steps of them.
        x16 = test[0].reshape(4, -1).contiguous()
        o16 = torch.empty_like(x16)
        for _ in range(3):
            m.infer(x16.data_ptr(), o16.data_ptr(), 16)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(10):
            m.infer(x16.data_ptr(), o16.data_ptr(), 16)
        torch.cuda.synchronize()
        t_inf = (time.perf_counter() - t0) / 10
        # Rollout of the held-out domains by the surrogate alone, against the lattice Boltzmann run.
        d = x16.clone()
        tmp = torch.empty_like(d)
        for _ in range(WIN):
            m.infer(d.data_ptr(), tmp.data_ptr(), 16)
            torch.cuda.synchronize()
            d.copy_(tmp)
        ref = test[WIN].reshape(4, -1)
        roll = float((d[0] - ref[0]).norm() / ref[0].norm())
    print(f"\nvalidation loss {val:.4f} (persistence ~1); one-window rho error {err:.3e} vs persistence {pers:.3e}; "
          f"window cost: surrogate {t_inf * 1e3:.2f} ms vs lattice Boltzmann {t_lb * 1e3:.2f} ms "
          f"({t_lb / t_inf:.2f}x); {WIN}-window surrogate-only rollout rho error {roll:.3e}")
    assert val < 0.25
    assert err < 0.5 * pers
    assert t_inf < t_lb
