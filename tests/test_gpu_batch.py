"""Batched ensembles (persistent kernel under a CUDA graph): each domain matches a
single-domain context bit for bit at the same launch shape and the FP64 oracle
within the FP32 tolerance; autotuning keeps the state; a wait that gives up is
reported as LBM_ETIMEOUT and the batch stays usable."""
import numpy as np
import pytest

import oracle
import oracle.eos as E
import paper_2508_00577_gb300 as ev
from paper_2508_00577_gb300 import inputs

pytestmark = pytest.mark.gpu

A, B = 0.1, 4.0
SIZES = [(96, 80), (64, 144), (130, 70), (200, 96), (48, 40), (7, 5)]


def ensemble(sizes, thermal=1, seed=3):
    _, Tc = E.critical_point(E.CS, A, B)
    rng = np.random.default_rng(seed)
    fields = []
    for nx, ny in sizes:
        tr = float(rng.uniform(0.75, 0.9))
        RT = tr * Tc
        rv, rl = E.maxwell(E.CS, A, B, RT)
        r1 = max(2.0, 0.15 * min(nx, ny))
        fields.append(inputs.two_droplets(nx, ny, r1, 0.8 * r1, 3.0, rv, rl, RT))
    kappa = E.kappa_for_width(E.CS, A, B, 0.8 * Tc, 4.0)
    p = ev.lbm_params.make(eos=ev.LBM_EOS_CS, a=A, b=B, kappa=kappa, thermal=thermal, precision=ev.LBM_FP32)
    return p, fields, kappa


@pytest.mark.parametrize("thermal", [1, 0])
def test_batch_matches_single_domains_and_oracle(thermal):
    p, fields, kappa = ensemble(SIZES, thermal)
    rho = [f[0] for f in fields]
    u = [f[1] for f in fields]
    T = [f[2] for f in fields]
    with ev.Batch(p, SIZES, rho, u, T) as bt:
        bt.set_tile(128, 64)
        bt.step(17)          # one persistent launch
        bt.step(13)          # odd counts: buffer parity flips between calls
        for d, (nx, ny) in enumerate(SIZES):
            r_b, u_b, T_b = bt.moments(d)
            sp = ev.lbm_params.make(nx=nx, ny=ny, eos=ev.LBM_EOS_CS, a=A, b=B, kappa=kappa, thermal=thermal,
                                    precision=ev.LBM_FP32)
            with ev.Lattice(sp, *fields[d]) as one:
                ev.lbm_set_tile(one.ctx, 128, 64)
                one.step(30)
                r_1, u_1, T_1, _ = one.moments()
            assert np.array_equal(r_b, r_1), d
            assert np.array_equal(u_b, u_1), d
            o = oracle.State(oracle.Params(Q=9, nx=nx, ny=ny, eos=E.CS, a=A, b=B, kappa=kappa, tau=0.3,
                                           thermal=thermal), *fields[d])
            o.step(30)
            ro = o.macro()[0]
            assert np.max(np.abs(r_b - ro) / ro) <= 1e-5, d


def test_batch_autotune_keeps_state():
    p, fields, _ = ensemble(SIZES[:4])
    with ev.Batch(p, SIZES[:4], [f[0] for f in fields], [f[1] for f in fields], [f[2] for f in fields]) as bt:
        bt.step(4)
        before = [bt.moments(d)[0] for d in range(4)]
        w, h = bt.autotune(1)
        assert w in (64, 96, 128, 192) and h >= 1
        after = [bt.moments(d)[0] for d in range(4)]
        for x, y in zip(before, after):
            assert np.array_equal(x, y)
        bt.step(3)
        assert all(np.isfinite(bt.moments(d)[0]).all() for d in range(4))


def test_batch_wait_timeout_is_reported():
    """Every item waits on a flag nothing sets; the bounded wait gives up, the launch
    ends, LBM_ETIMEOUT is returned and the batch runs again once the probe is off."""
    p, fields, _ = ensemble(SIZES[:3])
    with ev.Batch(p, SIZES[:3], [f[0] for f in fields], [f[1] for f in fields], [f[2] for f in fields]) as bt:
        bt.set_wait_limit(2000, probe_unset_flag=1)
        with pytest.raises(ev.LBMError) as e:
            bt.step(2)
        assert e.value.code == ev.LBM_ETIMEOUT
        bt.set_wait_limit(1 << 24, probe_unset_flag=0)
        bt.step(2)
        assert np.isfinite(bt.moments(0)[0]).all()


def test_batch_rejects_unsupported():
    p, fields, _ = ensemble(SIZES[:1])
    p.precision = ev.LBM_FP64
    with pytest.raises(ev.LBMError):
        ev.Batch(p, SIZES[:1], [fields[0][0]], [fields[0][1]], [fields[0][2]])
