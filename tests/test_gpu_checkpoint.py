"""Checkpoint and resume (lbm_save / lbm_load): a run that is saved after k steps and
resumed in a fresh context continues bit for bit like the run that never stopped, for
every storage type, both lattices and the frozen-temperature mode; files that do not
fit the context are rejected with the field named."""
import os

import numpy as np
import pytest

import oracle.eos as E
import paper_2508_00577_gb300 as ev
from paper_2508_00577_gb300 import inputs

pytestmark = pytest.mark.gpu

A, B = 0.1, 4.0


def state(lattice, nx, ny, nz, seed):
    _, Tc = E.critical_point(E.CS, A, B)
    RT = 0.85 * Tc
    s1, s2 = E.spinodal(E.CS, A, B, RT)
    kappa = E.kappa_for_width(E.CS, A, B, RT, 4.0)
    D = 2 if lattice == ev.LBM_D2Q9 else 3
    fields = inputs.spinodal_noise(nx, ny, nz, 0.5 * (s1 + s2), RT, amplitude=0.05, seed=seed, D=D)
    return fields, kappa


@pytest.mark.parametrize("lattice,nx,ny,nz,precision,thermal", [
    (ev.LBM_D2Q9, 70, 48, 1, ev.LBM_FP64, 1),
    (ev.LBM_D2Q9, 130, 66, 2, ev.LBM_FP32, 1),
    (ev.LBM_D2Q9, 64, 40, 1, ev.LBM_FP32, 0),
    (ev.LBM_D2Q9, 48, 40, 1, ev.LBM_FP16_DEV, 1),
    (ev.LBM_D2Q9, 48, 40, 1, ev.LBM_BF16_DEV, 0),
    (ev.LBM_D3Q27, 20, 18, 11, ev.LBM_FP32, 1),
    (ev.LBM_D3Q27, 12, 10, 9, ev.LBM_FP64, 0),
])
def test_resume_is_bit_identical(tmp_path, lattice, nx, ny, nz, precision, thermal):
    fields, kappa = state(lattice, nx, ny, nz, seed=11)
    p = ev.lbm_params.make(lattice=lattice, nx=nx, ny=ny, nz=nz, eos=ev.LBM_EOS_CS, a=A, b=B, kappa=kappa,
                           thermal=thermal, precision=precision)
    path = str(tmp_path / "run.ckpt")
    with ev.Lattice(p, *fields) as run:
        run.step(7)
        run.save(path)
        assert not os.path.exists(path + ".tmp")
        run.step(9)
        f_ref, g_ref = run.populations()
        steps_ref = ev.lbm_step_count(run.ctx)
    other, _ = state(lattice, nx, ny, nz, seed=12)                # different initial fields
    with ev.Lattice(p, *other) as resumed:
        resumed.load(path)
        assert ev.lbm_step_count(resumed.ctx) == 7
        resumed.step(9)
        f, g = resumed.populations()
        assert ev.lbm_step_count(resumed.ctx) == steps_ref
    assert np.array_equal(f, f_ref)
    if thermal:
        assert np.array_equal(g, g_ref)


def test_mismatched_or_damaged_checkpoints_are_rejected(tmp_path):
    fields, kappa = state(ev.LBM_D2Q9, 40, 32, 1, seed=3)
    p = ev.lbm_params.make(nx=40, ny=32, eos=ev.LBM_EOS_CS, a=A, b=B, kappa=kappa, precision=ev.LBM_FP32)
    path = str(tmp_path / "a.ckpt")
    with ev.Lattice(p, *fields) as g:
        g.step(3)
        g.save(path)
    size = os.path.getsize(path)
    assert size == 136 + 2 * 9 * 40 * 32 * 4                    # header + f and g in FP32

    q = ev.lbm_params.make(nx=40, ny=32, eos=ev.LBM_EOS_CS, a=A, b=B, kappa=kappa * 1.5, precision=ev.LBM_FP32)
    with ev.Lattice(q, *fields) as g:
        with pytest.raises(ev.LBMError) as e:
            g.load(path)
        assert e.value.code == ev.LBM_EINVAL and "kappa" in str(e.value)
    r = ev.lbm_params.make(nx=40, ny=32, eos=ev.LBM_EOS_CS, a=A, b=B, kappa=kappa, precision=ev.LBM_FP64)
    with ev.Lattice(r, *fields) as g:
        with pytest.raises(ev.LBMError) as e:
            g.load(path)
        assert e.value.code == ev.LBM_EINVAL and "precision" in str(e.value)

    with ev.Lattice(p, *fields) as g:
        data = open(path, "rb").read()
        cut = str(tmp_path / "cut.ckpt")
        open(cut, "wb").write(data[:-4])
        with pytest.raises(ev.LBMError) as e:
            g.load(cut)
        assert e.value.code == ev.LBM_EIO
        bad = str(tmp_path / "bad.ckpt")
        open(bad, "wb").write(b"NOTACKPT" + data[8:])
        with pytest.raises(ev.LBMError) as e:
            g.load(bad)
        assert e.value.code == ev.LBM_EINVAL
        with pytest.raises(ev.LBMError) as e:
            g.load(str(tmp_path / "missing.ckpt"))
        assert e.value.code == ev.LBM_EIO
        assert ev.lbm_step_count(g.ctx) == 0                      # nothing was loaded
