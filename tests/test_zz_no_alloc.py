"""lbm_step_noalloc: the FP64 step for callers that cannot allocate device memory
while they run.  Its populations, over two calls in a row, must equal those of
the allocating entry point (lbm_step on an FP64 context) bit for bit -- the
tolerance the FP64 parity tests use.  This file is collected last on purpose."""
import numpy as np
import pytest

import oracle.eos as E
import paper_2508_00577_gb300 as ev
from paper_2508_00577_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("lattice,nx,ny,nz,thermal", [(ev.LBM_D2Q9, 40, 32, 1, 1), (ev.LBM_D3Q27, 12, 10, 9, 0)])
def test_noalloc_matches_allocating_step(lattice, nx, ny, nz, thermal):
    torch = pytest.importorskip("torch")
    a, b = 0.1, 4.0
    _, Tc = E.critical_point(E.CS, a, b)
    RT = 0.85 * Tc
    rv, rl = E.maxwell(E.CS, a, b, RT)
    kappa = E.kappa_for_width(E.CS, a, b, RT, 4.0)
    D = 2 if lattice == ev.LBM_D2Q9 else 3
    s1, s2 = E.spinodal(E.CS, a, b, RT)
    rho, u, T = inputs.spinodal_noise(nx, ny, nz, 0.5 * (s1 + s2), RT, amplitude=0.01, D=D)
    p = ev.lbm_params.make(lattice=lattice, nx=nx, ny=ny, nz=nz, eos=ev.LBM_EOS_CS, a=a, b=b, kappa=kappa,
                           thermal=thermal, precision=ev.LBM_FP64)
    with ev.Lattice(p, rho, u, T) as ref:
        f0, g0 = ref.populations()
        dev = torch.device("cuda")
        fa = torch.from_numpy(f0.copy()).to(dev)
        fb = torch.empty_like(fa)
        if thermal:
            ga = torch.from_numpy(g0.copy()).to(dev)
            gb = torch.empty_like(ga)
            rt = None
        else:
            ga = gb = None
            rt = torch.from_numpy(p.R * np.asarray(T, dtype=np.float64)).to(dev)
        st = torch.cuda.current_stream().cuda_stream
        ptr = lambda x: x.data_ptr() if x is not None else 0
        # two calls in a row: a -> b -> a
        ev.lbm_step_noalloc(p, ptr(fa), ptr(ga), ptr(rt), ptr(fb), ptr(gb), st)
        ev.lbm_step_noalloc(p, ptr(fb), ptr(gb), ptr(rt), ptr(fa), ptr(ga), st)
        torch.cuda.synchronize()
        ref.step(2)
        f_ref, g_ref = ref.populations()
        assert np.array_equal(fa.cpu().numpy(), f_ref)
        if thermal:
            assert np.array_equal(ga.cpu().numpy(), g_ref)


def test_noalloc_rejects_oversize_lattice():
    p = ev.lbm_params.make(nx=256, ny=256, precision=ev.LBM_FP64)
    with pytest.raises(ev.LBMError) as e:
        ev.lbm_step_noalloc(p, 1, 1, 0, 1, 1, 0)
    assert e.value.code == ev.LBM_EINVAL
