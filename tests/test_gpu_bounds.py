"""Bounds-checked build (libevlbm_bc.so, -DEVLBM_BOUNDS_CHECK): the fused kernels compare
every global and shared-memory index they use with the extent of its array, count an
index out of range and skip the access.  Ragged lattices through every launch shape of
the D2Q9 kernel, z-chunks of the D3Q27 kernel that do not divide nz or end on shorter
ones (FP32 and 16-bit storage), 16-bit storage through the D2Q9 kernel, the D2Q9 kernel's wall columns on a
ragged strip, and an ensemble of small
uneven domains must meet no such index, and the checked library must still agree with
the FP64 oracle (1e-5; 1e-3 for 16-bit storage).  The checked library runs in a child process (EVLBM_LIBRARY)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu

CHILD = r'''
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
import oracle, oracle.eos as E
import paper_2508_00577_gb300 as ev
from paper_2508_00577_gb300 import inputs
A, B = 0.1, 4.0
out = {"start": ev.lbm_bounds_violations(), "cases": []}
_, Tc = E.critical_point(E.CS, A, B)
RT = 0.85 * Tc
s1, s2 = E.spinodal(E.CS, A, B, RT)
kappa = E.kappa_for_width(E.CS, A, B, RT, 4.0)

def check(name, o, rho):
    ro = o.macro()[0]
    out["cases"].append((name, float(np.max(np.abs(rho - ro) / ro)), ev.lbm_bounds_violations()))

for (nx, ny, nz) in [(7, 5, 1), (130, 70, 2), (257, 33, 1), (1, 1, 1)]:
    for W in (64, 96, 128, 192):
        for H in (2, 6, 64, ev.LBM_TILE_BALANCED):
            f = inputs.spinodal_noise(nx, ny, nz, 0.5 * (s1 + s2), RT, amplitude=0.05, D=2)
            p = ev.lbm_params.make(nx=nx, ny=ny, nz=nz, eos=ev.LBM_EOS_CS, a=A, b=B, kappa=kappa, precision=ev.LBM_FP32)
            with ev.Lattice(p, *f) as g:
                ev.lbm_set_tile(g.ctx, W, H)
                g.step(5)
                rho = g.moments()[0]
            o = oracle.State(oracle.Params(Q=9, nx=nx, ny=ny, nz=nz, eos=E.CS, a=A, b=B, kappa=kappa, tau=0.3), *f)
            o.step(5)
            check(f"d2q9 {nx}x{ny}x{nz} W{W} H{H}", o, rho)
for (nx, ny, nz, hz) in [(20, 18, 11, 4), (33, 16, 7, 3), (5, 3, 4, 1), (17, 17, 17, 64), (20, 18, 50, 17)]:
    f = inputs.spinodal_noise(nx, ny, nz, 0.5 * (s1 + s2), RT, amplitude=0.05, D=3)
    p = ev.lbm_params.make(lattice=ev.LBM_D3Q27, nx=nx, ny=ny, nz=nz, eos=ev.LBM_EOS_CS, a=A, b=B, kappa=kappa,
                           precision=ev.LBM_FP32)
    with ev.Lattice(p, *f) as g:
        ev.lbm_set_tile(g.ctx, 0, hz)
        g.step(4)
        rho = g.moments()[0]
    o = oracle.State(oracle.Params(Q=27, nx=nx, ny=ny, nz=nz, eos=E.CS, a=A, b=B, kappa=kappa, tau=0.3), *f)
    o.step(4)
    check(f"d3q27 {nx}x{ny}x{nz} z-chunk {hz}", o, rho)
    if hz in (4, 1, 17):
        # 16-bit deviation storage through the same fused kernel (its TMEM stash included)
        for prec, tag in ((ev.LBM_FP16_DEV, "fp16"), (ev.LBM_BF16_DEV, "bf16")):
            p16 = ev.lbm_params.make(lattice=ev.LBM_D3Q27, nx=nx, ny=ny, nz=nz, eos=ev.LBM_EOS_CS, a=A, b=B,
                                     kappa=kappa, precision=prec)
            with ev.Lattice(p16, *f) as g:
                ev.lbm_set_tile(g.ctx, 0, hz)
                g.step(4)
                check(f"d3q27 {tag} {nx}x{ny}x{nz} z-chunk {hz}", o, g.moments()[0])
# 16-bit storage through the fused D2Q9 kernel: ragged strips, a chunk height that does not
# divide ny, the balanced grid.
for (nx, ny, nz) in [(130, 70, 2), (7, 5, 1)]:
    for W, H in ((128, 6), (64, ev.LBM_TILE_BALANCED)):
        f = inputs.spinodal_noise(nx, ny, nz, 0.5 * (s1 + s2), RT, amplitude=0.05, D=2)
        o = oracle.State(oracle.Params(Q=9, nx=nx, ny=ny, nz=nz, eos=E.CS, a=A, b=B, kappa=kappa, tau=0.3), *f)
        o.step(5)
        for prec, tag in ((ev.LBM_FP16_DEV, "fp16"), (ev.LBM_BF16_DEV, "bf16")):
            p16 = ev.lbm_params.make(nx=nx, ny=ny, nz=nz, eos=ev.LBM_EOS_CS, a=A, b=B, kappa=kappa, precision=prec)
            with ev.Lattice(p16, *f) as g:
                ev.lbm_set_tile(g.ctx, W, H)
                g.step(5)
                check(f"d2q9 {tag} {nx}x{ny}x{nz} W{W} H{H}", o, g.moments()[0])
# Wall columns of the fused D2Q9 kernel (thermal Couette set-up, kappa = 0), ragged strip.
for H in (4, ev.LBM_TILE_BALANCED):
    nx, ny = 33, 5
    y = np.repeat(np.arange(ny), nx)
    x = np.tile(np.arange(nx), ny)
    rho0 = 1.0 + 0.01 * np.sin(2 * np.pi * y / ny) * np.sin(np.pi * x / (nx - 1))
    u0 = np.zeros((2, nx * ny))
    u0[1, x == nx - 1] = 0.3
    T0 = np.full(nx * ny, 0.2)
    walls = ((0, 0, 0), (0, 0.3, 0), 0.2)
    p = ev.lbm_params.make(nx=nx, ny=ny, eos=ev.LBM_EOS_VDW, a=0.05, b=0.1, kappa=0.0, tau=0.5, thermal=1,
                           precision=ev.LBM_FP32)
    with ev.Lattice(p, rho0, u0, T0) as g:
        ev.lbm_set_walls(g.ctx, 1, *walls)
        ev.lbm_set_tile(g.ctx, 128, H)
        g.step(20)
        rho = g.moments()[0]
    o = oracle.State(oracle.Params(Q=9, nx=nx, ny=ny, eos=E.VDW, a=0.05, b=0.1, kappa=0.0, tau=0.5, thermal=1,
                                   walls=walls), rho0, u0, T0)
    o.step(20)
    check(f"d2q9 walls {nx}x{ny} H{H}", o, rho)
doms = inputs.ensemble_domains(12, seed=9, side_min=64, side_max=208, tr_range=(0.85, 0.9))
fields, sizes = [], []
for dm in doms:
    rv, rl = E.maxwell(E.CS, A, B, dm["tr"] * Tc)
    fields.append(inputs.two_droplets(dm["nx"], dm["ny"], dm["r1"], dm["r2"], dm["gap"], rv, rl, dm["tr"] * Tc))
    sizes.append((dm["nx"], dm["ny"]))
p = ev.lbm_params.make(eos=ev.LBM_EOS_CS, a=A, b=B, kappa=0.116, tau=0.3, precision=ev.LBM_FP32)
bt = ev.Batch(p, sizes, [f[0] for f in fields], [f[1] for f in fields], [f[2] for f in fields])
bt.set_tile(64, 32)
bt.step(6)
for d in (0, 5, 11):
    o = oracle.State(oracle.Params(Q=9, nx=sizes[d][0], ny=sizes[d][1], eos=E.CS, a=A, b=B, kappa=0.116, tau=0.3),
                     *fields[d])
    o.step(6)
    check(f"ensemble domain {d} {sizes[d]}", o, bt.moments(d)[0])
bt.close()
print("RESULT " + json.dumps(out))
'''


def test_checked_library_meets_no_out_of_range_index():
    from paper_2508_00577_gb300 import _build
    lib = _build.build(bounds_check=True)
    env = dict(os.environ, EVLBM_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + CHILD], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.split("RESULT ", 1)[1])
    assert res["start"] == 0
    assert len(res["cases"]) == 4 * 4 * 4 + 5 + 3 * 2 + 2 * 2 * 2 + 2 + 3
    for name, err, oob in res["cases"]:
        assert oob == 0, f"{name}: {oob} out-of-range indices"
        assert err <= (1e-3 if ("fp16" in name or "bf16" in name) else 1e-5), f"{name}: max rel rho error {err}"
