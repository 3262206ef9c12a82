"""The seeded input generators shared by the CUDA path and the oracle
(paper_2508_00577_gb300/inputs.py): the counter-based random numbers against the
published SplitMix64 outputs (tests/golden/splitmix64.txt), and the geometry of the
synthetic initial states."""
import pathlib

import numpy as np

from paper_2508_00577_gb300 import inputs

GOLDEN = pathlib.Path(__file__).parent / "golden" / "splitmix64.txt"
GAMMA = 0x9E3779B97F4A7C15
MASK = (1 << 64) - 1


def test_splitmix64_matches_published_outputs():
    rows = [l.split() for l in GOLDEN.read_text().splitlines() if l.strip() and not l.startswith("#")]
    assert len(rows) == 2
    for seed, *outs in rows:
        s = int(seed, 0)
        for k, out in enumerate(outs):
            assert int(inputs.splitmix64((s + k * GAMMA) & MASK)) == int(out, 0)


def test_uniform01_range_and_moments():
    u = inputs.uniform01(inputs.DEFAULT_SEED, 1 << 20)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 2e-3 and abs(u.var() - 1 / 12) < 2e-3
    assert np.array_equal(u, inputs.uniform01(inputs.DEFAULT_SEED, 1 << 20))      # counter based
    assert not np.array_equal(u[:1000], inputs.uniform01(inputs.DEFAULT_SEED + 1, 1000))


def test_tanh_profile_and_slab_symmetry():
    assert inputs.tanh_profile(0.0, 1.0, 3.0) == 2.0
    rho, u, T = inputs.slab(64, 4, 0.1, 1.0, 0.5, thickness=32.0, width=4.0)
    r = rho.reshape(4, 64)
    assert np.allclose(r, r[:, ::-1]) and np.all(u == 0) and np.all(T == 0.5)
    assert r[0, 32] > 0.99 and r[0, 0] < 0.11


def test_two_droplets_pair_is_centred_and_clear_of_the_boundary():
    nx, ny, r1, r2, gap = 200, 120, 30.0, 10.0, 5.0
    rho = inputs.two_droplets(nx, ny, r1, r2, gap, 0.1, 1.0, 0.5)[0].reshape(ny, nx)
    row = rho[(ny - 1) // 2]
    dense = np.nonzero(row > 0.55)[0]                       # nodes inside either droplet
    left_edge, right_edge = dense.min(), dense.max()
    assert abs(0.5 * (left_edge + right_edge) - 0.5 * (nx - 1)) <= 1.0
    assert right_edge - left_edge + 1 >= 2 * (r1 + r2) + gap - 2
    assert row[0] < 0.11 and row[-1] < 0.11
    c_gap = int(round(0.5 * (nx - 1) - 0.5 * (2 * r1 + gap + 2 * r2) + 2 * r1 + 0.5 * gap))
    assert row[c_gap] < 0.55                               # the gap is open


def test_ensemble_domains_follow_the_recipe():
    doms = inputs.ensemble_domains(512)
    assert doms == inputs.ensemble_domains(512)            # seeded
    sides = set(range(64, 513, 16))
    for d in doms:
        assert d["nx"] in sides and d["ny"] in sides
        assert 2.0 <= d["gap"] <= 10.0 and 0.7 <= d["tr"] <= 0.9
        assert 2 * (d["r1"] + d["r2"]) + d["gap"] + 16 <= d["nx"] + 1e-9
        assert 2 * max(d["r1"], d["r2"]) + 8 <= d["ny"] + 1e-9
    nodes = sum(d["nx"] * d["ny"] for d in doms)
    assert nodes == 41311232                               # the ensemble workload's node count
