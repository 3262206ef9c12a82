"""The oracle's operation count per lattice update (oracle/flopcount.cpp: the oracle's
source compiled with a counting number type), and the values bench.py reports from it."""
import subprocess

import oracle
import bench


def test_counter_counts_each_arithmetic_operation():
    """(a b + c)/d - e, then x += y, x *= 2, x = -x: 6 operations (negation is not one),
    and the counted type computes the same value as plain doubles."""
    oracle.build()
    ops, val = subprocess.check_output([oracle._FC_PATH, "selftest"], text=True).split()
    assert int(ops) == 6
    assert float(val) == -(3.0 + ((1.5 * 2.0 + 0.25) / 4.0 - 1.0)) * 2.0


def test_counts_are_per_node_and_ordered():
    """The count is affine in the node count (checked on three lattices inside
    flops_per_update); removing the g population, the divergence form or a dimension
    each lowers it."""
    d2t = oracle.flops_per_update(9, 1, 1, 0)
    assert oracle.flops_per_update(9, 0, 1, 0) < d2t
    assert oracle.flops_per_update(9, 1, 1, 1) < d2t            # literal force: no stress tensor
    assert oracle.flops_per_update(9, 1, 0, 0) < d2t            # vdW EOS is cheaper than CS
    assert oracle.flops_per_update(27, 1, 1, 0) > 3 * d2t


def test_bench_reports_the_counted_values():
    assert bench.ORACLE_FLOPS_PER_LU["d2q9_thermal"] == oracle.flops_per_update(9, 1, 1, 0)
    assert bench.ORACLE_FLOPS_PER_LU["d3q27_thermal"] == oracle.flops_per_update(27, 1, 1, 0)


def test_alu_check_arithmetic():
    """bench.alu_check: peak = 2 x 152 x 128 lanes x clock; operations per second =
    operations per update x updates per second."""
    r = bench.alu_check(1000.0, 2000, 2000.0)          # 1 GLUPS, 2000 ops per update, 2 GHz
    assert r["fp32_peak_tflops"] == 2 * 152 * 128 * 2.0e9 / 1e12
    assert abs(r["oracle_equivalent_tflops"] - 2.0) < 1e-12
    assert abs(r["frac"] - 2.0 / r["fp32_peak_tflops"]) < 1e-12
    assert abs(r["alu_bound_mlups_at_oracle_flops"] - r["fp32_peak_tflops"] * 1e12 / 2000 / 1e6) < 1e-6
