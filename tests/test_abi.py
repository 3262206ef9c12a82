"""The C ABI library builds, loads and exports every symbol include/evlbm.h declares;
argument validation happens on the host before any GPU work (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle.eos as E
import paper_2508_00577_gb300 as ev

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "evlbm.h")
SUR_HEADER = os.path.join(ROOT, "include", "evsur.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:int|long long|const char \*)\s*(lbm_\w+)\s*\(", text, re.M)))


def test_header_declares_the_binding_names():
    assert declared_symbols() == sorted(ev.EXPORTED_SYMBOLS)


def test_surrogate_header_declares_the_binding_names():
    from paper_2508_00577_gb300 import surrogate as S
    text = open(SUR_HEADER).read()
    names = sorted(set(re.findall(r"^(?:int|long long|const char \*)\s*(sur_\w+)\s*\(", text, re.M)))
    assert names == sorted(S.EXPORTED_SYMBOLS)
    L = S.lib()
    for name in names:
        assert hasattr(L, name), name


def test_surrogate_structs_match_header():
    """Field order of sur_operand, sur_gemm_args and sur_rollout_cfg as in the header."""
    from paper_2508_00577_gb300 import surrogate as S
    text = open(SUR_HEADER).read()
    for cname, cls in (("sur_operand", S.sur_operand), ("sur_gemm_args", S.sur_gemm_args),
                       ("sur_rollout_cfg", S.sur_rollout_cfg)):
        body = text[text.index(f"typedef struct {cname} {{"):text.index(f"}} {cname};")]
        body = body[body.index("{") + 1:]
        flat = []
        for decl in re.findall(r"^\s*(?:const\s+)?(?:int|float|void|sur_operand)\s*\**\s*([\w, *]+);", body, re.M):
            flat += [n.strip().lstrip("*") for n in decl.split(",")]
        assert [f[0] for f in cls._fields_] == flat, cname


def test_surrogate_layout_matches_oracle():
    from paper_2508_00577_gb300 import surrogate as S
    import oracle.unet as U
    layout, n = S.param_layout()
    assert n == U.unpack(np.zeros(n))["_n"]


def test_library_exports_every_declared_symbol():
    L = ev.lib()
    for name in declared_symbols():
        assert hasattr(L, name), name


def test_params_struct_matches_header():
    """Field order and types of lbm_params as in the header."""
    text = open(HEADER).read()
    body = text[text.index("typedef struct {"):text.index("} lbm_params;")]
    names = re.findall(r"^\s*(?:int|double)\s+([\w, ]+);", body, re.M)
    flat = [n.strip() for group in names for n in group.split(",")]
    assert [f[0].rstrip("_") for f in ev.lbm_params._fields_] == flat


@pytest.mark.parametrize("field,value", [("nx", 0), ("lattice", 5), ("tau", 0.0), ("lambda_", -1.0),
                                         ("precision", 7), ("R", 0.0), ("thermal", 3), ("eos", 9)])
def test_invalid_params_rejected_on_host(field, value):
    p = ev.lbm_params.make(nx=4, ny=4)
    setattr(p, field, value)
    N = 16
    with pytest.raises(ev.LBMError) as e:
        ev.lbm_init(p, np.ones(N), np.zeros((2, N)), np.ones(N))
    assert e.value.code == ev.LBM_EINVAL
    assert ev.lbm_last_error(None)


def test_init_without_a_gpu_fails_cleanly():
    """The initial fields are checked on the device (tests/test_gpu_parity.py covers the
    check); without a usable GPU lbm_init returns LBM_ECUDA with a message, whatever the
    fields, and leaves nothing allocated."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = ev.lbm_params.make(nx=4, ny=4)
    rho = np.ones(16)
    rho[5] = -1.0
    for r in (rho, np.ones(16)):
        with pytest.raises(ev.LBMError) as e:
            ev.lbm_init(p, r, np.zeros((2, 16)), np.ones(16))
        assert e.value.code == ev.LBM_ECUDA
        assert ev.lbm_last_error(None)


def test_bounds_check_query():
    """The default library has no bounds checks (-1); the checked variant, when built,
    loads and exports every declared symbol."""
    assert ev.lib().lbm_bounds_violations() == -1
    from paper_2508_00577_gb300 import _build
    if not os.path.exists(_build.LIB_BC):
        pytest.skip("bounds-checked library not built")
    L = ctypes.CDLL(_build.LIB_BC)
    for name in declared_symbols():
        assert hasattr(L, name), name


def test_null_context_is_invalid():
    L = ev.lib()
    assert L.lbm_step(None, 1) == ev.LBM_EINVAL
    assert L.lbm_free(None) == ev.LBM_OK
    assert L.lbm_step_count(None) == -1
    assert L.lbm_save(None, b"x.ckpt") == ev.LBM_EINVAL
    assert L.lbm_load(None, b"x.ckpt") == ev.LBM_EINVAL


@pytest.mark.parametrize("eos,a,b", [(ev.LBM_EOS_CS, 0.1, 4.0), (ev.LBM_EOS_VDW, 9 / 392, 2 / 21)])
def test_critical_point_host(eos, a, b):
    rc, Tc = ev.lbm_critical_point(eos, a, b)
    orc, oTc = E.critical_point(eos, a, b)
    assert rc == pytest.approx(orc, rel=1e-10)
    assert Tc == pytest.approx(oTc, rel=1e-10)


@pytest.mark.parametrize("eos,a,b", [(ev.LBM_EOS_CS, 0.1, 4.0), (ev.LBM_EOS_VDW, 9 / 392, 2 / 21)])
def test_spinodal_host(eos, a, b):
    """lbm_spinodal is a host computation: checked against the oracle without a GPU."""
    _, Tc = E.critical_point(eos, a, b)
    for tr in (0.6, 0.8, 0.95):
        s1, s2 = ev.lbm_spinodal(eos, a, b, tr * Tc)
        o1, o2 = E.spinodal(eos, a, b, tr * Tc)
        assert s1 == pytest.approx(o1, rel=1e-12) and s2 == pytest.approx(o2, rel=1e-12)


def test_thermo_helpers_reject_invalid_arguments_on_host():
    _, Tc = ev.lbm_critical_point(ev.LBM_EOS_CS, 0.1, 4.0)
    L = ev.lib()
    out = np.zeros(2)
    ptr = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert L.lbm_spinodal(ev.LBM_EOS_CS, 0.1, 4.0, 1.01 * Tc, ptr) == ev.LBM_EINVAL
    assert L.lbm_spinodal(ev.LBM_EOS_CS, 0.1, 4.0, 0.8 * Tc, None) == ev.LBM_EINVAL
    assert L.lbm_interface(ev.LBM_EOS_CS, 0.1, 4.0, 0.8 * Tc, 0.0, ptr) == ev.LBM_EINVAL
    assert L.lbm_interface(ev.LBM_EOS_CS, 0.1, 4.0, 1.2 * Tc, 1.0, ptr) == ev.LBM_EINVAL


def test_coexistence_rejects_supercritical_on_host():
    _, Tc = ev.lbm_critical_point(ev.LBM_EOS_CS, 0.1, 4.0)
    with pytest.raises(ev.LBMError) as e:
        ev.lbm_coexistence(ev.LBM_EOS_CS, 0.1, 4.0, 1.01 * Tc)
    assert e.value.code == ev.LBM_EINVAL


def test_surrogate_rejects_invalid_arguments_on_host():
    """Invalid sizes and layouts are rejected before any CUDA call (no GPU needed)."""
    from paper_2508_00577_gb300 import surrogate as S
    for H, W, base in ((15, 16, 32), (16, 24, 32), (8, 16, 32), (16, 16, 16)):
        with pytest.raises(S.SurError) as e:
            S.sur_init(H, W, base)
        assert e.value.code == S.SUR_EINVAL
    g = S.sur_gemm_args()
    g.a = S.sur_operand(16, S.SUR_OP_DENSE, 64, 0, 0, 128, 0, 0)
    g.b = S.sur_operand(16, S.SUR_OP_DENSE, 64, 0, 0, 48, 0, 0)
    g.M, g.N, g.K, g.splits, g.epi = 128, 48, 64, 1, S.SUR_EPI_F32      # N not a multiple of 32
    g.out, g.ldo = 16, 48
    cases = []
    c = S.sur_gemm_args(); c.a, c.b, c.M, c.N, c.K, c.splits, c.epi, c.out, c.ldo = g.a, g.b, 128, 48, 64, 1, 1, 16, 48
    cases.append(c)                                                         # N % 32 != 0
    c = S.sur_gemm_args(); c.a, c.b, c.M, c.N, c.K, c.splits, c.epi, c.out, c.ldo = g.a, g.b, 128, 32, 64, 2, 1, 16, 32
    cases.append(c)                                                         # split-K without the atomic epilogue
    c = S.sur_gemm_args(); c.a, c.b, c.M, c.N, c.K, c.splits, c.epi, c.out, c.ldo = g.a, g.b, 128, 32, 72, 1, 1, 16, 32
    cases.append(c)                                                         # dense K tail beyond ld
    bad_c = S.sur_operand(16, S.SUR_OP_CONV3, 64, 0, 24, 128, 16, 8)      # C not a power of two
    c = S.sur_gemm_args(); c.a, c.b, c.M, c.N, c.K, c.splits, c.epi, c.out, c.ldo = bad_c, g.b, 128, 32, 64, 1, 1, 16, 32
    cases.append(c)
    for c in cases:
        with pytest.raises(S.SurError) as e:
            S.sur_gemm(c, 16)
        assert e.value.code == S.SUR_EINVAL


def test_binding_constants_match_header():
    """Every LBM_* constant the header defines has the same value in the binding."""
    text = open(HEADER).read()
    defs = dict(re.findall(r"^#define\s+(LBM_\w+)\s+\(?(-?\d+)\)?", text, re.M))
    assert {"LBM_OK", "LBM_EINVAL", "LBM_TILE_BALANCED", "LBM_FP32", "LBM_EOS_CS"} <= set(defs)
    for name, value in defs.items():
        assert getattr(ev, name) == int(value), name


def test_surrogate_binding_constants_match_header():
    """Every SUR_* enumerator of the surrogate header has the same value in the binding."""
    from paper_2508_00577_gb300 import surrogate as S
    text = open(SUR_HEADER).read()
    vals = dict(re.findall(r"\b(SUR_[A-Z0-9_]+)\s*=\s*(\d+)", text))
    assert len(vals) >= 18
    for name, value in vals.items():
        assert getattr(S, name) == int(value), name


def test_batch_split_keeps_launch_items_below_2_31():
    """lbm_batch_step splits a call whose n_steps x items per step would overflow the
    persistent launch's 32-bit work counter: every launch but the last takes
    lbm_batch_launch_steps steps, an even count (the buffer parity, and so the captured
    graph, stays the same) whose items number fewer than 2^31."""
    L = ev.lib()
    for items in (1, 2, 3, 3001, 65536, 2**20 + 7, 2**30 - 1, 2**30 + 1, 2**31 - 1):
        n = L.lbm_batch_launch_steps(items)
        assert n >= 1
        assert n * items < 2**31, items
        assert n == 1 or n % 2 == 0
        assert n == 1 or (n + 2) * items >= 2**31 - 1      # the largest such even count
    assert L.lbm_batch_launch_steps(0) == -1
    # a call of INT_MAX steps on the ensemble's ~3000 items per step: a few thousand launches
    n = L.lbm_batch_launch_steps(3000)
    launches = -(-(2**31 - 1) // n)
    assert 2000 < launches < 4000
