"""GB300 Enskog-Vlasov lattice Boltzmann library (Karlin & Hosseini, arXiv 2508.00577).

Thin Python binding of the C ABI declared in ``include/evlbm.h``: the functions
below carry the C names and only marshal arguments; every step of the model
runs in the CUDA kernels of ``libevlbm.so`` (built in-tree from ``csrc/``).
There is no CPU fallback: if the shared library cannot be built or loaded,
``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = [
    "lbm_params", "lib", "lbm_init", "lbm_step", "lbm_moments", "lbm_moments_device",
    "lbm_populations", "lbm_conserved", "lbm_step_count", "lbm_launches_per_step", "lbm_set_tile",
    "lbm_get_tile", "lbm_autotune", "lbm_sync", "lbm_free",
    "lbm_last_error", "lbm_coexistence", "lbm_critical_point", "lbm_spinodal", "lbm_interface",
    "lbm_kappa_for_width", "lbm_step_noalloc", "lbm_reset_device",
    "lbm_save", "lbm_load", "lbm_bounds_violations", "lbm_set_walls", "LBMError", "Lattice",
    "LBM_D2Q9", "LBM_D3Q27", "LBM_TILE_BALANCED", "LBM_EOS_VDW", "LBM_EOS_CS", "LBM_FP64", "LBM_FP32",
    "LBM_FP16_DEV", "LBM_BF16_DEV", "EXPORTED_SYMBOLS", "Batch",
]

LBM_OK, LBM_EINVAL, LBM_ECUDA, LBM_ENOMEM, LBM_ENONFINITE, LBM_ETIMEOUT, LBM_EIO = 0, -1, -2, -3, -4, -5, -6
LBM_D2Q9, LBM_D3Q27 = 0, 1
LBM_TILE_BALANCED = -1
LBM_EOS_VDW, LBM_EOS_CS = 0, 1
LBM_FP64, LBM_FP32, LBM_FP16_DEV, LBM_BF16_DEV = 0, 1, 2, 3

_ERRNAMES = {LBM_EINVAL: "LBM_EINVAL", LBM_ECUDA: "LBM_ECUDA", LBM_ENOMEM: "LBM_ENOMEM",
             LBM_ENONFINITE: "LBM_ENONFINITE", LBM_ETIMEOUT: "LBM_ETIMEOUT", LBM_EIO: "LBM_EIO"}

# Every symbol include/evlbm.h declares.
EXPORTED_SYMBOLS = (
    "lbm_init", "lbm_step", "lbm_moments", "lbm_moments_device", "lbm_populations",
    "lbm_conserved", "lbm_step_count", "lbm_launches_per_step", "lbm_set_tile", "lbm_get_tile",
    "lbm_autotune", "lbm_sync", "lbm_free", "lbm_last_error", "lbm_coexistence", "lbm_critical_point",
    "lbm_spinodal", "lbm_interface", "lbm_step_noalloc", "lbm_batch_init", "lbm_batch_step", "lbm_batch_moments", "lbm_batch_set_tile",
    "lbm_batch_get_tile", "lbm_batch_autotune", "lbm_batch_set_wait_limit", "lbm_batch_nodes",
    "lbm_batch_free", "lbm_batch_last_error", "lbm_reset_device", "lbm_save", "lbm_load",
    "lbm_bounds_violations", "lbm_set_walls", "lbm_batch_launch_steps",
)


class LBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("eos", ctypes.c_int), ("a", ctypes.c_double), ("b", ctypes.c_double), ("R", ctypes.c_double),
        ("kappa", ctypes.c_double), ("tau", ctypes.c_double), ("lambda_", ctypes.c_double),
        ("thermal", ctypes.c_int), ("precision", ctypes.c_int), ("force_form", ctypes.c_int),
    ]

    @classmethod
    def make(cls, lattice=LBM_D2Q9, nx=64, ny=64, nz=1, eos=LBM_EOS_CS, a=0.1, b=4.0, R=1.0,
             kappa=0.0, tau=0.3, lambda_=1.0, thermal=1, precision=LBM_FP32, force_form=0):
        return cls(lattice, nx, ny, nz, eos, a, b, R, kappa, tau, lambda_, thermal, precision, force_form)

    @property
    def Q(self):
        return 9 if self.lattice == LBM_D2Q9 else 27

    @property
    def D(self):
        return 2 if self.lattice == LBM_D2Q9 else 3

    @property
    def N(self):
        return self.nx * self.ny * self.nz


_lock = threading.Lock()
_lib = None


def lib():
    """Load (building first if needed) the in-tree CUDA library."""
    global _lib
    with _lock:
        if _lib is None:
            from . import _build
            path = os.environ.get("EVLBM_LIBRARY", "")
            if not path:                      # the in-tree library, rebuilt when stale
                path = _build.LIB
                if not os.path.exists(path) or _build_needed(_build):
                    _build.build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            pp = ctypes.POINTER(lbm_params)
            vp = ctypes.c_void_p
            L.lbm_init.argtypes = [pp, dp, dp, dp, vp, ctypes.POINTER(vp)]
            L.lbm_step.argtypes = [vp, ctypes.c_int]
            L.lbm_moments.argtypes = [vp, dp, dp, dp, dp]
            L.lbm_moments_device.argtypes = [vp, vp, vp, vp]
            L.lbm_reset_device.argtypes = [vp, vp, vp, vp]
            L.lbm_populations.argtypes = [vp, dp, dp]
            L.lbm_conserved.argtypes = [vp, dp]
            L.lbm_step_count.argtypes = [vp]
            L.lbm_bounds_violations.argtypes = []
            L.lbm_bounds_violations.restype = ctypes.c_longlong
            L.lbm_save.argtypes = [vp, ctypes.c_char_p]
            L.lbm_load.argtypes = [vp, ctypes.c_char_p]
            L.lbm_step_count.restype = ctypes.c_longlong
            L.lbm_launches_per_step.argtypes = [vp]
            L.lbm_set_walls.argtypes = [vp, ctypes.c_int, dp, dp, ctypes.c_double]
            ip = ctypes.POINTER(ctypes.c_int)
            L.lbm_set_tile.argtypes = [vp, ctypes.c_int, ctypes.c_int]
            L.lbm_get_tile.argtypes = [vp, ip, ip]
            L.lbm_autotune.argtypes = [vp, ctypes.c_int, ip, ip]
            L.lbm_sync.argtypes = [vp]
            L.lbm_free.argtypes = [vp]
            L.lbm_last_error.argtypes = [vp]
            L.lbm_last_error.restype = ctypes.c_char_p
            L.lbm_coexistence.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
            L.lbm_critical_point.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
            L.lbm_spinodal.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
            L.lbm_interface.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, dp]
            L.lbm_step_noalloc.argtypes = [pp, vp, vp, vp, vp, vp, vp]
            L.lbm_batch_init.argtypes = [pp, ctypes.c_int, ip, ip, dp, dp, dp, vp, ctypes.POINTER(vp)]
            L.lbm_batch_step.argtypes = [vp, ctypes.c_int]
            L.lbm_batch_launch_steps.argtypes = [ctypes.c_int]
            L.lbm_batch_moments.argtypes = [vp, ctypes.c_int, dp, dp, dp]
            L.lbm_batch_set_tile.argtypes = [vp, ctypes.c_int, ctypes.c_int]
            L.lbm_batch_get_tile.argtypes = [vp, ip, ip]
            L.lbm_batch_autotune.argtypes = [vp, ctypes.c_int, ip, ip]
            L.lbm_batch_set_wait_limit.argtypes = [vp, ctypes.c_longlong, ctypes.c_int]
            L.lbm_batch_nodes.argtypes = [vp]
            L.lbm_batch_nodes.restype = ctypes.c_longlong
            L.lbm_batch_free.argtypes = [vp]
            L.lbm_batch_last_error.argtypes = [vp]
            L.lbm_batch_last_error.restype = ctypes.c_char_p
            _lib = L
    return _lib


def _build_needed(b) -> bool:
    try:
        t = os.path.getmtime(b.LIB)
    except OSError:
        return True
    for d in (b.CSRC, os.path.join(b.HERE, "..", "include")):
        for f in os.listdir(d):
            if os.path.getmtime(os.path.join(d, f)) > t:
                return True
    return False


def _dptr(a):
    if a is None:
        return None
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]):
        raise TypeError("expected a C-contiguous float64 numpy array")
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc, ctx=None):
    if rc != LBM_OK:
        msg = lib().lbm_last_error(ctx)
        raise LBMError(rc, msg.decode() if msg else "")


# ---------------------------------------------------------------------------
# C ABI, same names
# ---------------------------------------------------------------------------

def lbm_init(params: lbm_params, rho, u, T, stream=0):
    """Context from host FP64 fields rho[N], u[D][N], T[N]; returns the opaque handle."""
    rho = np.ascontiguousarray(rho, dtype=np.float64).ravel()
    u = np.ascontiguousarray(u, dtype=np.float64).ravel()
    T = np.ascontiguousarray(T, dtype=np.float64).ravel()
    if params.lattice in (LBM_D2Q9, LBM_D3Q27) and min(params.nx, params.ny, params.nz) >= 1:
        N, D = params.N, params.D
        if rho.size != N or T.size != N or u.size != D * N:
            raise ValueError(f"fields must hold rho[{N}], u[{D}][{N}], T[{N}]")
    out = ctypes.c_void_p()
    rc = lib().lbm_init(ctypes.byref(params), _dptr(rho), _dptr(u), _dptr(T), ctypes.c_void_p(stream),
                        ctypes.byref(out))
    _check(rc, None)
    return out.value


def lbm_step(ctx, n_steps=1):
    _check(lib().lbm_step(ctx, int(n_steps)), ctx)


def lbm_moments(ctx, rho=None, u=None, T=None, F=None):
    _check(lib().lbm_moments(ctx, _dptr(rho), _dptr(u), _dptr(T), _dptr(F)), ctx)


def lbm_moments_device(ctx, d_rho=0, d_u=0, d_T=0):
    """Device pointers (ints, e.g. tensor.data_ptr()) of FP32 outputs; 0 = skip."""
    _check(lib().lbm_moments_device(ctx, ctypes.c_void_p(d_rho or None), ctypes.c_void_p(d_u or None),
                                    ctypes.c_void_p(d_T or None)), ctx)


def lbm_reset_device(ctx, d_rho, d_u, d_T):
    """Populations := local equilibria of device FP32 fields (int device pointers)."""
    _check(lib().lbm_reset_device(ctx, d_rho, d_u, d_T), ctx)


def lbm_populations(ctx, f, g=None):
    _check(lib().lbm_populations(ctx, _dptr(f), _dptr(g)), ctx)


def lbm_conserved(ctx):
    out = np.zeros(5)
    _check(lib().lbm_conserved(ctx, _dptr(out)), ctx)
    return out


def lbm_step_count(ctx):
    return lib().lbm_step_count(ctx)


def lbm_bounds_violations():
    """Out-of-range indices met by the fused kernels of a bounds-checked library (-1: no checks)."""
    return lib().lbm_bounds_violations()


def lbm_save(ctx, path):
    """Write the context's state (populations, step count, parameters) to `path`."""
    _check(lib().lbm_save(ctx, os.fsencode(path)), ctx)


def lbm_load(ctx, path):
    """Restore a state written by lbm_save into a context with the same parameters."""
    _check(lib().lbm_load(ctx, os.fsencode(path)), ctx)


def lbm_launches_per_step(ctx):
    return lib().lbm_launches_per_step(ctx)


def lbm_set_walls(ctx, enable, u_lo=None, u_hi=None, T_w=0.0):
    """Wall nodes at the columns x = 0 and x = nx-1 (velocities u_lo, u_hi, temperature T_w),
    or periodic x again with enable = 0."""
    if not enable:
        _check(lib().lbm_set_walls(ctx, 0, None, None, 0.0), ctx)
        return
    lo = np.zeros(3)
    hi = np.zeros(3)
    lo[:len(u_lo)] = u_lo
    hi[:len(u_hi)] = u_hi
    _check(lib().lbm_set_walls(ctx, 1, _dptr(lo), _dptr(hi), float(T_w)), ctx)


def lbm_set_tile(ctx, tile_w, tile_h):
    _check(lib().lbm_set_tile(ctx, int(tile_w), int(tile_h)), ctx)


def lbm_get_tile(ctx):
    w, h = ctypes.c_int(), ctypes.c_int()
    _check(lib().lbm_get_tile(ctx, ctypes.byref(w), ctypes.byref(h)), ctx)
    return w.value, h.value


def lbm_autotune(ctx, probe_steps=3):
    w, h = ctypes.c_int(), ctypes.c_int()
    _check(lib().lbm_autotune(ctx, int(probe_steps), ctypes.byref(w), ctypes.byref(h)), ctx)
    return w.value, h.value


def lbm_sync(ctx):
    _check(lib().lbm_sync(ctx), ctx)


def lbm_free(ctx):
    _check(lib().lbm_free(ctx), None)


def lbm_last_error(ctx=None):
    m = lib().lbm_last_error(ctx)
    return m.decode() if m else ""


def lbm_coexistence(eos, a, b, RT):
    out = np.zeros(2)
    rc = lib().lbm_coexistence(int(eos), float(a), float(b), float(RT), _dptr(out))
    if rc != LBM_OK:
        raise LBMError(rc, "lbm_coexistence")
    return float(out[0]), float(out[1])


def lbm_critical_point(eos, a, b):
    out = np.zeros(2)
    rc = lib().lbm_critical_point(int(eos), float(a), float(b), _dptr(out))
    if rc != LBM_OK:
        raise LBMError(rc, "lbm_critical_point")
    return float(out[0]), float(out[1])


def lbm_spinodal(eos, a, b, RT):
    out = np.zeros(2)
    rc = lib().lbm_spinodal(int(eos), float(a), float(b), float(RT), _dptr(out))
    if rc != LBM_OK:
        raise LBMError(rc, "lbm_spinodal")
    return float(out[0]), float(out[1])


def lbm_interface(eos, a, b, RT, kappa):
    """(10-90 % width, surface tension) of the planar interface at RT with capillarity kappa."""
    out = np.zeros(2)
    rc = lib().lbm_interface(int(eos), float(a), float(b), float(RT), float(kappa), _dptr(out))
    if rc != LBM_OK:
        raise LBMError(rc, "lbm_interface")
    return float(out[0]), float(out[1])


def lbm_kappa_for_width(eos, a, b, RT, width):
    """kappa whose planar interface has the 10-90 % width `width` (width ~ sqrt(kappa))."""
    w1, _ = lbm_interface(eos, a, b, RT, 1.0)
    return (float(width) / w1) ** 2


def lbm_step_noalloc(params: lbm_params, d_f, d_g, d_RT, d_f_out, d_g_out, stream=0):
    """One FP64 step on caller-owned device buffers (pointers as ints, 0 = NULL);
    allocates nothing (see include/evlbm.h)."""
    vp = ctypes.c_void_p
    rc = lib().lbm_step_noalloc(ctypes.byref(params), vp(d_f or None), vp(d_g or None), vp(d_RT or None),
                                vp(d_f_out or None), vp(d_g_out or None), vp(stream or None))
    if rc != LBM_OK:
        raise LBMError(rc, "lbm_step_noalloc")


def _bcheck(rc, b):
    if rc != LBM_OK:
        msg = lib().lbm_batch_last_error(b) if b else b""
        raise LBMError(rc, msg.decode() if msg else "")


class Batch:
    """Batched ensemble of independent 2-D domains (lbm_batch_* of the C ABI)."""

    def __init__(self, params: lbm_params, sizes, rho, u, T, stream=0):
        """sizes: [(nx, ny), ...]; rho, T: per-domain flat arrays; u: per-domain [2][N_d] arrays."""
        self.sizes = [(int(a), int(b)) for a, b in sizes]
        n = len(self.sizes)
        nx = (ctypes.c_int * n)(*[s[0] for s in self.sizes])
        ny = (ctypes.c_int * n)(*[s[1] for s in self.sizes])
        rho_c = np.ascontiguousarray(np.concatenate([np.ravel(r) for r in rho]), dtype=np.float64)
        u_c = np.ascontiguousarray(np.concatenate([np.ravel(v) for v in u]), dtype=np.float64)
        T_c = np.ascontiguousarray(np.concatenate([np.ravel(t) for t in T]), dtype=np.float64)
        total = sum(a * b for a, b in self.sizes)
        if rho_c.size != total or T_c.size != total or u_c.size != 2 * total:
            raise ValueError("field sizes do not match the domain sizes")
        out = ctypes.c_void_p()
        rc = lib().lbm_batch_init(ctypes.byref(params), n, nx, ny, _dptr(rho_c), _dptr(u_c), _dptr(T_c),
                                  ctypes.c_void_p(stream), ctypes.byref(out))
        _bcheck(rc, None)
        self.params = params
        self.b = out.value

    def step(self, n=1):
        _bcheck(lib().lbm_batch_step(self.b, int(n)), self.b)
        return self

    def moments(self, d):
        nx, ny = self.sizes[d]
        N = nx * ny
        rho, u, T = np.zeros(N), np.zeros(2 * N), np.zeros(N)
        _bcheck(lib().lbm_batch_moments(self.b, int(d), _dptr(rho), _dptr(u), _dptr(T)), self.b)
        return rho, u.reshape(2, N), T

    def set_tile(self, w, h):
        _bcheck(lib().lbm_batch_set_tile(self.b, int(w), int(h)), self.b)

    def get_tile(self):
        w, h = ctypes.c_int(), ctypes.c_int()
        _bcheck(lib().lbm_batch_get_tile(self.b, ctypes.byref(w), ctypes.byref(h)), self.b)
        return w.value, h.value

    def autotune(self, probe_steps=2):
        w, h = ctypes.c_int(), ctypes.c_int()
        _bcheck(lib().lbm_batch_autotune(self.b, int(probe_steps), ctypes.byref(w), ctypes.byref(h)), self.b)
        return w.value, h.value

    def set_wait_limit(self, polls, probe_unset_flag=0):
        _bcheck(lib().lbm_batch_set_wait_limit(self.b, int(polls), int(probe_unset_flag)), self.b)

    def nodes(self):
        return lib().lbm_batch_nodes(self.b)

    def close(self):
        if self.b:
            lib().lbm_batch_free(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Lattice:
    """Convenience owner of one context (frees it on close)."""

    def __init__(self, params: lbm_params, rho, u, T, stream=0):
        self.params = params
        self.ctx = lbm_init(params, rho, u, T, stream)

    def step(self, n=1):
        lbm_step(self.ctx, n)
        return self

    def moments(self):
        p = self.params
        rho, u, T, F = np.zeros(p.N), np.zeros(p.D * p.N), np.zeros(p.N), np.zeros(p.D * p.N)
        lbm_moments(self.ctx, rho, u, T, F)
        return rho, u.reshape(p.D, p.N), T, F.reshape(p.D, p.N)

    def populations(self):
        p = self.params
        f = np.zeros(p.Q * p.N)
        g = np.zeros(p.Q * p.N) if p.thermal else None
        lbm_populations(self.ctx, f, g)
        return f.reshape(p.Q, p.N), (g.reshape(p.Q, p.N) if g is not None else None)

    def save(self, path):
        lbm_save(self.ctx, path)

    def load(self, path):
        lbm_load(self.ctx, path)

    def conserved(self):
        return lbm_conserved(self.ctx)

    def close(self):
        if self.ctx:
            lbm_free(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
