"""Binding of the learned-surrogate C ABI declared in ``include/evsur.h``.

Same names as the C functions; arguments are marshalled only.  Device arrays
are passed as integer device pointers (e.g. ``tensor.data_ptr()``); the U-Net
forward and backward passes, Adam and the rollout run in the CUDA kernels of
``libevlbm.so``.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import lib as _lib_loader

SUR_OK, SUR_EINVAL, SUR_ECUDA, SUR_ENOMEM, SUR_ETIMEOUT, SUR_EUNPHYSICAL = 0, 1, 2, 3, 4, 5
SUR_OP_DENSE, SUR_OP_PIX, SUR_OP_CONV3, SUR_OP_UPADJ, SUR_OP_TPIX, SUR_OP_TCONV3, SUR_OP_TUP = range(7)
SUR_EPI_BF16, SUR_EPI_F32, SUR_EPI_F32_ATOMIC, SUR_EPI_CONV, SUR_EPI_SHUF = range(5)

_ERRNAMES = {SUR_EINVAL: "SUR_EINVAL", SUR_ECUDA: "SUR_ECUDA", SUR_ENOMEM: "SUR_ENOMEM",
             SUR_ETIMEOUT: "SUR_ETIMEOUT", SUR_EUNPHYSICAL: "SUR_EUNPHYSICAL"}

# Every symbol include/evsur.h declares.
EXPORTED_SYMBOLS = (
    "sur_gemm", "sur_set_tma", "sur_init", "sur_free", "sur_num_params", "sur_get_params", "sur_set_params", "sur_get_grads",
    "sur_set_norm", "sur_forward_backward", "sur_train_step", "sur_forward_backward_unrolled",
    "sur_train_step_unrolled", "sur_infer", "sur_indicators", "sur_rollout", "sur_last_error",
)

# Architecture tables (same as the C runtime): 3x3 convolutions (Cin, Cout) in
# execution order, transposed convolutions (Cin, Cout), head width.
CONV_IO = ((8, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128), (128, 256), (256, 256),
           (256, 128), (128, 128), (128, 64), (64, 64), (64, 32), (32, 32))
UP_IO = ((256, 128), (128, 64), (64, 32))
BASE = 32


class SurError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class sur_operand(ctypes.Structure):
    _fields_ = [("p", ctypes.c_void_p), ("kind", ctypes.c_int), ("ld", ctypes.c_int), ("c0", ctypes.c_int),
                ("C", ctypes.c_int), ("rows", ctypes.c_int), ("H", ctypes.c_int), ("W", ctypes.c_int)]


class sur_gemm_args(ctypes.Structure):
    _fields_ = [("a", sur_operand), ("b", sur_operand), ("M", ctypes.c_int), ("N", ctypes.c_int),
                ("K", ctypes.c_int), ("splits", ctypes.c_int), ("epi", ctypes.c_int),
                ("bias", ctypes.c_void_p), ("out", ctypes.c_void_p), ("ldo", ctypes.c_int), ("co0", ctypes.c_int),
                ("y", ctypes.c_void_p), ("ldy", ctypes.c_int), ("cy0", ctypes.c_int), ("shuf_cout", ctypes.c_int)]


class sur_rollout_cfg(ctypes.Structure):
    _fields_ = [("windows", ctypes.c_int), ("steps", ctypes.c_int), ("rho_mid", ctypes.c_float),
                ("max_mass_drift", ctypes.c_float), ("max_area_change", ctypes.c_float),
                ("project_mass", ctypes.c_int), ("max_interface_shift", ctypes.c_float)]


_lock = threading.Lock()
_ready = False


def lib():
    global _ready
    L = _lib_loader()
    with _lock:
        if not _ready:
            vp, ip, fp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_float)
            L.sur_gemm.argtypes = [ctypes.POINTER(sur_gemm_args), vp, vp]
            L.sur_set_tma.argtypes = [ip]
            L.sur_init.argtypes = [ip, ip, ip, ctypes.c_uint64, vp, ctypes.POINTER(vp)]
            L.sur_free.argtypes = [vp]
            L.sur_num_params.argtypes = [vp]
            L.sur_num_params.restype = ctypes.c_longlong
            L.sur_get_params.argtypes = [vp, fp, ctypes.c_longlong]
            L.sur_set_params.argtypes = [vp, fp, ctypes.c_longlong]
            L.sur_get_grads.argtypes = [vp, fp, ctypes.c_longlong]
            L.sur_set_norm.argtypes = [vp, fp, fp, fp]
            L.sur_forward_backward.argtypes = [vp, vp, vp, ip, fp]
            L.sur_train_step.argtypes = [vp, vp, vp, ip, ctypes.c_float, fp]
            L.sur_forward_backward_unrolled.argtypes = [vp, vp, vp, ip, ip, fp]
            L.sur_train_step_unrolled.argtypes = [vp, vp, vp, ip, ip, ctypes.c_float, fp]
            L.sur_infer.argtypes = [vp, vp, vp, ip]
            L.sur_indicators.argtypes = [vp, ip, ip, ip, ctypes.c_float, vp, vp]
            L.sur_rollout.argtypes = [vp, vp, vp, ip, ctypes.POINTER(sur_rollout_cfg),
                                      ctypes.POINTER(ctypes.c_ubyte), ctypes.POINTER(ctypes.c_int)]
            L.sur_last_error.argtypes = [vp]
            L.sur_last_error.restype = ctypes.c_char_p
            _ready = True
    return L


def _check(rc, model=None):
    if rc != SUR_OK:
        msg = lib().sur_last_error(model) if model else b""
        raise SurError(rc, msg.decode() if msg else "")


def _f32(a):
    if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]):
        raise TypeError("expected a C-contiguous float32 numpy array")
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


# ---------------------------------------------------------------------------
# C ABI, same names
# ---------------------------------------------------------------------------

def sur_gemm(args: sur_gemm_args, d_status, stream=0):
    _check(lib().sur_gemm(ctypes.byref(args), d_status, stream))


def sur_set_tma(enable):
    _check(lib().sur_set_tma(1 if enable else 0))


def sur_init(H, W, base_ch=BASE, seed=0, stream=0):
    out = ctypes.c_void_p()
    _check(lib().sur_init(H, W, base_ch, seed, stream, ctypes.byref(out)))
    return out.value


def sur_free(model):
    _check(lib().sur_free(model))


def sur_num_params(model):
    return int(lib().sur_num_params(model))


def sur_get_params(model, out):
    _check(lib().sur_get_params(model, _f32(out), out.size), model)


def sur_set_params(model, params):
    _check(lib().sur_set_params(model, _f32(params), params.size), model)


def sur_get_grads(model, out):
    _check(lib().sur_get_grads(model, _f32(out), out.size), model)


def sur_set_norm(model, in_mean, in_scale, out_scale):
    a = [np.ascontiguousarray(v, dtype=np.float32) for v in (in_mean, in_scale, out_scale)]
    _check(lib().sur_set_norm(model, *(_f32(v) for v in a)), model)


def sur_forward_backward(model, d_x, d_y, batch, want_loss=True):
    loss = ctypes.c_float(0.0)
    _check(lib().sur_forward_backward(model, d_x, d_y, batch, ctypes.byref(loss) if want_loss else None), model)
    return loss.value if want_loss else None


def sur_train_step(model, d_x, d_y, batch, lr, want_loss=True):
    loss = ctypes.c_float(0.0)
    _check(lib().sur_train_step(model, d_x, d_y, batch, lr, ctypes.byref(loss) if want_loss else None), model)
    return loss.value if want_loss else None


def sur_forward_backward_unrolled(model, d_x0, d_targets, windows, batch, want_loss=True):
    loss = ctypes.c_float(0.0)
    _check(lib().sur_forward_backward_unrolled(model, d_x0, d_targets, windows, batch,
                                               ctypes.byref(loss) if want_loss else None), model)
    return loss.value if want_loss else None


def sur_train_step_unrolled(model, d_x0, d_targets, windows, batch, lr, want_loss=True):
    loss = ctypes.c_float(0.0)
    _check(lib().sur_train_step_unrolled(model, d_x0, d_targets, windows, batch, lr,
                                         ctypes.byref(loss) if want_loss else None), model)
    return loss.value if want_loss else None


def sur_infer(model, d_x, d_y, batch):
    _check(lib().sur_infer(model, d_x, d_y, batch), model)


def sur_indicators(d_fields, batch, H, W, rho_mid, d_out, stream=0):
    _check(lib().sur_indicators(d_fields, batch, H, W, rho_mid, d_out, stream))


def sur_rollout(model, lb_ctx, d_fields, batch, windows, steps, rho_mid, max_mass_drift, max_area_change,
                project_mass=False, max_interface_shift=1.0):
    cfg = sur_rollout_cfg(windows, steps, rho_mid, max_mass_drift, max_area_change, 1 if project_mass else 0,
                          max_interface_shift)
    used = (ctypes.c_ubyte * max(windows, 1))()
    nfb = ctypes.c_int(0)
    _check(lib().sur_rollout(model, lb_ctx, d_fields, batch, ctypes.byref(cfg), used, ctypes.byref(nfb)), model)
    return nfb.value, np.frombuffer(bytes(used), dtype=np.uint8)[:windows].copy()


def sur_last_error(model):
    msg = lib().sur_last_error(model)
    return msg.decode() if msg else ""


def param_layout():
    """(name, offset, shape) of every parameter tensor in canonical order."""
    out, off = [], 0
    for i, (ci, co) in enumerate(CONV_IO):
        kp = -(-9 * ci // 64) * 64
        out.append((f"conv{i}.w", off, (kp, co)))
        off += kp * co
        out.append((f"conv{i}.b", off, (co,)))
        off += co
    for j, (ci, co) in enumerate(UP_IO):
        out.append((f"up{j}.w", off, (4 * co, ci)))
        off += 4 * co * ci
        out.append((f"up{j}.b", off, (co,)))
        off += co
    out.append(("head.w", off, (4, BASE)))
    off += 4 * BASE
    out.append(("head.b", off, (4,)))
    off += 4
    return out, off


class Surrogate:
    """Owner of one sur_model (frees it on close)."""

    def __init__(self, H, W, seed=0, stream=0):
        self.H, self.W = H, W
        self.m = sur_init(H, W, BASE, seed, stream)
        self.n = sur_num_params(self.m)

    def params(self):
        p = np.zeros(self.n, np.float32)
        sur_get_params(self.m, p)
        return p

    def set_params(self, p):
        sur_set_params(self.m, np.ascontiguousarray(p, dtype=np.float32))

    def grads(self):
        g = np.zeros(self.n, np.float32)
        sur_get_grads(self.m, g)
        return g

    def set_norm(self, in_mean, in_scale, out_scale):
        sur_set_norm(self.m, in_mean, in_scale, out_scale)

    def forward_backward(self, d_x, d_y, batch):
        return sur_forward_backward(self.m, d_x, d_y, batch)

    def train_step(self, d_x, d_y, batch, lr, want_loss=True):
        return sur_train_step(self.m, d_x, d_y, batch, lr, want_loss)

    def forward_backward_unrolled(self, d_x0, d_targets, windows, batch):
        return sur_forward_backward_unrolled(self.m, d_x0, d_targets, windows, batch)

    def train_step_unrolled(self, d_x0, d_targets, windows, batch, lr, want_loss=True):
        return sur_train_step_unrolled(self.m, d_x0, d_targets, windows, batch, lr, want_loss)

    def infer(self, d_x, d_y, batch):
        sur_infer(self.m, d_x, d_y, batch)

    def rollout(self, lb_ctx, d_fields, batch, windows, steps, rho_mid, max_mass_drift=1e-3, max_area_change=0.02,
                project_mass=False, max_interface_shift=1.0):
        return sur_rollout(self.m, lb_ctx, d_fields, batch, windows, steps, rho_mid, max_mass_drift, max_area_change,
                           project_mass, max_interface_shift)

    def close(self):
        if self.m:
            sur_free(self.m)
            self.m = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
