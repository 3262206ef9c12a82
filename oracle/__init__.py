"""FP64 CPU oracle of the Enskog-Vlasov lattice Boltzmann step (arXiv 2508.00577).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it; the product package never imports it.
It shares no code with the CUDA path.

The step itself is plain C (``evlbm_oracle.c``, compiled with
``-ffp-contract=off``); ``eos`` holds the equation-of-state thermodynamics
(critical point, Maxwell construction, square-gradient interface) in NumPy.
This module compiles the C file on first use and wraps it with ctypes.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, textbook special cases or an independent
derivation; none is unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "evlbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libevlbm_oracle.so")
_FC_SRC = os.path.join(_HERE, "flopcount.cpp")
_FC_PATH = os.path.join(_BUILD, "flopcount")
_lock = threading.Lock()
_lib = None


class orc_params(ctypes.Structure):
    _fields_ = [
        ("Q", ctypes.c_int),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("nz", ctypes.c_int),
        ("eos", ctypes.c_int),
        ("a", ctypes.c_double),
        ("b", ctypes.c_double),
        ("R", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("lambda_", ctypes.c_double),
        ("thermal", ctypes.c_int),
        ("force_form", ctypes.c_int),
        ("walls", ctypes.c_int),
        ("wall_u", (ctypes.c_double * 3) * 2),
        ("wall_RT", ctypes.c_double),
    ]


def _fresh(out, *srcs):
    return os.path.exists(out) and all(os.path.getmtime(out) >= os.path.getmtime(s) for s in srcs)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build`` (gcc, FP contraction off, OpenMP), and
    its operation counter (``flopcount.cpp``, g++)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not _fresh(_FC_PATH, _FC_SRC, _SRC):
        tmp = _FC_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-o", tmp, _FC_SRC])
        os.replace(tmp, _FC_PATH)
    if not force and _fresh(_LIB_PATH, _SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def flops_per_update(Q=9, thermal=1, eos=1, force_form=0):
    """Floating-point operations (+, -, *, /) per lattice update of the oracle's step,
    counted by running the oracle's own source with a counting number type
    (``flopcount.cpp``).  The step's cost is a N + c (c: a few per-step constants);
    a is solved from two lattice sizes and checked on a third."""
    build()
    runs = []
    for nx, ny, nz in ((12, 10, 1), (16, 14, 1), (9, 7, 3)):
        if Q == 9:
            nz = 1
        out = subprocess.check_output([_FC_PATH, str(Q), str(thermal), str(eos), str(force_form),
                                       str(nx), str(ny), str(nz)], text=True).split()
        one, two, n = (int(v) for v in out)
        runs.append((n, two - one))
    (n1, s1), (n2, s2), (n3, s3) = runs
    a, rem = divmod(s2 - s1, n2 - n1)
    c = s1 - a * n1
    if rem or s3 != a * n3 + c:
        raise RuntimeError(f"operation count is not affine in the node count: {runs}")
    return a


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            pp = ctypes.POINTER(orc_params)
            L.orc_init.argtypes = [pp, dp, dp, dp, dp, dp]
            L.orc_step.argtypes = [pp, ctypes.c_int, dp, dp, dp]
            L.orc_macro.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp]
            L.orc_totals.argtypes = [pp, dp, dp, dp]
            L.orc_force.argtypes = [pp, dp, dp]
            L.orc_feq.argtypes = [ctypes.c_int, ctypes.c_double, dp, ctypes.c_double, dp]
            L.orc_geq.argtypes = [ctypes.c_int, ctypes.c_double, dp, ctypes.c_double, ctypes.c_double, dp]
            L.orc_eos.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp, dp]
            for name in ("orc_init", "orc_step", "orc_macro", "orc_totals", "orc_force"):
                getattr(L, name).restype = ctypes.c_int
            L.orc_num_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Params:
    """Model parameters (the paper's lattice, EOS constants a, b, R, kappa, tau, lambda)."""

    def __init__(self, Q=9, nx=64, ny=64, nz=1, eos=1, a=1.0, b=4.0, R=1.0, kappa=0.0,
                 tau=0.3, lambda_=1.0, thermal=1, force_form=0, walls=None):
        """walls: None (periodic), or (u_lo, u_hi, T_w): the columns x = 0 and x = nx-1 are
        wall nodes moving with the velocities u_lo, u_hi (3-vectors) at temperature T_w."""
        self.Q, self.nx, self.ny, self.nz = Q, nx, ny, nz
        self.eos, self.a, self.b, self.R, self.kappa = eos, a, b, R, kappa
        self.tau, self.lambda_, self.thermal, self.force_form = tau, lambda_, thermal, force_form
        self.walls = walls

    @property
    def D(self):
        return 2 if self.Q == 9 else 3

    @property
    def N(self):
        return self.nx * self.ny * self.nz

    def c(self):
        wu = ((ctypes.c_double * 3) * 2)()
        wRT = 0.0
        if self.walls is not None:
            lo, hi, Tw = self.walls
            for a in range(3):
                wu[0][a], wu[1][a] = float(lo[a]), float(hi[a])
            wRT = self.R * float(Tw)
        return orc_params(self.Q, self.nx, self.ny, self.nz, self.eos, self.a, self.b, self.R,
                          self.kappa, self.tau, self.lambda_, self.thermal, self.force_form,
                          1 if self.walls is not None else 0, wu, wRT)


class State:
    """Oracle state: post-collision populations f [Q][N] and g [Q][N] (FP64)."""

    def __init__(self, p: Params, rho, u, T):
        self.p = p
        N, Q, D = p.N, p.Q, p.D
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(N)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(D, N)
        T = np.ascontiguousarray(T, dtype=np.float64).reshape(N)
        self.T_iso = T.copy()
        self.f = np.zeros((Q, N))
        self.g = np.zeros((Q, N))
        pc = p.c()
        rc = lib().orc_init(ctypes.byref(pc), _ptr(rho), _ptr(u), _ptr(T), _ptr(self.f), _ptr(self.g))
        if rc != 0:
            raise ValueError(f"orc_init failed ({rc})")

    def step(self, n: int = 1):
        pc = self.p.c()
        rc = lib().orc_step(ctypes.byref(pc), int(n), _ptr(self.f), _ptr(self.g), _ptr(self.T_iso))
        if rc != 0:
            raise RuntimeError(f"orc_step failed ({rc})")
        return self

    def macro(self):
        """(rho [N], u [D][N], T [N], F [D][N]) as the next step would compute them."""
        p = self.p
        rho = np.zeros(p.N)
        u = np.zeros((p.D, p.N))
        T = np.zeros(p.N)
        F = np.zeros((p.D, p.N))
        pc = p.c()
        rc = lib().orc_macro(ctypes.byref(pc), _ptr(self.f), _ptr(self.g), _ptr(self.T_iso),
                             _ptr(rho), _ptr(u), _ptr(T), _ptr(F))
        if rc != 0:
            raise RuntimeError(f"orc_macro failed ({rc})")
        return rho, u, T, F

    def totals(self):
        """(sum rho, sum j_x, sum j_y, sum j_z, sum g) of the raw populations."""
        out = np.zeros(5)
        pc = self.p.c()
        lib().orc_totals(ctypes.byref(pc), _ptr(self.f), _ptr(self.g), _ptr(out))
        return out


def feq(Q, rho, u, theta0):
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).ravel())
    u3 = np.zeros(3)
    u3[: u.size] = u
    out = np.zeros(Q)
    lib().orc_feq(Q, rho, _ptr(u3), theta0, _ptr(out))
    return out


def geq(Q, rho, u, theta0, RT):
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).ravel())
    u3 = np.zeros(3)
    u3[: u.size] = u
    out = np.zeros(Q)
    lib().orc_geq(Q, rho, _ptr(u3), theta0, RT, _ptr(out))
    return out


def eos_state(eos_kind, b, rho, RT, thermal=1):
    """(P0, theta0 = P0/rho, gamma0) in the Enskog gauge P0 = P_E."""
    P0 = ctypes.c_double()
    th = ctypes.c_double()
    g0 = ctypes.c_double()
    lib().orc_eos(eos_kind, thermal, b, rho, RT, ctypes.byref(P0), ctypes.byref(th), ctypes.byref(g0))
    return P0.value, th.value, g0.value


def force(p: Params, rho):
    """Non-local force F [D][N] of the Enskog gauge for the density field rho [N]."""
    rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(p.N)
    F = np.zeros((p.D, p.N))
    pc = p.c()
    rc = lib().orc_force(ctypes.byref(pc), _ptr(rho), _ptr(F))
    if rc != 0:
        raise RuntimeError(f"orc_force failed ({rc})")
    return F


def num_threads():
    return lib().orc_num_threads()


def lattice(Q):
    """(c [Q][3], w [Q]) in the oracle's ordering i = (cx+1) + 3(cy+1) + 9(cz+1)."""
    c = np.zeros((Q, 3), dtype=np.int64)
    w = np.zeros(Q)
    D = 2 if Q == 9 else 3
    for i in range(Q):
        c[i] = (i % 3 - 1, (i // 3) % 3 - 1, (i // 9 - 1) if Q == 27 else 0)
        w[i] = np.prod([(2 / 3 if c[i, a] == 0 else 1 / 6) for a in range(D)])
    return c, w
