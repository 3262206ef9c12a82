"""Seeded synthetic inputs of the workloads (initial density, velocity and temperature fields).

This module holds no arithmetic of the lattice Boltzmann method: only the
shapes of the initial conditions (tanh interfaces of slabs and droplets,
i.i.d. density noise, uneven ensemble sizes) and their random draws.  Both the
CUDA path and the CPU oracle are fed from here; the coexisting densities a
profile connects are arguments, supplied by the caller.

Fields are flat SoA arrays with x fastest: rho[N], u[D][N], T[N].
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 20250801
_MASK64 = (1 << 64) - 1


def splitmix64(x):
    """SplitMix64 finaliser applied element-wise to uint64 values (public-domain mixer)."""
    z = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & np.uint64(_MASK64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, n: int):
    """n uniforms in [0, 1) with 53 random bits: splitmix64(seed xor node index)."""
    idx = np.arange(n, dtype=np.uint64) ^ np.uint64(seed & _MASK64)
    return (splitmix64(idx) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def tanh_profile(d, rho_v: float, rho_l: float, width: float = 4.0):
    """rho_v + (rho_l - rho_v)/2 (1 + tanh(2 d / width)); d > 0 inside the dense phase."""
    return rho_v + 0.5 * (rho_l - rho_v) * (1.0 + np.tanh(2.0 * np.asarray(d) / width))


def slab(nx: int, ny: int, rho_v: float, rho_l: float, T: float, thickness: float = 32.0,
         width: float = 4.0, nz: int = 1, D: int = 2):
    """Planar liquid slab normal to x, centred, tanh interfaces; u = 0, uniform T."""
    x = np.arange(nx, dtype=np.float64)
    d = 0.5 * thickness - np.abs(x - 0.5 * (nx - 1))
    prof = tanh_profile(d, rho_v, rho_l, width)
    rho = np.broadcast_to(prof, (nz, ny, nx)).reshape(-1).copy()
    N = rho.size
    return rho, np.zeros((D, N)), np.full(N, float(T))


def droplet(nx: int, ny: int, R: float, rho_v: float, rho_l: float, T: float, width: float = 4.0,
            centre=None):
    """Centred circular droplet of radius R (2-D), tanh interface; u = 0, uniform T."""
    cx, cy = centre if centre is not None else (0.5 * (nx - 1), 0.5 * (ny - 1))
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    d = R - np.hypot(x - cx, y - cy)
    rho = tanh_profile(d, rho_v, rho_l, width).reshape(-1)
    N = rho.size
    return rho, np.zeros((2, N)), np.full(N, float(T))


def droplet_stack(nx: int, ny: int, cases, width: float = 4.0):
    """Independent 2-D layers stacked along z, one droplet per layer.
    cases: sequence of (R, rho_v, rho_l, T)."""
    rhos, us, Ts = [], [], []
    for R, rv, rl, T in cases:
        r, u, t = droplet(nx, ny, R, rv, rl, T, width)
        rhos.append(r); us.append(u); Ts.append(t)
    return np.concatenate(rhos), np.concatenate(us, axis=1), np.concatenate(Ts)


def spinodal_noise(nx: int, ny: int, nz: int, rho_mean: float, T: float, amplitude: float = 0.01,
                   seed: int = DEFAULT_SEED, D: int = 3):
    """Uniform density rho_mean (1 + 2 amplitude (U - 1/2)), U ~ U[0,1) per node; u = 0."""
    N = nx * ny * nz
    U = uniform01(seed, N)
    rho = rho_mean * (1.0 + 2.0 * amplitude * (U - 0.5))
    return rho, np.zeros((D, N)), np.full(N, float(T))


def shear_wave(nx: int, ny: int, rho0: float, T: float, U: float = 1e-4):
    """u_x = U sin(2 pi y / ny) on a uniform state."""
    N = nx * ny
    y = np.repeat(np.arange(ny, dtype=np.float64), nx)
    u = np.zeros((2, N))
    u[0] = U * np.sin(2.0 * np.pi * y / ny)
    return np.full(N, float(rho0)), u, np.full(N, float(T))


def sound_wave(nx: int, ny: int, rho0: float, T: float, amplitude: float = 1e-4):
    """rho = rho0 (1 + A cos(2 pi x / nx)), u = 0, uniform T."""
    N = nx * ny
    x = np.tile(np.arange(nx, dtype=np.float64), ny)
    return rho0 * (1.0 + amplitude * np.cos(2.0 * np.pi * x / nx)), np.zeros((2, N)), np.full(N, float(T))


def ensemble_domains(n: int = 512, seed: int = DEFAULT_SEED, side_min: int = 64, side_max: int = 512,
                     side_step: int = 16, r_range=(8.0, 48.0), gap_range=(2.0, 10.0), tr_range=(0.7, 0.9)):
    """Uneven 2-D domains, each with two droplets on the x axis through its centre.
    Returns a list of dicts: nx, ny, r1, r2, gap, tr (T/Tc)."""
    rng = np.random.default_rng(seed)
    sides = np.arange(side_min, side_max + 1, side_step)
    out = []
    for _ in range(n):
        nx, ny = int(rng.choice(sides)), int(rng.choice(sides))
        gap = float(rng.uniform(*gap_range))
        tr = float(rng.uniform(*tr_range))
        for _attempt in range(1000):
            r1, r2 = (float(v) for v in rng.uniform(*r_range, size=2))
            if 2 * (r1 + r2) + gap + 16 <= nx and 2 * max(r1, r2) + 8 <= ny:
                break
        else:
            r1 = r2 = max(r_range[0], min((nx - gap - 16) / 4.0, (ny - 8) / 2.0))
        out.append(dict(nx=nx, ny=ny, r1=r1, r2=r2, gap=gap, tr=tr))
    return out


def two_droplets(nx: int, ny: int, r1: float, r2: float, gap: float, rho_v: float, rho_l: float, T: float,
                 width: float = 4.0):
    """Two droplets on the x axis through the domain centre, surfaces `gap` apart; the
    pair (extent 2 r1 + gap + 2 r2) is centred in the domain, so droplets of unequal
    radii stay clear of the periodic boundary when the pair fits."""
    cy = 0.5 * (ny - 1)
    left = 0.5 * (nx - 1) - 0.5 * (2.0 * r1 + gap + 2.0 * r2)
    c1 = left + r1
    c2 = c1 + r1 + gap + r2
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    d = np.maximum(r1 - np.hypot(x - c1, y - cy), r2 - np.hypot(x - c2, y - cy))
    rho = tanh_profile(d, rho_v, rho_l, width).reshape(-1)
    N = rho.size
    return rho, np.zeros((2, N)), np.full(N, float(T))
