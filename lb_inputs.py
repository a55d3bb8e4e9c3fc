"""Seeded synthetic inputs for the binary-fluid D3Q19 lattice Boltzmann step.

This module is the only code shared by the CUDA path's callers and by the
CPU oracle's callers.  It holds no arithmetic of the method itself (no
equilibrium, stencil, collision or streaming): only the counter-based random
generator and the recipes that turn its output into initial fields and
parameter tables.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: output k of stream ``seed`` is the SplitMix64 finaliser applied to
``seed + (k + 1) * 0x9E3779B97F4A7C15`` (mod 2**64), and a uniform double in
[0, 1) is its top 53 bits times 2**-53.

Site order everywhere is x fastest: ``idx = x + nx * (y + ny * z)``; a field
is a flat float64 array of ``nx * ny * nz`` values (vector fields are SoA,
``[3][N]``).
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Parameters shared by every workload of the binary-fluid benchmark family:
# tau = 1, rho0 = 1, u = 0, Gamma = 0.5, A = -0.0625, B = 0.0625,
# kappa = 0.04; the order-parameter relaxation time tau_g defaults to 1.
DEFAULT_PARAMS = dict(tau=1.0, tau_g=1.0, rho0=1.0, gamma=0.5,
                      A=-0.0625, B=0.0625, kappa=0.04)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+n-1`` of the SplitMix64 stream ``seed``."""
    k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0,
            offset: int = 0) -> np.ndarray:
    """``n`` doubles uniform in [lo, hi) from stream ``seed``."""
    u = (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64)
    u *= 2.0 ** -53
    return lo + (hi - lo) * u


def uniform_int(seed: int, n: int, lo: int, hi: int, offset: int = 0) -> np.ndarray:
    """``n`` integers uniform in the closed range [lo, hi]."""
    u = uniform(seed, n, 0.0, 1.0, offset)
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)


def spinodal_phi0(nx: int, ny: int, nz: int, seed: int, amp: float = 0.01) -> np.ndarray:
    """phi0 i.i.d. uniform in [-amp, amp] (the spinodal-decomposition start)."""
    return uniform(seed, nx * ny * nz, -amp, amp)


def interface_width(A: float, kappa: float) -> float:
    """Width xi = sqrt(-2 kappa / A) of the symmetric tanh interface."""
    return math.sqrt(-2.0 * kappa / A)


def flat_interface_phi0(nx: int, ny: int, nz: int, amplitude: float, xi: float) -> np.ndarray:
    """Two flat interfaces normal to x on a periodic box.

    phi = a*tanh((x - L/4)/xi) for x < L/2 and a*tanh((3L/4 - x)/xi)
    otherwise, evaluated at integer x; uniform in y and z.
    """
    L = nx
    x = np.arange(nx, dtype=np.float64)
    prof = np.where(x < L / 2, amplitude * np.tanh((x - L / 4) / xi),
                    amplitude * np.tanh((3 * L / 4 - x) / xi))
    return np.ascontiguousarray(np.broadcast_to(prof, (nz, ny, nx))).reshape(-1).copy()


def shear_wave_u0(nx: int, ny: int, nz: int, amp: float = 0.01, mode: int = 1) -> np.ndarray:
    """Velocity [3][N] with u_y = amp * sin(2 pi mode x / nx), u_x = u_z = 0."""
    n = nx * ny * nz
    x = np.arange(nx, dtype=np.float64)
    uy = amp * np.sin(2.0 * math.pi * mode * x / nx)
    u = np.zeros((3, n))
    u[1] = np.broadcast_to(uy, (nz, ny, nx)).reshape(-1)
    return u


def cosine_mode_phi0(nx: int, ny: int, nz: int, eps: float, mode: int) -> np.ndarray:
    """phi0 = eps * cos(2 pi mode x / nx), uniform in y and z."""
    x = np.arange(nx, dtype=np.float64)
    prof = eps * np.cos(2.0 * math.pi * mode * x / nx)
    return np.ascontiguousarray(np.broadcast_to(prof, (nz, ny, nx))).reshape(-1).copy()


def droplet_target(nx: int, ny: int, nz: int, radius: float, xi: float,
                   seed: int, phi_star: float = 1.0) -> np.ndarray:
    """phi_target = phi* tanh((R - r)/xi), positive inside a droplet.

    Centre = box centre plus a seeded offset in [-4, 4]^3; r is the
    minimum-image distance on the periodic box.
    """
    off = uniform(seed, 3, -4.0, 4.0)
    cx, cy, cz = nx / 2 + off[0], ny / 2 + off[1], nz / 2 + off[2]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")

    def mi(d, L):
        return d - L * np.round(d / L)

    r = np.sqrt(mi(x - cx, nx) ** 2 + mi(y - cy, ny) ** 2 + mi(z - cz, nz) ** 2)
    return (phi_star * np.tanh((radius - r) / xi)).reshape(-1)


def ensemble(seed: int, n: int, lo: int = 16, hi: int = 64):
    """Parameter table of an ensemble of ``n`` independent periodic lattices.

    Side lengths i.i.d. uniform integers in [lo, hi] (non-cubic allowed),
    tau ~ U[0.55, 1.5], kappa ~ U[0.01, 0.08]; the other parameters are
    ``DEFAULT_PARAMS``.  Returns a list of dicts with keys nx, ny, nz and the
    parameter names.
    """
    dims = uniform_int(seed, 3 * n, lo, hi).reshape(n, 3)
    tau = uniform(seed + 1, n, 0.55, 1.5)
    kappa = uniform(seed + 2, n, 0.01, 0.08)
    out = []
    for k in range(n):
        p = dict(DEFAULT_PARAMS)
        p.update(nx=int(dims[k, 0]), ny=int(dims[k, 1]), nz=int(dims[k, 2]),
                 tau=float(tau[k]), kappa=float(kappa[k]))
        out.append(p)
    return out
