"""CPU oracle of the binary-fluid D3Q19 lattice Boltzmann timestep.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package smoke check
and by the benchmark's CPU-baseline leg, never by the CUDA library or its
Python binding.  It shares no code with the CUDA path.

The arithmetic lives in ``lb_oracle.c`` (plain FP64 C, built with
``-O2 -ffp-contract=off``); this module compiles it with gcc on first use
and wraps it with ctypes over numpy arrays.  Three builds of the one source
are made: ``serial`` (the oracle proper), ``omp`` (the same loops with
OpenMP on, used only to time the baseline on all host cores) and
``complex`` (``-DORC_COMPLEX``: every value is ``double complex``, for
complex-step derivatives).

Parameters are a dict with keys tau, tau_g, rho0, gamma, A, B, kappa.
Fields are flat arrays in site order ``x + nx*(y + ny*z)``; distributions
are ``[19][N]`` in the oracle's own velocity order (``velocity_set()``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = [os.path.join(_HERE, "lb_oracle.c")]
_FLAGS = {
    "serial": ["-O2", "-ffp-contract=off"],
    "omp": ["-O2", "-ffp-contract=off", "-fopenmp"],
    "complex": ["-O2", "-ffp-contract=off", "-DORC_COMPLEX"],
}
_LIBS: dict = {}
_LOCK = threading.Lock()

PARAM_ORDER = ("tau", "tau_g", "rho0", "gamma", "A", "B", "kappa")
NV = 19


def _so_path(kind: str) -> str:
    return os.path.join(_BUILD, f"liblb_oracle_{kind}.so")


def build(force: bool = False) -> None:
    """Compile every oracle build with gcc (no-op when up to date)."""
    os.makedirs(_BUILD, exist_ok=True)
    src_m = max(os.path.getmtime(s) for s in _SRC)
    for kind, flags in _FLAGS.items():
        so = _so_path(kind)
        if not force and os.path.exists(so) and os.path.getmtime(so) >= src_m:
            continue
        tmp = so + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c99", "-shared", "-fPIC", *flags, *_SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, so)


def _lib(kind: str = "serial"):
    with _LOCK:
        if kind not in _LIBS:
            build()
            _LIBS[kind] = ctypes.CDLL(_so_path(kind))
        return _LIBS[kind]


def _dtype(kind):
    return np.complex128 if kind == "complex" else np.float64


def _arr(a, kind):
    a = np.ascontiguousarray(a, dtype=_dtype(kind))
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _prm(params, kind):
    vals = [params[k] for k in PARAM_ORDER]
    dt = np.complex128 if kind == "complex" else np.float64
    return _arr(np.array(vals, dtype=dt), kind)


def threads(kind: str = "omp") -> int:
    """Threads the parallel loops of build ``kind`` use (1 for serial)."""
    return int(_lib(kind).orc_threads())


def velocity_set():
    """(c[19,3] int, w[19] float64) in the oracle's order."""
    c = np.zeros(57, dtype=np.int32)
    w = np.zeros(19)
    _lib().orc_velocity_set(c.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p))
    return c.reshape(19, 3), w


STENCILS = (7, 19, 27)


def _npts(npts):
    if npts not in STENCILS:
        raise ValueError(f"stencil must be one of {STENCILS}")
    return int(npts)


def gradients(dims, phi, kind="serial", npts=7):
    """(grad [3][N], lap [N]) of phi by the 7-point stencils, or the
    isotropic 19- / 27-point ones (``npts``)."""
    nx, ny, nz = dims
    n = nx * ny * nz
    phi, pp = _arr(phi, kind)
    grad = np.zeros(3 * n, dtype=_dtype(kind))
    lap = np.zeros(n, dtype=_dtype(kind))
    _lib(kind).orc_gradients_n(nx, ny, nz, _npts(npts), pp, grad.ctypes.data_as(ctypes.c_void_p),
                               lap.ctypes.data_as(ctypes.c_void_p))
    return grad.reshape(3, n), lap


def site_thermo(params, phi, d, lap, kind="serial"):
    """(mu, P[3,3]) at one site."""
    prm, pp = _prm(params, kind)
    d, dp = _arr(d, kind)
    mu = np.zeros(1, dtype=_dtype(kind))
    P = np.zeros(9, dtype=_dtype(kind))
    lib = _lib(kind)
    if kind == "complex":
        raise NotImplementedError("site_thermo is exposed for the FP64 build")
    lib.orc_site_thermo(pp, ctypes.c_double(phi), dp, ctypes.c_double(lap),
                        mu.ctypes.data_as(ctypes.c_void_p), P.ctypes.data_as(ctypes.c_void_p))
    return float(mu[0]), P.reshape(3, 3)


def site_equilibrium(params, rho, j, phi, d, lap):
    """(feq[19], geq[19]) at one site (FP64 build)."""
    prm, pp = _prm(params, "serial")
    j, jp = _arr(j, "serial")
    d, dp = _arr(d, "serial")
    feq = np.zeros(19)
    geq = np.zeros(19)
    _lib().orc_site_equilibrium(pp, ctypes.c_double(rho), jp, ctypes.c_double(phi), dp,
                                ctypes.c_double(lap), feq.ctypes.data_as(ctypes.c_void_p),
                                geq.ctypes.data_as(ctypes.c_void_p))
    return feq, geq


def init(dims, params, phi0, u0=None, kind="serial", npts=7):
    """Equilibrium initial state (f, g), each [19][N] (stencils of ``npts``
    points for the initial gradients)."""
    nx, ny, nz = dims
    n = nx * ny * nz
    prm, pp = _prm(params, kind)
    phi0, php = _arr(phi0, kind)
    if u0 is not None:
        u0, up = _arr(np.reshape(u0, (3 * n,)), kind)
    else:
        up = None
    f = np.zeros(19 * n, dtype=_dtype(kind))
    g = np.zeros(19 * n, dtype=_dtype(kind))
    _lib(kind).orc_init_n(nx, ny, nz, _npts(npts), pp, php, up, f.ctypes.data_as(ctypes.c_void_p),
                          g.ctypes.data_as(ctypes.c_void_p))
    return f.reshape(19, n), g.reshape(19, n)


def step(dims, params, f, g, nsteps, kind="serial", npts=7):
    """Advance (f, g) by ``nsteps`` with the ``npts``-point stencils; returns
    new arrays (inputs untouched)."""
    nx, ny, nz = dims
    n = nx * ny * nz
    prm, pp = _prm(params, kind)
    f = np.array(f, dtype=_dtype(kind), copy=True).reshape(-1)
    g = np.array(g, dtype=_dtype(kind), copy=True).reshape(-1)
    _lib(kind).orc_step_n(nx, ny, nz, _npts(npts), pp, f.ctypes.data_as(ctypes.c_void_p),
                          g.ctypes.data_as(ctypes.c_void_p), int(nsteps))
    return f.reshape(19, n), g.reshape(19, n)


def step_mrt(dims, params, f, g, nsteps, tau_bulk, tau_ghost, force=(0.0, 0.0, 0.0), kind="serial", npts=7):
    """Advance (f, g) by ``nsteps`` with the multiple-relaxation-time
    collision of f (shear rate 1/tau, bulk 1/tau_bulk, ghosts 1/tau_ghost)
    and the Guo body force ``force``; returns new arrays."""
    nx, ny, nz = dims
    n = nx * ny * nz
    prm, pp = _prm(params, kind)
    mrt, mp = _arr(np.array([tau_bulk, tau_ghost, *force], dtype=_dtype(kind)), kind)
    f = np.array(f, dtype=_dtype(kind), copy=True).reshape(-1)
    g = np.array(g, dtype=_dtype(kind), copy=True).reshape(-1)
    _lib(kind).orc_step_mrt(nx, ny, nz, _npts(npts), pp, mp, f.ctypes.data_as(ctypes.c_void_p),
                            g.ctypes.data_as(ctypes.c_void_p), int(nsteps))
    return f.reshape(19, n), g.reshape(19, n)


def moments(dims, f, g, kind="serial"):
    """(rho [N], u [3][N], phi [N])."""
    nx, ny, nz = dims
    n = nx * ny * nz
    f, fp = _arr(np.reshape(f, -1), kind)
    g, gp = _arr(np.reshape(g, -1), kind)
    rho = np.zeros(n, dtype=_dtype(kind))
    u = np.zeros(3 * n, dtype=_dtype(kind))
    phi = np.zeros(n, dtype=_dtype(kind))
    _lib(kind).orc_moments(nx, ny, nz, fp, gp, rho.ctypes.data_as(ctypes.c_void_p),
                           u.ctypes.data_as(ctypes.c_void_p), phi.ctypes.data_as(ctypes.c_void_p))
    return rho, u.reshape(3, n), phi


def reduce(dims, f, g, kind="serial"):
    """[sum rho, sum rho u (3), sum phi]."""
    nx, ny, nz = dims
    f, fp = _arr(np.reshape(f, -1), kind)
    g, gp = _arr(np.reshape(g, -1), kind)
    out = np.zeros(5, dtype=_dtype(kind))
    _lib(kind).orc_reduce(nx, ny, nz, fp, gp, out.ctypes.data_as(ctypes.c_void_p))
    return out


def step_adjoint(dims, params, f, g, af, ag):
    """One reverse step: given F(t) = (f, g) and F_bar(t+1) = (af, ag),
    returns (F_bar(t) f-part, g-part, dJ/dkappa of this step)."""
    nx, ny, nz = dims
    n = nx * ny * nz
    prm, pp = _prm(params, "serial")
    f, fp = _arr(np.reshape(f, -1), "serial")
    g, gp = _arr(np.reshape(g, -1), "serial")
    af = np.array(af, dtype=np.float64, copy=True).reshape(-1)
    ag = np.array(ag, dtype=np.float64, copy=True).reshape(-1)
    dk = np.zeros(1)
    _lib().orc_step_adjoint(nx, ny, nz, pp, fp, gp, af.ctypes.data_as(ctypes.c_void_p),
                            ag.ctypes.data_as(ctypes.c_void_p), dk.ctypes.data_as(ctypes.c_void_p))
    return af.reshape(19, n), ag.reshape(19, n), float(dk[0])


def init_adjoint(dims, params, phi0, af0, ag0, u0=None):
    """Reverse of the initialisation: (dJ/dphi0 [N], dJ/dkappa of init)."""
    nx, ny, nz = dims
    n = nx * ny * nz
    prm, pp = _prm(params, "serial")
    phi0, php = _arr(phi0, "serial")
    up = None
    if u0 is not None:
        u0, up = _arr(np.reshape(u0, (3 * n,)), "serial")
    af0, ap = _arr(np.reshape(af0, -1), "serial")
    ag0, gp = _arr(np.reshape(ag0, -1), "serial")
    out = np.zeros(n)
    dk = np.zeros(1)
    _lib().orc_init_adjoint(nx, ny, nz, pp, php, up, ap, gp, out.ctypes.data_as(ctypes.c_void_p),
                            dk.ctypes.data_as(ctypes.c_void_p))
    return out, float(dk[0])


def trajectory_gradient(dims, params, phi0, phi_target, nsteps):
    """J = sum_x (phi_T - phi_target)^2 after ``nsteps`` from the equilibrium
    start, and (dJ/dphi0, dJ/dkappa) by the reverse sweep (all states kept:
    small lattices only)."""
    f, g = init(dims, params, phi0)
    states = [(f, g)]
    for _ in range(nsteps):
        f, g = step(dims, params, f, g, 1)
        states.append((f, g))
    phi_t = g.sum(0)
    J = float(np.sum((phi_t - phi_target) ** 2))
    af = np.zeros_like(f)
    ag = np.tile(2.0 * (phi_t - phi_target), (19, 1))
    dk = 0.0
    for t in range(nsteps - 1, -1, -1):
        af, ag, d = step_adjoint(dims, params, *states[t], af, ag)
        dk += d
    phi_bar, d = init_adjoint(dims, params, phi0, af, ag)
    return J, phi_bar, dk + d


def trajectory_loss(dims, params, phi0, phi_target, nsteps, kind="serial"):
    """J alone (any build; complex inputs give the complex-step derivative)."""
    f, g = init(dims, params, phi0, kind=kind)
    f, g = step(dims, params, f, g, nsteps, kind=kind)
    phi_t = g.sum(0)
    return np.sum((phi_t - phi_target) ** 2)


def select_sites(x, mask):
    """The values of x (last axis: sites in site order) at the sites whose
    mask byte is non-zero, in site order -- the masked copy-out of the
    paper's copyFromTargetMasked (Sec. III.B)."""
    x = np.asarray(x)
    keep = np.asarray(mask).reshape(-1) != 0
    return x[..., keep]


def scatter_sites(x, mask, values):
    """A copy of x with ``values`` (last axis: the selected sites in site
    order) written at the sites whose mask byte is non-zero -- the masked
    copy-in of copyToTargetMasked (Sec. III.B)."""
    out = np.array(x, copy=True)
    keep = np.asarray(mask).reshape(-1) != 0
    out[..., keep] = values
    return out
