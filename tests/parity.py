"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the CPU oracle on the same seeded inputs and compare."""
import numpy as np

import lb_inputs as L
import oracle
from tests import bruteforce_lb as BF

P0 = dict(L.DEFAULT_PARAMS)

# Per-field error used throughout: max |a - b| scaled by the field's max-norm
# (fields such as u and phi can be ~0 at many sites, so a per-site relative
# error would be undefined there).
TOL_FP64 = 1e-12


def rel(a, b, scale=None):
    a = np.asarray(a, dtype=float)
    b = np.asarray(b, dtype=float)
    scale = np.abs(b).max() if scale is None else max(scale, np.abs(b).max())
    d = np.abs(a - b).max()
    return d / scale if scale > 0 else d


def u_scale(f):
    """Size of the terms whose sum gives u = sum_i f_i c_i / rho: the max over
    sites and components of sum_i |f_i c_ia| / rho (oracle-order state).

    Any floating-point evaluation of the sum carries an absolute error of
    about eps times this, so u's error is measured against it: early in a
    spinodal or interface run |u| is ~1e-8 while the summands are ~0.1, and
    a scale of max|u| alone would ask for more digits than the data hold.
    """
    c, _ = oracle.velocity_set()
    f = np.asarray(f, dtype=float)
    rho = f.sum(0)
    s = np.abs(f).T @ np.abs(c).astype(float)          # [N, 3]
    return float((s / rho[:, None]).max())


def abi_order():
    """Index map o2a with abi_row = o2a[oracle_row]."""
    from paper_1405_6162_gb300 import VELOCITIES
    c, _ = oracle.velocity_set()
    return BF.map_order(c, VELOCITIES)


def to_abi(x):
    o2a = abi_order()
    out = np.empty_like(x)
    out[o2a] = x
    return out


def to_oracle(x):
    return np.asarray(x)[abi_order()]


def gpu_lattice(dims, params, precision="fp64", kernel="auto", block=(0, 0, 0)):
    from paper_1405_6162_gb300 import Lattice
    lat = Lattice.from_params(dims, params, precision=precision)
    lat.set_kernel(kernel, *block)
    return lat


def nonequilibrium_state(dims, params, seed, amp=0.5):
    """A seeded state away from equilibrium (oracle order): equilibrium of a
    random phi field with random flow, then perturbed per direction."""
    n = int(np.prod(dims))
    f, g = oracle.init(dims, params, L.spinodal_phi0(*dims, seed=seed, amp=amp),
                       0.02 * L.uniform(seed + 1, 3 * n, -1, 1).reshape(3, n))
    f = f * (1 + 0.05 * L.uniform(seed + 2, 19 * n, -1, 1).reshape(19, n))
    g = g + 0.01 * L.uniform(seed + 3, 19 * n, -1, 1).reshape(19, n)
    return f, g
