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
    try:
        lat.set_kernel(kernel, *block)
    except Exception:
        lat.close()
        raise
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


# ------------------------------------------------------------------ the 64-lattice ensemble workload

ENSEMBLE_STEPS = 500


def ensemble_workload():
    """The 64 lattices (sides U{16..64}, tau ~ U[0.55, 1.5], kappa ~
    U[0.01, 0.08], seed 3) and their spinodal starts (seed 1000 + k)."""
    specs = L.ensemble(3, 64)
    phis = [L.spinodal_phi0(d["nx"], d["ny"], d["nz"], seed=1000 + k) for k, d in enumerate(specs)]
    return specs, phis


def sites(spec):
    return spec["nx"] * spec["ny"] * spec["nz"]


def spinodal_rate(spec):
    """Largest linear growth rate per step of a small phi perturbation about
    phi = 0: sigma_max = M A^2 / (4 kappa), M = Gamma (tau_g - 1/2) (the
    maximum over k of -M k^2 (A + kappa k^2); pinned in the oracle tests)."""
    return spec["gamma"] * (spec["tau_g"] - 0.5) * spec["A"] ** 2 / (4.0 * spec["kappa"])


def ensemble_subsample(specs):
    """At least 8 lattices that cover the workload's extremes: the two
    largest (longest work lists, deepest CTA groups), the smallest, the most
    and least unstable (smallest and largest kappa), the smallest and largest
    tau, and the lattice whose growth factor over the run is next after the
    two most unstable."""
    idx = range(len(specs))
    by_size = sorted(idx, key=lambda k: sites(specs[k]))
    by_rate = sorted(idx, key=lambda k: spinodal_rate(specs[k]))
    by_tau = sorted(idx, key=lambda k: specs[k]["tau"])
    pick = [by_size[-1], by_size[-2], by_size[0], by_rate[-1], by_rate[0], by_tau[0], by_tau[-1], by_rate[-3]]
    out = []
    for k in pick:
        if k not in out:
            out.append(k)
    for k in reversed(by_size):            # top up with the next largest
        if len(out) >= 9:
            break
        if k not in out:
            out.append(k)
    return out


_ENSEMBLE_ORACLE = {}


def ensemble_oracle(k, nsteps=ENSEMBLE_STEPS):
    """Oracle moments of lattice k of the workload after nsteps, and the
    scale of u's summands (cached for the session: both ensemble forms are
    compared with the same runs)."""
    if (k, nsteps) not in _ENSEMBLE_ORACLE:
        specs, phis = ensemble_workload()
        d = specs[k]
        dims = (d["nx"], d["ny"], d["nz"])
        f, g = oracle.step(dims, d, *oracle.init(dims, d, phis[k]), nsteps, kind="omp")
        _ENSEMBLE_ORACLE[(k, nsteps)] = (oracle.moments(dims, f, g), u_scale(f))
    return _ENSEMBLE_ORACLE[(k, nsteps)]


# FP32-shifted bounds of the 64^3 x 1000 spinodal run (kappa = 0.04):
# phi 1e-5 (measured 3.0e-6), rho and u 1e-7 (measured ~3e-8).  Float
# rounding is injected every step and amplified by the spinodal instability
# at most by the growth factor exp(sigma_max t) of the run, 446 for that
# reference (sigma_max T = 6.10).
FP32_SPINODAL_BOUNDS = {"rho": 1e-7, "u": 1e-7, "phi": 1e-5}
FP32_REFERENCE_GROWTH = 6.1035  # sigma_max T of the 64^3 x 1000 run at the default parameters


def fp32_spinodal_bounds(spec, nsteps):
    """The reference bounds, scaled by how much more unstable this run is
    (exp(sigma_max T) beyond the reference's); never looser for a more
    stable run."""
    excess = max(0.0, spinodal_rate(spec) * nsteps - FP32_REFERENCE_GROWTH)
    return {k: v * float(np.exp(excess)) for k, v in FP32_SPINODAL_BOUNDS.items()}
