"""Long runs of the benchmark workloads, checked against the oracle and
against closed forms.

* Spinodal decomposition, 64^3, 1000 steps (seed 1): per-field error of the
  FP64 and FP32-shifted forms against the FP64 oracle.  The instability
  amplifies rounding by ~e^(sigma_max t) (sigma_max ~ 0.006/step at these
  parameters, ~400x over 1000 steps), which bounds what any precision can
  reproduce; the measured errors are printed.
* Shear wave at 256^3: u_y = U sin(2 pi x/256) decays at nu k^2,
  nu = (tau - 1/2)/3.
* Flat interfaces at 256^3 started on the discrete mu = 0 profile (Newton)
  stay on it.
"""
import math

import numpy as np
import pytest

import lb_inputs as L
import oracle
from tests.parity import P0, rel, u_scale

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    import paper_1405_6162_gb300 as lbpkg
    lbpkg.build()
    oracle.build()


@pytest.fixture(scope="module")
def spinodal_reference():
    dims = (64, 64, 64)
    phi0 = L.spinodal_phi0(*dims, seed=1)
    f, g = oracle.step(dims, P0, *oracle.init(dims, P0, phi0), 1000, kind="omp")
    return dims, phi0, oracle.moments(dims, f, g), u_scale(f)


@pytest.mark.parametrize("precision,kernel,bounds", [
    ("fp64", "auto", {"rho": 1e-12, "u": 1e-12, "phi": 1e-12}),
    ("fp32_shifted", "auto", {"rho": 1e-7, "u": 1e-7, "phi": 1e-5}),
    ("fp64", "taug1", {"rho": 1e-12, "u": 1e-12, "phi": 1e-12}),
    ("fp32_shifted", "taug1", {"rho": 1e-7, "u": 1e-7, "phi": 1e-5}),
])
def test_spinodal_64cubed_1000_steps(spinodal_reference, precision, kernel, bounds):
    """FP64 at the 1e-12 bar (measured: rho 1.5e-15, u 1.1e-15, phi 1.4e-13);
    the FP32 bounds are the 1e-5 aimed for (measured: phi 3.0e-6 two-pass,
    6.5e-6 reduced form; rho, u ~3e-8)."""
    from paper_1405_6162_gb300 import Lattice
    dims, phi0, want, us = spinodal_reference
    with Lattice.from_params(dims, P0, precision=precision) as lat:
        lat.set_kernel(kernel)
        lat.init(phi0)
        r0 = lat.reduce()
        lat.step(1000)
        r1 = lat.reduce()
        got = lat.moments()
    errs = {k: rel(a, b, us if k == "u" else None) for k, a, b in zip(("rho", "u", "phi"), got, want)}
    print(f"spinodal 64^3 x 1000 {precision} {kernel}: {errs}  (max|phi| = {np.abs(want[2]).max():.3f})")
    for k, e in errs.items():
        assert e <= bounds[k], (k, e)
    # sum phi is conserved up to unbiased rounding (float weights that do not
    # sum to 1 would drift it by ~1.5e-8 of sum |phi| per step, 1.5e-5 here)
    drift = abs(r1[4] - r0[4]) / np.abs(got[2]).sum()
    assert drift < (1e-13 if precision == "fp64" else 1e-6), drift


@pytest.mark.parametrize("precision", ["fp64", "fp32_shifted"])
@pytest.mark.parametrize("tau", [0.6, 0.8, 1.0])
def test_shear_wave_decay_rate_256cubed(precision, tau):
    from paper_1405_6162_gb300 import Lattice
    n = 256
    dims = (n, n, n)
    p = dict(P0, tau=tau)
    u0 = L.shear_wave_u0(*dims, amp=0.01)
    k = 2 * math.pi / n
    x = np.arange(n)
    steps = 1000 if precision == "fp64" else 2000
    ts, amps = [], []
    with Lattice.from_params(dims, p, precision=precision) as lat:
        lat.init(np.zeros(n ** 3), u0)
        t = 0
        for t_next in range(0, steps + 1, steps // 5):
            lat.step(t_next - t)
            t = t_next
            _, u, _ = lat.moments(device=True)
            uy = u[1].reshape(n, n, n)[0, 0].cpu().numpy()     # one x-line (uniform in y, z)
            ts.append(t)
            amps.append(2 / n * np.sum(uy * np.sin(k * x)))
    ts = np.array(ts)
    sel = ts >= steps // 5
    rate = -np.polyfit(ts[sel], np.log(np.array(amps))[sel], 1)[0]
    nu = (tau - 0.5) / 3
    print(f"shear wave tau={tau} {precision}: rate {rate:.6e} vs nu k^2 {nu * k * k:.6e}")
    # FP64: the lattice rate equals nu k^2 to O(k^2) (1e-3).  FP32: each step
    # changes a stored value by a fraction nu k^2 of itself, only ~1/(nu k^2)
    # ulps, so float rounding bounds the measured rate to ~2^-23 / (nu k^2)
    # (6e-3 at tau = 0.6, 1.2e-3 at tau = 1)
    tol = 1e-3 if precision == "fp64" else max(1e-3, 2.0 ** -23 / (nu * k * k))
    assert abs(rate / (nu * k * k) - 1) < tol


def _newton_profile(n, amplitude=1.0):
    A, B, kap = P0["A"], P0["B"], P0["kappa"]
    xi = L.interface_width(A, kap)
    p = L.flat_interface_phi0(n, 1, 1, amplitude, xi)
    idx = np.arange(n)
    for _ in range(50):
        r = A * p + B * p ** 3 - kap * (np.roll(p, 1) + np.roll(p, -1) - 2 * p)
        J = np.zeros((n, n))
        J[idx, idx] = A + 3 * B * p ** 2 + 2 * kap
        J[idx, (idx + 1) % n] -= kap
        J[idx, (idx - 1) % n] -= kap
        p = p - np.linalg.solve(J, r)
    return p


# the start has uniform density, so the pressure balance across the
# interfaces is restored by a transient that advects phi by ~1e-4 (both
# precisions alike) -- still 100x below the continuum profile's deviation
@pytest.mark.parametrize("precision,tol", [("fp64", 5e-4), ("fp32_shifted", 5e-4)])
def test_discrete_interface_profile_is_kept_256cubed(precision, tol):
    """Started on the discrete mu = 0 profile (the LB steady state), two flat
    interfaces stay on it; the continuum tanh(x/xi) differs from it by the
    stencil's discretisation error (a few 1e-2 at xi ~ 1.13)."""
    from paper_1405_6162_gb300 import Lattice
    n = 256
    pn = _newton_profile(n)
    xi = L.interface_width(P0["A"], P0["kappa"])
    cont = L.flat_interface_phi0(n, 1, 1, 1.0, xi)
    assert 0.005 < np.abs(pn - cont).max() < 0.05
    with Lattice.from_params((n, n, n), P0, precision=precision) as lat:
        lat.init(np.ascontiguousarray(np.broadcast_to(pn, (n * n, n))).reshape(-1))
        lat.step(500)
        _, _, phi = lat.moments(device=True)
        line = phi.reshape(n, n, n)[7, 3].cpu().numpy()
        spread = float((phi.reshape(n * n, n) - phi.reshape(n * n, n)[0]).abs().max())
    dev = np.abs(line - pn).max()
    print(f"interface 256^3 {precision}: max |phi - newton| after 500 steps {dev:.3e}, y/z spread {spread:.1e}")
    assert dev <= tol and spread <= 1e-12
