"""Pins of the oracle's multiple-relaxation-time collision and Guo body force
(no GPU).

The collision relaxes the shear stress at 1/tau, the bulk stress at
1/tau_bulk and the 9 ghost directions of D3Q19 at 1/tau_ghost; the Guo force
F adds F to the momentum of every site per step.  Each test checks the oracle
against a fact that does not come from its code: the BGK limit, exact
per-mode decay factors on uniform states (the perturbations are built here
from the lattice tensors and a numpy null space), an exact one-step closed
form of the forced collision at tau = 1, exact momentum gain, the shear-wave
decay rate (independent of the bulk and ghost rates) and the attenuation of
a sound wave (which the bulk rate sets).
"""
import math

import numpy as np
import pytest

import lb_inputs as L
import oracle

P0 = dict(L.DEFAULT_PARAMS)
CS2 = 1.0 / 3.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _lattice():
    c, w = oracle.velocity_set()
    return c.astype(float), w


def _herm2(w, c, E):
    """w_i Q_i:E / (2 cs2^2) for a symmetric 3x3 E."""
    Q = np.einsum("ia,ib->iab", c, c) - CS2 * np.eye(3)
    return w * np.einsum("iab,ab->i", Q, E) / (2 * CS2 * CS2)


def _ghost_basis(c):
    """Orthonormal basis (rows) of the vectors whose moments 1, c_a, c_a c_b
    all vanish: 19 - 10 = 9 of them."""
    rows = [np.ones(19)] + [c[:, a] for a in range(3)]
    rows += [c[:, a] * c[:, b] for a in range(3) for b in range(a, 3)]
    M = np.array(rows)
    _, s, vt = np.linalg.svd(M)
    assert (s > 1e-10).sum() == 10
    return vt[10:]


def _uniform(n, rho, u, phi=0.0):
    """Uniform equilibrium (oracle order) of a fluid at rest in a frame
    moving with u; built by the oracle's init at rho0 = rho."""
    p = dict(P0, rho0=rho)
    dims = (n, 1, 1)
    return oracle.init(dims, p, np.full(n, phi), np.tile(np.asarray(u, float)[:, None], (1, n))), p


def test_equal_rates_without_force_is_bgk():
    dims = (8, 6, 5)
    n = 240
    p = dict(P0, tau=0.7, tau_g=0.9)
    f, g = oracle.init(dims, p, L.spinodal_phi0(*dims, seed=601, amp=0.5),
                       0.02 * L.uniform(602, 3 * n, -1, 1).reshape(3, n))
    f = f * (1 + 0.05 * L.uniform(603, 19 * n, -1, 1).reshape(19, n))
    for npts in (7, 19):
        fb, gb = oracle.step(dims, p, f, g, 6, npts=npts)
        fm, gm = oracle.step_mrt(dims, p, f, g, 6, 0.7, 0.7, npts=npts)
        assert np.abs(fm - fb).max() < 1e-14 and np.abs(gm - gb).max() < 1e-14


@pytest.mark.parametrize("sector", ["shear", "bulk", "ghost"])
def test_uniform_mode_decays_by_its_own_rate(sector):
    c, w = _lattice()
    tau, tau_b, tau_gh = 0.7, 1.3, 0.55
    n = 3
    (f0, g0), p = _uniform(n, 1.1, (0.02, -0.01, 0.03), phi=0.2)
    p = dict(p, tau=tau)
    if sector == "shear":
        E = np.array([[0.3, 0.1, -0.2], [0.1, -0.5, 0.05], [-0.2, 0.05, 0.2]]) * 1e-3
        h, rate = _herm2(w, c, E), 1 / tau
    elif sector == "bulk":
        h, rate = _herm2(w, c, 1e-3 * np.eye(3)), 1 / tau_b
    else:
        h, rate = 1e-3 * L.uniform(604, 9, -1, 1) @ _ghost_basis(c), 1 / tau_gh
    f = f0 + h[:, None]
    for t in (1, 2, 5):
        ft, gt = oracle.step_mrt((n, 1, 1), p, f, g0, t, tau_b, tau_gh)
        want = (1 - rate) ** t * h
        assert np.abs(ft - f0 - want[:, None]).max() < 1e-15
        assert np.abs(gt - g0).max() < 1e-15


def test_forced_collision_closed_form_at_unit_rates():
    """tau = tau_bulk = tau_ghost = 1, uniform equilibrium at u0, phi = 0:
    one step gives w_i [rho + c.J/cs2 + Q:(rho v v - F F/(4 rho))/(2 cs2^2)]
    with J = rho u0 + F and v = J/rho."""
    c, w = _lattice()
    rho, u0, F = 1.05, np.array([0.01, 0.02, -0.015]), np.array([2e-4, -1e-4, 3e-4])
    n = 2
    (f0, g0), p = _uniform(n, rho, u0)
    p = dict(p, tau=1.0)
    f1, _ = oracle.step_mrt((n, 1, 1), p, f0, g0, 1, 1.0, 1.0, tuple(F))
    J = rho * u0 + F
    v = J / rho
    want = w * (rho + c @ J / CS2) + _herm2(w, c, rho * np.outer(v, v) - np.outer(F, F) / (4 * rho))
    assert np.abs(f1 - want[:, None]).max() < 2e-16


def test_force_adds_F_to_every_site_momentum():
    dims = (8, 6, 5)
    n = 240
    p = dict(P0, tau=0.8, tau_g=0.9)
    F = (3e-5, -2e-5, 1e-5)
    f, g = oracle.init(dims, p, L.spinodal_phi0(*dims, seed=605, amp=0.5),
                       0.02 * L.uniform(606, 3 * n, -1, 1).reshape(3, n))
    c, _ = _lattice()
    for t in (1, 4):
        ft, gt = oracle.step_mrt(dims, p, f, g, t, 1.2, 0.9, F)
        dj = (ft.T @ c).sum(0) - (f.T @ c).sum(0)
        assert np.abs(dj - t * n * np.array(F)).max() < 1e-13
        assert abs(ft.sum() - f.sum()) < 1e-12 and abs(gt.sum() - g.sum()) < 1e-12


@pytest.mark.parametrize("rates", [(1.5, 0.6), (0.6, 1.9)])
def test_shear_wave_decay_independent_of_bulk_and_ghost(rates):
    tau, n = 0.8, 128
    dims = (n, 1, 1)
    k = 2 * math.pi / n
    x = np.arange(n)
    f0, g0 = oracle.init(dims, dict(P0, tau=tau), np.zeros(n), L.shear_wave_u0(*dims, amp=0.01))

    def amp_series(step):
        f, g = f0, g0
        out = []
        for _ in range(6):
            f, g = step(f, g)
            _, u, _ = oracle.moments(dims, f, g)
            out.append(2 / n * np.sum(u[1] * np.sin(k * x)))
        return np.array(out)

    p = dict(P0, tau=tau)
    a_bgk = amp_series(lambda f, g: oracle.step(dims, p, f, g, 400))
    a_mrt = amp_series(lambda f, g: oracle.step_mrt(dims, p, f, g, 400, *rates))
    rate_b = -np.polyfit(400 * np.arange(1, 7), np.log(a_bgk), 1)[0]
    rate_m = -np.polyfit(400 * np.arange(1, 7), np.log(a_mrt), 1)[0]
    nu = (tau - 0.5) / 3
    # the bulk and ghost rates enter the shear-wave rate only at O(k^2)
    # relative (here k^2 = 2.4e-3)
    assert abs(rate_m / rate_b - 1) < 2e-3
    assert abs(rate_m / (nu * k * k) - 1) < 3e-3


@pytest.mark.parametrize("tau_b", [0.8, 1.6])
def test_sound_attenuation_sets_bulk_viscosity(tau_b):
    """A standing density wave rho = 1 + eps cos(kx) (u = 0, phi = 0) loses
    acoustic energy as exp(-2 Gamma t), Gamma = k^2 [(4/3) nu + nu_b] / 2,
    nu = (tau - 1/2)/3, nu_b = (2/9)(tau_bulk - 1/2)."""
    c, w = _lattice()
    tau, n, eps = 0.8, 64, 1e-4
    dims = (n, 1, 1)
    k = 2 * math.pi / n
    rho = 1 + eps * np.cos(k * np.arange(n))
    f = w[:, None] * rho[None, :]                 # equilibrium at u = 0, phi = 0
    g = np.zeros_like(f)
    p = dict(P0, tau=tau)
    ts, en = [], []
    for t in range(0, 1201, 4):
        if t:
            f, g = oracle.step_mrt(dims, p, f, g, 4, tau_b, 1.0)
        r = f.sum(0)
        j = f.T @ c
        en.append(np.sum(CS2 * (r - 1) ** 2 + (j ** 2).sum(1) / r))
        ts.append(t)
    ts, en = np.array(ts), np.array(en)
    m = ts >= 200
    gamma = -np.polyfit(ts[m], np.log(en[m]), 1)[0] / 2
    nu, nu_b = (tau - 0.5) / 3, 2 / 9 * (tau_b - 0.5)
    want = k * k * (4 / 3 * nu + nu_b) / 2
    assert abs(gamma / want - 1) < 0.03, (gamma, want)


def test_forced_stress_follows_the_momentum_at_any_rates():
    """Guo's (1 - w/2) factors make the post-collision second moment of a
    uniform forced fluid equal to the equilibrium one at the post-collision
    momentum, rho cs2 I + rho v v with v = (j + F)/rho, up to O(F^2) and for
    any shear / bulk / ghost rates (a wrong factor leaves an O(u.F) error)."""
    c, w = _lattice()
    rho, u0, F = 1.0, np.array([0.05, -0.03, 0.04]), np.array([1e-4, 2e-4, -1e-4])
    n = 2
    (f0, g0), p = _uniform(n, rho, u0)
    p = dict(p, tau=0.7)
    f1, _ = oracle.step_mrt((n, 1, 1), p, f0, g0, 1, 1.4, 0.9, tuple(F))
    v = (rho * u0 + F) / rho
    Pi = np.einsum("ia,ib,i->ab", c, c, f1[:, 0])
    want = rho * CS2 * np.eye(3) + rho * np.outer(v, v)
    # O(F^2) remainder: at most max(1/tau, 1/tau_bulk) max|F_a F_b| / (4 rho) = 1.4e-8
    assert np.abs(Pi - want).max() < 2e-8
