"""Pins of the CPU oracle against what the mathematics fixes (no GPU).

The paper (targetDP, Sec. II.A and IV) names the method -- a lattice
Boltzmann collision of a two-fluid mixture on D3Q19 with finite-difference
order-parameter dynamics -- but prints no formulas.  Each test here checks
the oracle against a fact that does not come from the oracle itself: lattice
tensor identities, exact Fourier eigenvalues of the stencils, fixed points,
conservation, a continuum thermodynamic identity, hydrodynamic closed forms
(shear-wave decay, Galilean advection, linear spinodal growth), a discrete
interface profile found by Newton's method, and an independent
definition-level implementation on tiny lattices.
"""
import math

import numpy as np
import pytest

import lb_inputs as L
import oracle
from tests import bruteforce_lb as BF

P0 = dict(L.DEFAULT_PARAMS)


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


# --------------------------------------------------------------- lattice

def test_velocity_set_tensor_identities():
    c, w = oracle.velocity_set()
    assert c.shape == (19, 3) and len({tuple(v) for v in c}) == 19
    assert all(tuple(-v) in {tuple(u) for u in c} for v in c)
    d = np.eye(3)
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs(np.einsum("i,ia->a", w, c)).max() < 1e-16
    assert np.abs(np.einsum("i,ia,ib->ab", w, c, c) - d / 3).max() < 1e-16
    assert np.abs(np.einsum("i,ia,ib,ic->abc", w, c, c, c)).max() < 1e-16
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.abs(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c) - iso).max() < 1e-16


# --------------------------------------------------------------- stencils

@pytest.mark.parametrize("m", [(1, 0, 0), (2, 3, 1), (0, 1, 4)])
def test_stencil_exact_on_fourier_modes(m):
    dims = (8, 12, 10)
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    k = [2 * math.pi * m[a] / dims[a] for a in range(3)]
    th = (k[0] * x + k[1] * y + k[2] * z).reshape(-1)
    grad, lap = oracle.gradients(dims, np.cos(th))
    lam = sum(2 * math.cos(ka) - 2 for ka in k)
    assert np.abs(lap - lam * np.cos(th)).max() < 1e-13
    for a in range(3):
        assert np.abs(grad[a] + math.sin(k[a]) * np.sin(th)).max() < 1e-13


# --------------------------------------------------------------- equilibria

def test_equilibrium_moments():
    rng = np.random.default_rng(5)
    c, w = oracle.velocity_set()
    for _ in range(20):
        rho = 1 + 0.2 * rng.standard_normal()
        j = 0.05 * rng.standard_normal(3)
        phi = rng.uniform(-1, 1)
        d = 0.3 * rng.standard_normal(3)
        lap = 0.3 * rng.standard_normal()
        feq, geq = oracle.site_equilibrium(P0, rho, j, phi, d, lap)
        mu, P = oracle.site_thermo(P0, phi, d, lap)
        u = j / rho
        assert abs(feq.sum() - rho) < 1e-14
        assert np.abs(feq @ c - j).max() < 1e-15
        M2 = np.einsum("i,ia,ib->ab", feq, c, c)
        assert np.abs(M2 - (rho / 3 * np.eye(3) + P + np.outer(j, j) / rho)).max() < 1e-14
        assert abs(geq.sum() - phi) < 1e-14
        assert np.abs(geq @ c - phi * u).max() < 1e-15
        G2 = np.einsum("i,ia,ib->ab", geq, c, c)
        assert np.abs(G2 - (P0["gamma"] * mu * np.eye(3) + phi * np.outer(u, u))).max() < 1e-14


def test_chemical_potential_is_free_energy_derivative():
    """mu equals dF/dphi of the discrete free energy (complex step)."""
    dims = (5, 4, 3)
    phi = L.uniform(11, 60, -0.8, 0.8)
    grad, lap = oracle.gradients(dims, phi)
    mu_bf = BF.chemical_potential(phi.reshape(3, 4, 5), P0["A"], P0["B"], P0["kappa"]).reshape(-1)
    mu = np.array([oracle.site_thermo(P0, phi[s], grad[:, s], lap[s])[0] for s in range(60)])
    assert np.abs(mu - mu_bf).max() < 1e-15


def _gibbs_duhem_residual(pressure_fn, prm):
    n = 48
    dims = (n, n, 1)
    x = np.arange(n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    phi = (0.6 * np.sin(2 * np.pi * X / n) + 0.4 * np.cos(4 * np.pi * Y / n)
           + 0.3 * np.sin(2 * np.pi * (X + Y) / n)).reshape(-1)
    grad, lap = oracle.gradients(dims, phi)
    mu = np.zeros(n * n)
    Pt = np.zeros((3, 3, n * n))
    for s in range(n * n):
        mu[s], p = oracle.site_thermo(prm, phi[s], grad[:, s], lap[s])
        Pt[:, :, s] = pressure_fn(p, phi[s], grad[:, s], lap[s])

    def d(fld, a):
        f3 = fld.reshape(n, n)
        ax = 1 if a == 0 else 0
        return ((np.roll(f3, -1, axis=ax) - np.roll(f3, 1, axis=ax)) / 2).reshape(-1)

    res = 0.0
    for a in range(2):
        rhs = phi * d(mu, a)
        res = max(res, np.abs(d(Pt[a, 0], 0) + d(Pt[a, 1], 1) - rhs).max() / np.abs(rhs).max())
    return res


def test_pressure_obeys_gibbs_duhem():
    """div P = phi grad mu holds to the O(k^2) error of the stencils.

    With A = B = 0 the gradient terms carry the whole identity, so a planted
    mistake in any of them (dropped or sign-flipped) is rejected."""
    assert _gibbs_duhem_residual(lambda p, *a: p, P0) < 0.03
    pg = dict(P0, A=0.0, B=0.0)
    assert _gibbs_duhem_residual(lambda p, *a: p, pg) < 0.05
    kap = P0["kappa"]
    dropped = lambda p, phi, d, lap: p + 0.5 * kap * (d @ d) * np.eye(3)
    flipped = lambda p, phi, d, lap: p + 2 * kap * phi * lap * np.eye(3)
    no_aniso = lambda p, phi, d, lap: p - kap * np.outer(d, d)
    for bad in (dropped, flipped, no_aniso):
        assert _gibbs_duhem_residual(bad, pg) > 0.3


# --------------------------------------------------------------- invariants

def test_uniform_state_is_fixed_point():
    dims = (6, 5, 4)
    n = 120
    phi0 = np.full(n, 0.37)
    u0 = np.tile(np.array([0.02, -0.01, 0.03])[:, None], (1, n))
    f, g = oracle.init(dims, P0, phi0, u0)
    f2, g2 = oracle.step(dims, P0, f, g, 10)
    # unchanged up to rounding (a few ulp per step)
    assert np.abs(f2 - f).max() < 1e-14 and np.abs(g2 - g).max() < 1e-14


def test_conservation_from_nonequilibrium_state():
    dims = (8, 6, 5)
    n = 240
    p = dict(P0, tau=0.8, tau_g=0.9)
    f, g = oracle.init(dims, p, L.spinodal_phi0(*dims, seed=3, amp=0.5))
    f = f * (1 + 0.05 * L.uniform(4, 19 * n, -1, 1).reshape(19, n))
    g = g + 0.01 * L.uniform(5, 19 * n, -1, 1).reshape(19, n)
    r0 = oracle.reduce(dims, f, g)
    f2, g2 = oracle.step(dims, p, f, g, 100)
    r1 = oracle.reduce(dims, f2, g2)
    assert abs(r1[0] - r0[0]) / r0[0] < 1e-13
    assert np.abs(r1[1:4] - r0[1:4]).max() / r0[0] < 1e-13
    assert abs(r1[4] - r0[4]) / np.abs(g).sum() < 1e-13


def test_one_dimensional_equivalence():
    """A field uniform in y and z evolves as the nx x 1 x 1 lattice."""
    nx = 12
    prof = L.spinodal_phi0(nx, 1, 1, seed=9, amp=0.3)
    u1 = np.zeros((3, nx))
    u1[1] = L.uniform(10, nx, -0.02, 0.02)
    d3 = (nx, 3, 4)
    f1, g1 = oracle.step((nx, 1, 1), P0, *oracle.init((nx, 1, 1), P0, prof, u1), 7)
    phi3 = np.tile(prof, 12)
    u3 = np.tile(u1, (1, 12))
    f3, g3 = oracle.step(d3, P0, *oracle.init(d3, P0, phi3, u3), 7)
    assert np.abs(f3.reshape(19, 12, nx) - f1[:, None, :]).max() < 1e-15
    assert np.abs(g3.reshape(19, 12, nx) - g1[:, None, :]).max() < 1e-15


# --------------------------------------------------------------- brute force

@pytest.mark.parametrize("dims", [(4, 4, 4), (3, 5, 2)])
def test_matches_definition_level_step(dims):
    n = int(np.prod(dims))
    p = dict(P0, tau=0.7, tau_g=0.85)
    c, _ = oracle.velocity_set()
    to_bf = BF.map_order(c, BF.VEL)           # oracle row k -> BF row to_bf[k]
    f, g = oracle.init(dims, p, L.spinodal_phi0(*dims, seed=21, amp=0.6),
                       0.03 * L.uniform(22, 3 * n, -1, 1).reshape(3, n))
    f = f * (1 + 0.1 * L.uniform(23, 19 * n, -1, 1).reshape(19, n))
    g = g + 0.02 * L.uniform(24, 19 * n, -1, 1).reshape(19, n)
    fo, go = oracle.step(dims, p, f, g, 3)
    fb_in = np.empty_like(f)
    gb_in = np.empty_like(g)
    fb_in[to_bf] = f
    gb_in[to_bf] = g
    fb, gb = BF.step(dims, p, fb_in, gb_in, 3)
    assert np.abs(fb[to_bf] - fo).max() < 1e-13
    assert np.abs(gb[to_bf] - go).max() < 1e-13


# --------------------------------------------------------------- hydrodynamics

@pytest.mark.parametrize("tau", [0.6, 0.8, 1.0])
def test_shear_wave_decay_rate(tau):
    """u_y = U sin(kx) decays at nu k^2 with nu = (tau - 1/2)/3."""
    p = dict(P0, tau=tau)
    n = 256
    dims = (n, 1, 1)
    k = 2 * math.pi / n
    x = np.arange(n)
    f, g = oracle.init(dims, p, np.zeros(n), L.shear_wave_u0(*dims, amp=0.01))
    ts, amps = [], []
    for t in range(0, 5001, 500):
        if t:
            f, g = oracle.step(dims, p, f, g, 500)
        _, u, phi = oracle.moments(dims, f, g)
        assert np.abs(phi).max() == 0.0
        ts.append(t)
        amps.append(2 / n * np.sum(u[1] * np.sin(k * x)))
    ts = np.array(ts)
    m = ts >= 500
    rate = -np.polyfit(ts[m], np.log(np.array(amps))[m], 1)[0]
    nu = (tau - 0.5) / 3
    assert abs(rate / (nu * k * k) - 1) < 1e-3


def test_galilean_advection_direction():
    """A phi mode in a uniform flow u_x = U moves by k U t in phase."""
    n, m, U, T = 64, 2, 0.05, 200
    dims = (n, 1, 1)
    k = 2 * math.pi * m / n
    u0 = np.zeros((3, n))
    u0[0] = U
    f, g = oracle.step(dims, P0, *oracle.init(dims, P0, L.cosine_mode_phi0(*dims, 0.01, m), u0), T)
    _, _, phi = oracle.moments(dims, f, g)
    shift = -np.angle(np.sum(phi * np.exp(-1j * k * np.arange(n))))
    assert abs(shift / (k * U * T) - 1) < 0.02


@pytest.mark.parametrize("m", [2, 4, 8])
def test_linear_spinodal_growth_rate(m):
    """eps cos(kx) grows at -M k^2 (A + kappa k^2), M = Gamma (tau_g - 1/2),
    with the lattice wavenumber k^2 -> 2 - 2 cos k."""
    n = 64
    dims = (n, 1, 1)
    k = 2 * math.pi * m / n
    kh2 = 2 - 2 * math.cos(k)
    M = P0["gamma"] * (P0["tau_g"] - 0.5)
    sigma = -M * kh2 * (P0["A"] + P0["kappa"] * kh2)
    f, g = oracle.init(dims, P0, L.cosine_mode_phi0(*dims, 1e-6, m))
    ts, amps = [], []
    for t in range(0, 1601, 200):
        if t:
            f, g = oracle.step(dims, P0, f, g, 200)
        _, _, phi = oracle.moments(dims, f, g)
        ts.append(t)
        amps.append(2 / n * np.sum(phi * np.cos(k * np.arange(n))))
    ts = np.array(ts)
    sel = ts >= 400
    rate = np.polyfit(ts[sel], np.log(np.array(amps))[sel], 1)[0]
    assert abs(rate / sigma - 1) < 0.05


def _newton_profile(phi0):
    A, B, kap = P0["A"], P0["B"], P0["kappa"]
    p = phi0.copy()
    n = len(p)
    for _ in range(40):
        r = A * p + B * p ** 3 - kap * (np.roll(p, 1) + np.roll(p, -1) - 2 * p)
        J = np.diag(A + 3 * B * p ** 2 + 2 * kap)
        for i in range(n):
            J[i, (i + 1) % n] -= kap
            J[i, (i - 1) % n] -= kap
        p = p - np.linalg.solve(J, r)
    return p


def test_flat_interface_relaxes_to_discrete_profile():
    """The LB steady state of two flat interfaces solves the discrete
    mu = 0 equation (found by Newton); the continuum tanh(x/xi) profile,
    xi = sqrt(-2 kappa/A), agrees only to the stencil's discretisation error."""
    n = 64
    dims = (n, 1, 1)
    xi = L.interface_width(P0["A"], P0["kappa"])
    phi0 = L.flat_interface_phi0(*dims, 1.0, xi)
    pn = _newton_profile(phi0)
    assert 0.005 < np.abs(pn - phi0).max() < 0.05
    f, g = oracle.init(dims, P0, phi0)
    devs = []
    for _ in range(10):
        f, g = oracle.step(dims, P0, f, g, 2000)
        _, u, phi = oracle.moments(dims, f, g)
        devs.append(np.abs(phi - pn).max())
    assert all(b < a for a, b in zip(devs, devs[1:]))
    assert devs[-1] < 3e-6
    assert np.abs(u).max() < 1e-9
