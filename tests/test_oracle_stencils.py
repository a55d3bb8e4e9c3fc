"""Pins of the oracle's isotropic 19- and 27-point stencils (no GPU).

The paper (Sec. II.A) advances the order parameter with "standard
finite-difference techniques"; the 19- and 27-point variants are read as the
lattice-weighted differences over the D3Q19 / D3Q27 neighbourhoods.  The
tests check the oracle against facts that do not come from it: the Fourier
symbols of the stencils, written here in closed product form (not as the
weighted sums the oracle evaluates), the isotropy of their leading error, and
the reduction to the 7-point stencils on fields that vary along one axis.
"""
import math

import numpy as np
import pytest

import lb_inputs as L
import oracle

P0 = dict(L.DEFAULT_PARAMS)


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _symbols(npts, k):
    """(lambda_a, Lambda): d_a cos(k.x) = -lambda_a sin(k.x) and
    lap cos(k.x) = Lambda cos(k.x), in closed form."""
    C = [math.cos(a) for a in k]
    S = [math.sin(a) for a in k]
    if npts == 7:
        return [S[0], S[1], S[2]], 2 * sum(C) - 6
    if npts == 19:
        lam = [S[a] * (1 + C[(a + 1) % 3] + C[(a + 2) % 3]) / 3 for a in range(3)]
        return lam, 2 / 3 * (C[0] + C[1] + C[2] + C[0] * C[1] + C[0] * C[2] + C[1] * C[2]) - 4
    # D3Q27 weights factorise: W(c) = V(c_x) V(c_y) V(c_z), V(0) = 2/3, V(+-1) = 1/6
    lam = [S[a] * (2 + C[(a + 1) % 3]) * (2 + C[(a + 2) % 3]) / 9 for a in range(3)]
    return lam, 6 * ((2 + C[0]) * (2 + C[1]) * (2 + C[2]) / 27 - 1)


def _mode(dims, m, phase=0.3):
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    k = [2 * math.pi * m[a] / dims[a] for a in range(3)]
    th = (k[0] * x + k[1] * y + k[2] * z).reshape(-1) + phase
    return k, th


@pytest.mark.parametrize("npts", [7, 19, 27])
@pytest.mark.parametrize("m", [(1, 0, 0), (2, 3, 1), (0, 1, 4), (3, 5, 2)])
def test_fourier_symbols(npts, m):
    dims = (8, 12, 10)
    k, th = _mode(dims, m)
    grad, lap = oracle.gradients(dims, np.cos(th), npts=npts)
    lam, Lam = _symbols(npts, k)
    assert np.abs(lap - Lam * np.cos(th)).max() < 1e-13
    for a in range(3):
        assert np.abs(grad[a] + lam[a] * np.sin(th)).max() < 1e-13


@pytest.mark.parametrize("npts", [19, 27])
def test_consistent_to_second_order(npts):
    """Symbols approach -k^2 and k_a with O(k^2) relative error."""
    for h in (1e-2, 5e-3):
        k = [h * 0.3, h * -0.8, h * 0.5]
        k2 = sum(a * a for a in k)
        lam, Lam = _symbols(npts, k)
        assert abs(Lam + k2) < 0.2 * k2 * k2
        for a in range(3):
            assert abs(lam[a] - k[a]) < 0.5 * abs(k[a]) * k2 + 1e-18


def test_isotropy_of_leading_error():
    """Two lattice modes of equal |k| in different directions, (3,0,0) and
    (1,2,2): the isotropic stencils give the same Laplacian and gradient
    magnitude to O(k^6); the 7-point stencil differs at O(k^4)."""
    dims = (48, 48, 48)
    diff = {}
    for npts in (7, 19, 27):
        vals = []
        for m in ((3, 0, 0), (1, 2, 2)):
            k, th = _mode(dims, m, phase=0.0)
            grad, lap = oracle.gradients(dims, np.cos(th), npts=npts)
            s = 0                                # site 0: cos = 1, sin = 0
            Lam = lap[s]
            # gradient magnitude from a quarter-period-shifted mode
            _, th2 = _mode(dims, m, phase=-math.pi / 2)
            g2, _ = oracle.gradients(dims, np.cos(th2), npts=npts)
            vals.append((Lam, math.sqrt(sum(g2[a][s] ** 2 for a in range(3)))))
        diff[npts] = (abs(vals[0][0] - vals[1][0]), abs(vals[0][1] - vals[1][1]))
    assert diff[7][0] > 5e-4 and diff[7][1] > 1e-3
    for npts in (19, 27):
        assert diff[npts][0] < 0.05 * diff[7][0]
        assert diff[npts][1] < 0.05 * diff[7][1]


@pytest.mark.parametrize("npts", [19, 27])
def test_one_axis_field_matches_seven_point(npts):
    """For phi(x) alone every stencil reduces to the 1-D central differences."""
    dims = (11, 4, 3)
    prof = L.spinodal_phi0(11, 1, 1, seed=41, amp=0.8)
    phi = np.tile(prof, 12)
    g7, l7 = oracle.gradients(dims, phi, npts=7)
    gn, ln = oracle.gradients(dims, phi, npts=npts)
    assert np.abs(gn - g7).max() < 1e-15 and np.abs(ln - l7).max() < 1e-15
    # and so do whole steps of the model
    u = np.zeros((3, 132))
    u[1] = np.tile(L.uniform(42, 11, -0.02, 0.02), 12)
    f7, g7s = oracle.step(dims, P0, *oracle.init(dims, P0, phi, u), 5)
    fn, gns = oracle.step(dims, P0, *oracle.init(dims, P0, phi, u, npts=npts), 5, npts=npts)
    assert np.abs(fn - f7).max() < 1e-14 and np.abs(gns - g7s).max() < 1e-14


@pytest.mark.parametrize("npts", [19, 27])
def test_conservation_and_fixed_point(npts):
    dims = (8, 6, 5)
    n = 240
    p = dict(P0, tau=0.8, tau_g=0.9)
    f, g = oracle.init(dims, p, L.spinodal_phi0(*dims, seed=43, amp=0.5), npts=npts)
    f = f * (1 + 0.05 * L.uniform(44, 19 * n, -1, 1).reshape(19, n))
    g = g + 0.01 * L.uniform(45, 19 * n, -1, 1).reshape(19, n)
    r0 = oracle.reduce(dims, f, g)
    f2, g2 = oracle.step(dims, p, f, g, 50, npts=npts)
    r1 = oracle.reduce(dims, f2, g2)
    assert abs(r1[0] - r0[0]) / r0[0] < 1e-13
    assert np.abs(r1[1:4] - r0[1:4]).max() / r0[0] < 1e-13
    assert abs(r1[4] - r0[4]) / np.abs(g).sum() < 1e-13
    # a uniform moving state does not change
    u0 = np.tile(np.array([0.02, -0.01, 0.03])[:, None], (1, n))
    f, g = oracle.init(dims, P0, np.full(n, -0.4), u0, npts=npts)
    f2, g2 = oracle.step(dims, P0, f, g, 10, npts=npts)
    assert np.abs(f2 - f).max() < 1e-14 and np.abs(g2 - g).max() < 1e-14


def test_stencils_differ_on_a_three_dimensional_field():
    """The choice matters away from one-axis fields (guards against a silently
    ignored argument)."""
    dims = (6, 5, 4)
    phi = L.spinodal_phi0(*dims, seed=46, amp=0.5)
    out = {k: oracle.gradients(dims, phi, npts=k)[1] for k in (7, 19, 27)}
    assert np.abs(out[19] - out[7]).max() > 1e-3
    assert np.abs(out[27] - out[19]).max() > 1e-4
    with pytest.raises(ValueError):
        oracle.gradients(dims, phi, npts=9)
