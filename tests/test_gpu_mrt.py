"""The multiple-relaxation-time collision and the Guo body force
(lb_set_collision, lb_set_force) against the oracle's orc_step_mrt, through
the C ABI.

FP64 must match the oracle to 1e-12 after 10 steps (five shapes, with and
without a force, 7- and 19-point stencils, from equilibrium and from
non-equilibrium states); FP32-shifted to the float bounds of the BGK step.
At 256^3, in the benchmark's launch: MRT with equal rates reproduces the BGK
kernel, and a forced run gains exactly N F per step of total momentum.
"""
import numpy as np
import pytest

import lb_inputs as L
import oracle
from tests.parity import P0, TOL_FP64, nonequilibrium_state, rel, to_abi, to_oracle, u_scale

pytestmark = pytest.mark.gpu

SHAPES = [(32, 32, 32), (13, 7, 5), (1, 1, 9), (40, 9, 35), (2, 3, 2)]
RATES = (1.3, 0.6)                      # tau_bulk, tau_ghost
FORCE = (1e-5, -2e-5, 3e-5)


@pytest.fixture(scope="module", autouse=True)
def _setup():
    import paper_1405_6162_gb300 as lbpkg
    lbpkg.build()
    oracle.build()


def _lat(dims, p, precision, rates=RATES, force=(0.0, 0.0, 0.0), npts=7, model="mrt"):
    from paper_1405_6162_gb300 import Lattice
    lat = Lattice.from_params(dims, p, precision=precision)
    lat.set_stencil(npts)
    lat.set_collision(model, *rates)
    lat.set_force(*force)
    return lat


def _oracle_moments(dims, f, g, force):
    rho, u, phi = oracle.moments(dims, f, g)
    return rho, u + np.asarray(force)[:, None] / (2 * rho[None, :]), phi


def _check(got, want, tol, f_oracle):
    for name, a, b in zip(("rho", "u", "phi"), got, want):
        e = rel(a, b, u_scale(f_oracle) if name == "u" else None)
        t = tol[name] if isinstance(tol, dict) else tol
        assert e <= t, (name, e)


@pytest.mark.parametrize("force", [(0.0, 0.0, 0.0), FORCE])
@pytest.mark.parametrize("dims", SHAPES)
def test_spinodal_fp64(dims, force):
    p = dict(P0, tau=0.8)
    phi0 = L.spinodal_phi0(*dims, seed=700, amp=0.4)
    fo, go = oracle.step_mrt(dims, p, *oracle.init(dims, p, phi0), 10, *RATES, force)
    with _lat(dims, p, "fp64", force=force) as lat:
        lat.init(phi0)
        lat.step(10)
        _check(lat.moments(), _oracle_moments(dims, fo, go, force), TOL_FP64, fo)
        f, g = lat.get_state()
    assert rel(to_oracle(f), fo) <= TOL_FP64 and rel(to_oracle(g), go) <= TOL_FP64


@pytest.mark.parametrize("npts", [7, 19])
def test_nonequilibrium_state_fp64(npts):
    dims = (12, 10, 8)
    p = dict(P0, tau=0.7, tau_g=0.85, kappa=0.06)
    f0, g0 = nonequilibrium_state(dims, p, seed=710)
    fo, go = oracle.step_mrt(dims, p, f0, g0, 5, 1.7, 0.55, FORCE, npts=npts)
    with _lat(dims, p, "fp64", (1.7, 0.55), FORCE, npts) as lat:
        lat.set_state(to_abi(f0), to_abi(g0))
        lat.step(5)
        f, g = lat.get_state()
    assert rel(to_oracle(f), fo) <= TOL_FP64 and rel(to_oracle(g), go) <= TOL_FP64


def test_bgk_with_force_is_mrt_with_equal_rates():
    dims = (16, 12, 10)
    p = dict(P0, tau=0.9)
    phi0 = L.spinodal_phi0(*dims, seed=720, amp=0.4)
    fo, go = oracle.step_mrt(dims, p, *oracle.init(dims, p, phi0), 10, 0.9, 0.9, FORCE)
    with _lat(dims, p, "fp64", force=FORCE, model="bgk") as lat:
        lat.init(phi0)
        lat.step(10)
        f, g = lat.get_state()
    assert rel(to_oracle(f), fo) <= TOL_FP64 and rel(to_oracle(g), go) <= TOL_FP64


@pytest.mark.parametrize("force", [(0.0, 0.0, 0.0), FORCE])
def test_spinodal_fp32_shifted(force):
    dims = (32, 32, 32)
    p = dict(P0, tau=0.8)
    phi0 = L.spinodal_phi0(*dims, seed=730)
    fo, go = oracle.step_mrt(dims, p, *oracle.init(dims, p, phi0), 10, *RATES, force)
    with _lat(dims, p, "fp32_shifted", force=force) as lat:
        lat.init(phi0)
        lat.step(10)
        _check(lat.moments(), _oracle_moments(dims, fo, go, force), {"rho": 1e-9, "u": 1e-7, "phi": 1e-5}, fo)


def test_validation():
    from paper_1405_6162_gb300 import LBError
    from paper_1405_6162_gb300 import _lib as LL
    dims = (8, 6, 5)
    with _lat(dims, P0, "fp64", model="bgk") as lat:
        for bad in ((0.5, 1.0), (1.0, 0.4), (float("nan"), 1.0)):
            with pytest.raises(LBError):
                lat.set_collision("mrt", *bad)
        with pytest.raises(LBError):
            lat.set_force(float("inf"), 0, 0)
        lat.set_kernel("fused")
        with pytest.raises(LBError):
            lat.set_collision("mrt", 1.0, 1.0)
        with pytest.raises(LBError):
            lat.set_force(1e-5, 0, 0)
        lat.set_kernel("auto")
        lat.set_collision("mrt", 1.2, 0.8)
        for k in ("fused", "staged", "slab", "lag", "taug1"):
            with pytest.raises(LBError):
                lat.set_kernel(k)
        lat.set_collision("bgk")
        lat.set_force(0, 1e-5, 0)
        with pytest.raises(LBError):
            lat.set_kernel("lag")
        lat.init(L.spinodal_phi0(*dims, seed=740))
        rc = LL.lib().lb_adjoint_init(lat.handle, None, None, None, None, None, None)
        assert rc == LL.LB_ERR_INVALID
        lat.set_force(0, 0, 0)
        lat.set_kernel("fused")


def test_equal_rates_reproduce_bgk_at_256cubed():
    dims = (256, 256, 256)
    p = dict(P0, tau=0.8)
    phi0 = L.spinodal_phi0(*dims, seed=1)
    out = {}
    for model in ("bgk", "mrt"):
        with _lat(dims, p, "fp32_shifted", (0.8, 0.8), model=model) as lat:
            lat.init(phi0)
            lat.step(5)
            out[model] = lat.moments()
    for a, b in zip(out["mrt"], out["bgk"]):
        assert rel(a, b) < 1e-6


def test_forced_momentum_gain_at_256cubed():
    dims = (256, 256, 256)
    n = 256 ** 3
    p = dict(P0, tau=0.8)
    with _lat(dims, p, "fp32_shifted", force=FORCE) as lat:
        lat.init(L.spinodal_phi0(*dims, seed=1))
        r0 = lat.reduce()
        lat.step(5)
        r1 = lat.reduce()
    gain = np.asarray(r1[1:4]) - np.asarray(r0[1:4])
    want = 5 * n * np.asarray(FORCE)
    assert np.abs(gain - want).max() < 1e-5 * np.abs(want).max()
    assert abs(r1[0] - r0[0]) < 1e-6 * r0[0]
