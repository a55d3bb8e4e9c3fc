"""The double-float precision (LB_FP64_DF: each value an unevaluated sum of
two floats, arithmetic on the FP32 units) against the FP64 oracle.

Its unit roundoff is ~2^-48 (3.6e-15) instead of 2^-53, so it is held to the
same 1e-12 bound as FP64 after 10 steps (spinodal starts on five shapes,
non-equilibrium states, the 19-point stencil and the MRT collision), and to
1e-11 after 1000 spinodal steps, where the instability amplifies rounding
about a thousandfold.
"""
import numpy as np
import pytest

import lb_inputs as L
import oracle
from tests.parity import P0, TOL_FP64, nonequilibrium_state, rel, to_abi, to_oracle, u_scale

pytestmark = pytest.mark.gpu

SHAPES = [(32, 32, 32), (13, 7, 5), (1, 1, 9), (40, 9, 35), (2, 3, 2)]


@pytest.fixture(scope="module", autouse=True)
def _setup():
    import paper_1405_6162_gb300 as lbpkg
    lbpkg.build()
    oracle.build()


def _lat(dims, p=P0):
    from paper_1405_6162_gb300 import Lattice
    return Lattice.from_params(dims, p, precision="fp64_df")


def _check(got, want, tol, f_oracle):
    for name, a, b in zip(("rho", "u", "phi"), got, want):
        e = rel(a, b, u_scale(f_oracle) if name == "u" else None)
        assert e <= tol, (name, e)


@pytest.mark.parametrize("dims", SHAPES)
def test_spinodal_matches_oracle(dims):
    phi0 = L.spinodal_phi0(*dims, seed=1000, amp=0.4)
    fo, go = oracle.step(dims, P0, *oracle.init(dims, P0, phi0), 10)
    with _lat(dims) as lat:
        lat.init(phi0)
        lat.step(10)
        _check(lat.moments(), oracle.moments(dims, fo, go), TOL_FP64, fo)
        f, g = lat.get_state()
    assert rel(to_oracle(f), fo) <= TOL_FP64 and rel(to_oracle(g), go) <= TOL_FP64


def test_nonequilibrium_state_matches_oracle():
    dims = (12, 10, 8)
    p = dict(P0, tau=0.7, tau_g=0.85, kappa=0.06)
    f0, g0 = nonequilibrium_state(dims, p, seed=1010)
    fo, go = oracle.step(dims, p, f0, g0, 5)
    with _lat(dims, p) as lat:
        lat.set_state(to_abi(f0), to_abi(g0))
        f, g = lat.get_state()
        # the state round trip keeps ~48 bits
        assert rel(to_oracle(f), f0) <= 1e-14 and rel(to_oracle(g), g0) <= 1e-14
        lat.step(5)
        f, g = lat.get_state()
    assert rel(to_oracle(f), fo) <= TOL_FP64 and rel(to_oracle(g), go) <= TOL_FP64


def test_stencil_and_mrt_match_oracle():
    dims = (16, 12, 10)
    p = dict(P0, tau=0.8)
    phi0 = L.spinodal_phi0(*dims, seed=1020, amp=0.4)
    fo, go = oracle.step_mrt(dims, p, *oracle.init(dims, p, phi0, npts=19), 10, 1.3, 0.6, (1e-5, 0, -2e-5),
                             npts=19)
    with _lat(dims, p) as lat:
        lat.set_stencil(19)
        lat.set_collision("mrt", 1.3, 0.6)
        lat.set_force(1e-5, 0, -2e-5)
        lat.init(phi0)
        lat.step(10)
        f, g = lat.get_state()
    assert rel(to_oracle(f), fo) <= TOL_FP64 and rel(to_oracle(g), go) <= TOL_FP64


@pytest.mark.parametrize("kernel", ["auto", "taug1"])
def test_spinodal_64cubed_1000_steps(kernel):
    dims = (64, 64, 64)
    phi0 = L.spinodal_phi0(*dims, seed=1)
    fo, go = oracle.step(dims, P0, *oracle.init(dims, P0, phi0), 1000, kind="omp")
    want = oracle.moments(dims, fo, go)
    with _lat(dims) as lat:
        lat.set_kernel(kernel)
        lat.init(phi0)
        lat.step(1000)
        got = lat.moments()
    errs = {k: rel(a, b, u_scale(fo) if k == "u" else None) for k, a, b in zip(("rho", "u", "phi"), got, want)}
    print(f"spinodal 64^3 x 1000 fp64_df {kernel}:", errs)
    for k, e in errs.items():
        assert e <= 1e-11, (k, e)


@pytest.mark.parametrize("dims", [(32, 32, 32), (13, 7, 5), (70, 37, 11), (1, 1, 9)])
def test_reduced_form_matches_oracle(dims):
    phi0 = L.spinodal_phi0(*dims, seed=1030, amp=0.4)
    fo, go = oracle.step(dims, P0, *oracle.init(dims, P0, phi0), 10)
    with _lat(dims) as lat:
        lat.set_kernel("taug1")
        lat.init(phi0)
        lat.step(10)
        _check(lat.moments(), oracle.moments(dims, fo, go), TOL_FP64, fo)
        f, g = lat.get_state()
    assert rel(to_oracle(f), fo) <= TOL_FP64 and rel(to_oracle(g), go) <= TOL_FP64


def test_limits():
    from paper_1405_6162_gb300 import Batch, LBError
    dims = (8, 6, 5)
    with _lat(dims) as lat:
        for k in ("fused", "staged", "slab", "lag"):
            with pytest.raises(LBError):
                lat.set_kernel(k)
        lat.set_kernel("taug1")
        lat.set_kernel("two_pass")
    with pytest.raises(LBError):
        Batch([dict(P0, nx=8, ny=6, nz=5)], precision="fp64_df")
