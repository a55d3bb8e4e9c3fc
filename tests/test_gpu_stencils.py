"""The isotropic 19- and 27-point phi stencils (lb_set_stencil) against the
oracle's orc_*_n entry points, through the C ABI.

FP64 must match the oracle to 1e-12 after 10 steps from a spinodal start and
from a non-equilibrium state, on the default two-pass step and on the
tau_g = 1 reduced form; FP32-shifted to the per-step float bounds used for
the 7-point step.  At 256^3 (the benchmark's lattice and launch) a field
that varies along x only must evolve exactly as under the 7-point stencil.
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


def _lat(dims, p, precision, npts, kernel="auto"):
    from paper_1405_6162_gb300 import Lattice
    lat = Lattice.from_params(dims, p, precision=precision)
    lat.set_kernel(kernel)
    lat.set_stencil(npts)
    return lat


def _check(got, want, tol, f_oracle):
    for name, a, b in zip(("rho", "u", "phi"), got, want):
        e = rel(a, b, u_scale(f_oracle) if name == "u" else None)
        t = tol[name] if isinstance(tol, dict) else tol
        assert e <= t, (name, e)


@pytest.mark.parametrize("npts", [19, 27])
@pytest.mark.parametrize("dims", SHAPES)
def test_spinodal_fp64(npts, dims):
    phi0 = L.spinodal_phi0(*dims, seed=500, amp=0.4)
    fo, go = oracle.step(dims, P0, *oracle.init(dims, P0, phi0, npts=npts), 10, npts=npts)
    with _lat(dims, P0, "fp64", npts) as lat:
        lat.init(phi0)
        lat.step(10)
        _check(lat.moments(), oracle.moments(dims, fo, go), TOL_FP64, fo)
        f, g = lat.get_state()
    assert rel(to_oracle(f), fo) <= TOL_FP64 and rel(to_oracle(g), go) <= TOL_FP64


@pytest.mark.parametrize("npts", [19, 27])
def test_init_matches_oracle(npts):
    dims = (10, 9, 8)
    n = 720
    phi0 = L.spinodal_phi0(*dims, seed=501, amp=0.5)
    u0 = 0.02 * L.uniform(502, 3 * n, -1, 1).reshape(3, n)
    fo, go = oracle.init(dims, P0, phi0, u0, npts=npts)
    with _lat(dims, P0, "fp64", npts) as lat:
        lat.init(phi0, u0)
        f, g = lat.get_state()
    assert rel(to_oracle(f), fo) <= 1e-15 and rel(to_oracle(g), go) <= 1e-15


@pytest.mark.parametrize("npts", [19, 27])
def test_nonequilibrium_state_fp64(npts):
    dims = (12, 10, 8)
    p = dict(P0, tau=0.7, tau_g=0.85, kappa=0.06)
    f0, g0 = nonequilibrium_state(dims, p, seed=510)
    fo, go = oracle.step(dims, p, f0, g0, 5, npts=npts)
    with _lat(dims, p, "fp64", npts) as lat:
        lat.set_state(to_abi(f0), to_abi(g0))
        lat.step(5)
        f, g = lat.get_state()
    assert rel(to_oracle(f), fo) <= TOL_FP64 and rel(to_oracle(g), go) <= TOL_FP64


@pytest.mark.parametrize("npts", [19, 27])
@pytest.mark.parametrize("dims", [(32, 32, 32), (13, 7, 5), (40, 9, 35)])
def test_reduced_form_fp64(npts, dims):
    phi0 = L.spinodal_phi0(*dims, seed=520, amp=0.4)
    fo, go = oracle.step(dims, P0, *oracle.init(dims, P0, phi0, npts=npts), 10, npts=npts)
    with _lat(dims, P0, "fp64", npts, kernel="taug1") as lat:
        lat.init(phi0)
        lat.step(10)
        _check(lat.moments(), oracle.moments(dims, fo, go), TOL_FP64, fo)
        f, g = lat.get_state()
    assert rel(to_oracle(f), fo) <= TOL_FP64 and rel(to_oracle(g), go) <= TOL_FP64


@pytest.mark.parametrize("kernel", ["auto", "taug1"])
@pytest.mark.parametrize("npts", [19, 27])
def test_spinodal_fp32_shifted(npts, kernel):
    dims = (32, 32, 32)
    phi0 = L.spinodal_phi0(*dims, seed=530)
    fo, go = oracle.step(dims, P0, *oracle.init(dims, P0, phi0, npts=npts), 10, npts=npts)
    with _lat(dims, P0, "fp32_shifted", npts, kernel) as lat:
        lat.init(phi0)
        lat.step(10)
        _check(lat.moments(), oracle.moments(dims, fo, go), {"rho": 1e-9, "u": 1e-7, "phi": 1e-5}, fo)


def test_choice_matters_and_is_validated():
    from paper_1405_6162_gb300 import LBError
    dims = (12, 10, 8)
    phi0 = L.spinodal_phi0(*dims, seed=540, amp=0.5)
    out = {}
    for npts in (7, 19, 27):
        with _lat(dims, P0, "fp64", npts) as lat:
            lat.init(phi0)
            lat.step(3)
            out[npts] = lat.moments()[2]
    assert rel(out[19], out[7]) > 1e-6 and rel(out[27], out[19]) > 1e-7
    with _lat(dims, P0, "fp64", 7) as lat:
        for bad in (0, 9, 26):
            with pytest.raises(LBError):
                lat.set_stencil(bad)
        lat.set_kernel("fused")
        with pytest.raises(LBError):
            lat.set_stencil(19)
        lat.set_kernel("two_pass")
        lat.set_stencil(27)
        for k in ("fused", "staged", "slab", "lag"):
            with pytest.raises(LBError):
                lat.set_kernel(k)
        lat.set_stencil(7)
        lat.set_kernel("fused")


def test_adjoint_refuses_isotropic_stencils():
    import torch
    from paper_1405_6162_gb300 import _lib as LL
    dims = (6, 5, 4)
    n = 120
    with _lat(dims, P0, "fp64", 19) as lat:
        lat.init(L.spinodal_phi0(*dims, seed=541))
        z = torch.zeros(19 * n, dtype=torch.float64, device="cuda")
        o = [torch.zeros_like(z) for _ in range(2)]
        dk = torch.zeros(1, dtype=torch.float64, device="cuda")
        rc = LL.lib().lb_adjoint_step(lat.handle, z.data_ptr(), z.data_ptr(), z.data_ptr(), z.data_ptr(),
                                      o[0].data_ptr(), o[1].data_ptr(), dk.data_ptr())
        assert rc == LL.LB_ERR_INVALID


@pytest.mark.parametrize("kernel", ["auto", "taug1"])
@pytest.mark.parametrize("npts", [19, 27])
def test_one_axis_field_at_256cubed(npts, kernel):
    """Full-size lattice, benchmark launch: a flat interface (phi varies along
    x only) evolves as under the 7-point stencil, and the totals are kept."""
    dims = (256, 256, 256)
    xi = L.interface_width(P0["A"], P0["kappa"])
    phi0 = L.flat_interface_phi0(*dims, amplitude=0.5, xi=xi)
    res = {}
    for k in (7, npts):
        with _lat(dims, P0, "fp32_shifted", k, kernel) as lat:
            lat.init(phi0)
            r0 = lat.reduce()
            lat.step(5)
            r1 = lat.reduce()
            res[k] = lat.moments()[2]
        assert abs(r1[0] - r0[0]) / r0[0] < 1e-6
        assert abs(r1[4] - r0[4]) < 1e-6 * np.abs(phi0).sum()
    assert rel(res[npts], res[7]) < 1e-6
