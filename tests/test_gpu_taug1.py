"""The tau_g = 1 reduced form (LB_KERNEL_TAUG1): g kept as (phi, mu, u).

With tau_g = 1 the oracle's g collision returns g_eq(phi, mu, u), so its
step depends on g only through phi = sum g: the reduced form must match the
oracle to the FP64 bound from any state, and its reconstructed g (streamed
equilibria) must equal the oracle's g after every step."""
import numpy as np
import pytest

import lb_inputs as L
import oracle
from tests.parity import P0, TOL_FP64, nonequilibrium_state, rel, to_abi, to_oracle, u_scale

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    import paper_1405_6162_gb300 as lbpkg
    lbpkg.build()
    oracle.build()


def _lat(dims, p, precision):
    from paper_1405_6162_gb300 import Lattice
    lat = Lattice.from_params(dims, p, precision=precision)
    lat.set_kernel("taug1")
    return lat


def _check(got, want, tol, f_oracle):
    for name, a, b in zip(("rho", "u", "phi"), got, want):
        e = rel(a, b, u_scale(f_oracle) if name == "u" else None)
        t = tol[name] if isinstance(tol, dict) else tol
        assert e <= t, (name, e)


@pytest.mark.parametrize("dims", [(32, 32, 32), (13, 7, 5), (1, 1, 9), (40, 9, 35), (2, 3, 2), (70, 37, 11)])
def test_reduced_form_matches_oracle_fp64(dims):
    p = dict(P0, tau=0.8)                          # tau_g = 1
    phi0 = L.spinodal_phi0(*dims, seed=300, amp=0.4)
    fo, go = oracle.step(dims, p, *oracle.init(dims, p, phi0), 10)
    with _lat(dims, p, "fp64") as lat:
        lat.init(phi0)
        lat.step(10)
        _check(lat.moments(), oracle.moments(dims, fo, go), TOL_FP64, fo)
        f, g = lat.get_state()
    assert rel(to_oracle(f), fo) <= TOL_FP64
    assert rel(to_oracle(g), go) <= TOL_FP64      # g rebuilt from the stored moments


def test_reduced_form_from_nonequilibrium_state():
    dims = (12, 10, 8)
    p = dict(P0, tau=0.7, kappa=0.06)
    f0, g0 = nonequilibrium_state(dims, p, seed=310)
    fo, go = oracle.step(dims, p, f0, g0, 5)
    with _lat(dims, p, "fp64") as lat:
        lat.set_state(to_abi(f0), to_abi(g0))
        lat.step(5)
        f, g = lat.get_state()
        _check(lat.moments(), oracle.moments(dims, fo, go), TOL_FP64, fo)
    assert rel(to_oracle(f), fo) <= TOL_FP64 and rel(to_oracle(g), go) <= TOL_FP64


def test_switching_forms_keeps_the_trajectory():
    """3 steps reduced, 3 general, 3 reduced again == 9 oracle steps."""
    dims = (16, 12, 10)
    phi0 = L.spinodal_phi0(*dims, seed=320, amp=0.3)
    fo, go = oracle.step(dims, P0, *oracle.init(dims, P0, phi0), 9)
    with _lat(dims, P0, "fp64") as lat:
        lat.init(phi0)
        lat.step(3)
        lat.set_kernel("two_pass")
        lat.step(3)
        lat.set_kernel("taug1")
        lat.step(3)
        f, g = lat.get_state()
    assert rel(to_oracle(f), fo) <= TOL_FP64 and rel(to_oracle(g), go) <= TOL_FP64


def test_init_state_and_totals():
    dims = (10, 9, 8)
    phi0 = L.spinodal_phi0(*dims, seed=330, amp=0.5)
    fo, go = oracle.init(dims, P0, phi0)
    with _lat(dims, P0, "fp64") as lat:
        lat.init(phi0)
        f, g = lat.get_state()                      # the equilibrium at each site
        r0 = lat.reduce()
        lat.step(50)
        r1 = lat.reduce()
    assert rel(to_oracle(f), fo) <= 1e-15 and rel(to_oracle(g), go) <= 1e-15
    assert np.abs(r1 - r0).max() <= 1e-13 * r0[0]


def test_rejected_unless_tau_g_is_one():
    from paper_1405_6162_gb300 import LBError, Lattice
    with Lattice.from_params((8, 8, 8), dict(P0, tau_g=0.9), precision="fp64") as lat:
        with pytest.raises(LBError):
            lat.set_kernel("taug1")


TOL_FP32_PER_STEP = {"rho": 2.5e-8, "u": 2.5e-8, "phi": 1e-7}


@pytest.mark.parametrize("dims", [(32, 32, 32), (13, 7, 5)])
def test_reduced_form_fp32_shifted(dims):
    phi0 = L.spinodal_phi0(*dims, seed=340, amp=0.3)
    fo, go = oracle.step(dims, P0, *oracle.init(dims, P0, phi0), 10)
    with _lat(dims, P0, "fp32_shifted") as lat:
        lat.init(phi0)
        lat.step(10)
        got = lat.moments()
    _check(got, oracle.moments(dims, fo, go), {k: v * 10 for k, v in TOL_FP32_PER_STEP.items()}, fo)


@pytest.mark.parametrize("precision", ["fp64", "fp32_shifted"])
def test_reduced_form_256cubed_flat_interface_equals_1d_oracle(precision):
    n = 256
    nsteps = 40
    xi = L.interface_width(P0["A"], P0["kappa"])
    line = L.flat_interface_phi0(n, 1, 1, 1.0, xi)
    d1 = (n, 1, 1)
    f1, g1 = oracle.step(d1, P0, *oracle.init(d1, P0, line), nsteps)
    want = oracle.moments(d1, f1, g1)
    with _lat((n, n, n), P0, precision) as lat:
        lat.init(np.ascontiguousarray(np.broadcast_to(line, (n * n, n))).reshape(-1))
        lat.step(nsteps)
        rho, u, phi = lat.moments()
    tol = TOL_FP64 if precision == "fp64" else None
    e_phi = rel(phi.reshape(-1, n), want[2][None, :])
    e_rho = rel(rho.reshape(-1, n), want[0][None, :])
    print(f"taug1 256^3 {precision}: rho {e_rho:.2e} phi {e_phi:.2e}")
    if precision == "fp64":
        assert e_phi <= tol and e_rho <= tol
    else:
        assert e_phi <= TOL_FP32_PER_STEP["phi"] * nsteps and e_rho <= TOL_FP32_PER_STEP["rho"] * nsteps


# phi-pass launch shapes (y rows per warp, warps per block, z run): one, two
# and four rows per lane (FP32: the even ones as paired FP32 arithmetic on row
# pairs), ragged y (an odd last row pair), several z runs with a ragged last
# one, and runs longer than nz
PHI_SHAPES = [(1, 4, 0), (2, 4, 0), (4, 8, 64), (2, 1, 3), (4, 2, 5), (2, 8, 7)]


@pytest.mark.parametrize("shape", PHI_SHAPES)
@pytest.mark.parametrize("dims", [(40, 9, 35), (70, 37, 11), (13, 7, 5)])
def test_phi_pass_shapes_fp64(dims, shape):
    p = dict(P0, tau=0.8)
    phi0 = L.spinodal_phi0(*dims, seed=350, amp=0.4)
    fo, go = oracle.step(dims, p, *oracle.init(dims, p, phi0), 6)
    from paper_1405_6162_gb300 import Lattice
    with Lattice.from_params(dims, p, precision="fp64") as lat:
        lat.set_kernel("taug1", *shape)
        lat.init(phi0)
        lat.step(6)
        _check(lat.moments(), oracle.moments(dims, fo, go), TOL_FP64, fo)
        f, g = lat.get_state()
    assert rel(to_oracle(g), go) <= TOL_FP64


@pytest.mark.parametrize("shape", PHI_SHAPES)
@pytest.mark.parametrize("dims", [(40, 9, 35), (70, 37, 11), (32, 32, 32),
                                  (64, 9, 35), (128, 7, 11), (192, 5, 6), (1024, 3, 4)])
def test_phi_pass_shapes_fp32_shifted(dims, shape):
    """FP32 at the per-step bounds of the default shape, and within a few
    FP32 roundings per step of the default shape's phi."""
    phi0 = L.spinodal_phi0(*dims, seed=360, amp=0.3)
    nsteps = 10
    fo, go = oracle.step(dims, P0, *oracle.init(dims, P0, phi0), nsteps)
    from paper_1405_6162_gb300 import Lattice
    out = []
    for s in ((0, 0, 0), shape):
        with Lattice.from_params(dims, P0, precision="fp32_shifted") as lat:
            lat.set_kernel("taug1", *s)
            lat.init(phi0)
            lat.step(nsteps)
            out.append(lat.moments())
    _check(out[1], oracle.moments(dims, fo, go), {k: v * nsteps for k, v in TOL_FP32_PER_STEP.items()}, fo)
    assert np.abs(out[1][2] - out[0][2]).max() <= 8 * nsteps * 2.0 ** -24 * np.abs(out[0][2]).max()


def test_phi_pass_shape_refusals():
    from paper_1405_6162_gb300 import LBError, Lattice
    with Lattice.from_params((16, 8, 8), P0, precision="fp64_df") as lat:
        with pytest.raises(LBError):
            lat.set_kernel("taug1", 4, 0, 0)      # four rows per lane spill in double-float
    with Lattice.from_params((16, 8, 8), P0, precision="fp32_shifted") as lat:
        for bad in ((3, 0, 0), (8, 0, 0), (0, 9, 0)):
            with pytest.raises(LBError):
                lat.set_kernel("taug1", *bad)
        lat.set_kernel("taug1", 4, 8, 100)     # a z run longer than nz is cut to nz
        lat.init(np.zeros(16 * 8 * 8))
        lat.step(2)
        lat.sync()


@pytest.mark.parametrize("dims", [(64, 6, 5), (128, 3, 7)])
def test_reduced_state_and_form_switches_fp32(dims):
    """FP32: the g rebuilt from the stored moments matches the oracle's g, and
    switching to the general form and back (which rebuilds g from them) keeps
    the trajectory."""
    phi0 = L.spinodal_phi0(*dims, seed=370, amp=0.3)
    fo, go = oracle.step(dims, P0, *oracle.init(dims, P0, phi0), 3)
    f9, g9 = oracle.step(dims, P0, *oracle.init(dims, P0, phi0), 9)
    tol_g = 3 * 4e-7
    with _lat(dims, P0, "fp32_shifted") as lat:
        lat.init(phi0)
        lat.step(3)
        f, g = lat.get_state()
        assert rel(to_oracle(g), go) <= tol_g
        lat.set_kernel("two_pass")
        lat.step(3)
        lat.set_kernel("taug1")
        lat.step(3)
        got = lat.moments()
    _check(got, oracle.moments(dims, f9, g9), {k: v * 9 for k, v in TOL_FP32_PER_STEP.items()}, f9)
