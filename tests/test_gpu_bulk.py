"""The bulk-copy single-pass kernel (LB_KERNEL_BULK) against the oracle.

One CTA per x-row marching z; g rows staged in shared memory by bulk
asynchronous copies; phi rows shared along y inside a thread-block cluster,
the cluster's outer halo rows formed by a halo warp.  Shapes cover several
z chunks with a ragged last chunk, clusters of 1, 2, 4 and 8 CTAs (every
CTA of a cluster of 1 forms both halo rows itself), degenerate extents
(ny = 1, nz = 1 and 2: the rows and planes wrap onto themselves) and rows of
4 up to 256 sites.
"""
import numpy as np
import pytest

import lb_inputs as L
import oracle
from tests.parity import P0, TOL_FP64, gpu_lattice, nonequilibrium_state, rel, to_abi, to_oracle, u_scale

pytestmark = pytest.mark.gpu

# (dims, (g slots, CTAs per cluster, planes per CTA))
CASES = [((8, 8, 5), (0, 0, 0)),
         ((12, 8, 9), (3, 1, 1)),
         ((12, 8, 9), (3, 2, 4)),
         ((32, 16, 35), (4, 8, 8)),
         ((40, 9, 11), (3, 1, 5)),
         ((4, 1, 3), (3, 1, 2)),
         ((20, 12, 2), (4, 4, 1)),
         ((16, 8, 1), (3, 2, 7)),
         ((256, 4, 3), (3, 4, 2)),
         ((24, 6, 13), (5, 2, 32))]


@pytest.fixture(scope="module", autouse=True)
def _setup():
    import paper_1405_6162_gb300 as lbpkg
    lbpkg.build()
    oracle.build()


@pytest.mark.parametrize("dims,shape", CASES)
def test_bulk_fp64_matches_oracle(dims, shape):
    p = dict(P0, tau=0.7, tau_g=0.9, kappa=0.06)
    f0, g0 = nonequilibrium_state(dims, p, seed=131)
    fo, go = oracle.step(dims, p, f0, g0, 4)
    mo = oracle.moments(dims, fo, go)
    with gpu_lattice(dims, p, "fp64", "bulk", shape) as lat:
        lat.set_state(to_abi(f0), to_abi(g0))
        lat.step(4)
        lat.sync()
        rho, u, phi = lat.moments()
        f, g = lat.get_state()
    assert rel(to_oracle(f), fo) <= TOL_FP64
    assert rel(to_oracle(g), go) <= TOL_FP64
    assert rel(rho, mo[0]) <= TOL_FP64 and rel(phi, mo[2]) <= TOL_FP64
    assert rel(u, mo[1], u_scale(fo)) <= TOL_FP64 and rel(u, mo[1]) <= TOL_FP64


@pytest.mark.parametrize("dims,shape", [((32, 32, 32), (0, 0, 0)), ((32, 32, 32), (4, 8, 7)),
                                        ((64, 16, 24), (3, 1, 16)), ((32, 32, 32), (2, 2, 5)),
                                        ((256, 8, 9), (2, 4, 4)), ((40, 9, 11), (2, 1, 3))])
def test_bulk_spinodal_fp32_shifted(dims, shape):
    """10 spinodal steps in FP32-shifted storage against the FP64 oracle, at
    the bounds of the other kernels' FP32 tests."""
    phi0 = L.spinodal_phi0(*dims, seed=0)
    fo, go = oracle.step(dims, P0, *oracle.init(dims, P0, phi0), 10)
    mo = oracle.moments(dims, fo, go)
    with gpu_lattice(dims, P0, "fp32_shifted", "bulk", shape) as lat:
        lat.init(phi0)
        lat.step(10)
        got = lat.moments()
    tol = {"rho": 1e-9, "u": 1e-7, "phi": 1e-5}
    for name, a, b in zip(("rho", "u", "phi"), got, mo):
        e = rel(a, b, u_scale(fo) if name == "u" else None)
        assert e <= tol[name], (name, e)


@pytest.mark.parametrize("precision", ["fp64", "fp32_shifted"])
def test_bulk_equals_two_pass(precision):
    """The same per-site arithmetic as the default two-pass step, phi summed
    in the same order everywhere (own rows, pushed rows, halo-warp rows): the
    states agree to a few ulps after 6 steps, and are usually identical."""
    dims = (48, 20, 17)
    p = dict(P0, tau=0.8)
    f0, g0 = nonequilibrium_state(dims, p, seed=141)
    out = []
    blocks = [("two_pass", (0, 0, 0)), ("bulk", (3, 4, 6)), ("bulk", (4, 2, 5)), ("bulk", (3, 1, 17))]
    if precision == "fp32_shifted":
        blocks += [("bulk", (2, 2, 7)), ("bulk", (2, 1, 4))]     # the lean form
    for kernel, block in blocks:
        with gpu_lattice(dims, p, precision, kernel, block) as lat:
            lat.set_state(to_abi(f0), to_abi(g0))
            lat.step(6)
            out.append(lat.get_state())
    ulp = 2.0 ** -52 if precision == "fp64" else 2.0 ** -23
    for f, g in out[1:]:
        assert np.abs(f - out[0][0]).max() <= 16 * ulp * np.abs(out[0][0]).max()
        assert np.abs(g - out[0][1]).max() <= 16 * ulp * np.abs(out[0][1]).max()


def test_bulk_y_uniform_field_stays_y_uniform():
    """A field uniform in y and z gives every row the same phi however it was
    formed (own row, pushed by a peer, or by the halo warp), so it stays
    exactly uniform in y and z (no spurious y gradient at cluster edges)."""
    n = 64
    dims = (n, 16, 8)
    xi = L.interface_width(P0["A"], P0["kappa"])
    line = L.flat_interface_phi0(n, 1, 1, 1.0, xi)
    phi0 = np.ascontiguousarray(np.broadcast_to(line, (16 * 8, n))).reshape(-1)
    for precision in ("fp32_shifted", "fp64"):
        with gpu_lattice(dims, P0, precision, "bulk", (4, 4, 3)) as lat:
            lat.init(phi0)
            lat.step(20)
            rho, u, phi = lat.moments()
        assert np.abs(u[1:]).max() <= 1e-15
        ph = phi.reshape(-1, n)
        assert np.array_equal(ph, np.broadcast_to(ph[0], ph.shape))


def test_bulk_refuses_shapes_it_cannot_take():
    from paper_1405_6162_gb300 import LBError
    for dims, shape, prec in (((13, 8, 4), (0, 0, 0), "fp32_shifted"),    # 52-byte rows
                              ((6, 8, 4), (0, 0, 0), "fp32_shifted"),     # 24-byte rows
                              ((260, 4, 4), (0, 0, 0), "fp32_shifted"),   # rows longer than 256
                              ((16, 6, 4), (0, 4, 0), "fp32_shifted"),    # 4 does not divide ny = 6
                              ((16, 8, 4), (0, 3, 0), "fp32_shifted"),    # cluster of 3
                              ((16, 8, 4), (1, 0, 0), "fp32_shifted"),    # one slot
                              ((16, 8, 4), (2, 0, 0), "fp64"),            # the lean form is FP32 only
                              ((16, 8, 4), (0, 0, 0), "fp64_df")):
        with gpu_lattice(dims, P0, prec) as lat:
            with pytest.raises(LBError):
                lat.set_kernel("bulk", *shape)
    with gpu_lattice((16, 8, 4), P0, "fp64") as lat:
        lat.set_kernel("bulk")
        with pytest.raises(LBError):
            lat.set_stencil(19)
        with pytest.raises(LBError):
            lat.set_collision("mrt", 1.2, 0.8)


@pytest.mark.parametrize("shape", [(3, 4, 4), (4, 1, 3), (2, 2, 5)])
def test_bulk_wait_timeout_is_reported_and_recoverable(shape):
    """With the test hook every CTA's copy producer stops after its first
    plane: the consumers' bounded waits give up, the kernel returns, the host
    sees LB_ERR_TIMEOUT, and after re-initialisation the context is exact
    again."""
    from paper_1405_6162_gb300 import LBError
    from paper_1405_6162_gb300 import _lib as LL
    dims = (32, 8, 12)
    phi0 = L.spinodal_phi0(*dims, seed=12, amp=0.3)
    fo, go = oracle.step(dims, P0, *oracle.init(dims, P0, phi0), 3)
    mo = oracle.moments(dims, fo, go)
    with gpu_lattice(dims, P0, "fp64" if shape[0] > 2 else "fp32_shifted", "bulk", shape) as lat:
        lat.set_wait_timeout(0.05)
        LL.check(LL.lib().lb_debug_wait_skew(lat.handle, 1), "hook")
        lat.init(phi0)
        lat.step(2)
        with pytest.raises(LBError) as ei:
            lat.sync()
        assert ei.value.code == LL.LB_ERR_TIMEOUT
        lat.sync()
        LL.check(LL.lib().lb_debug_wait_skew(lat.handle, 0), "hook")
        lat.init(phi0)
        lat.step(3)
        lat.sync()
        got = lat.moments()
    # FP64, or the lean form's FP32 at the per-step bounds of the other FP32 tests
    tol = TOL_FP64 if shape[0] > 2 else {"rho": 1e-7, "u": 1e-7, "phi": 1e-6}
    for name, a, b in zip(("rho", "u", "phi"), got, mo):
        t = tol[name] if isinstance(tol, dict) else tol
        assert rel(a, b, u_scale(fo) if name == "u" else None) <= t, name
