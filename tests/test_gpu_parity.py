"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

FP64: every field within 1e-12 of the oracle (max-norm scaled) after N
steps.  FP32-shifted: float storage and arithmetic of f_i - w_i rho0 and g_i;
its tolerance is stated per test from the arithmetic (float rounding of
O(1e-2) distribution values, accumulated over the steps run).
"""
import numpy as np
import pytest

import lb_inputs as L
import oracle
from tests.parity import (P0, TOL_FP64, gpu_lattice, nonequilibrium_state, rel, to_abi,
                          to_oracle, u_scale)

pytestmark = pytest.mark.gpu

# every kernel, default and ragged-forcing launch shapes (valid in FP64 too)
KERNEL_CASES = [("two_pass", (0, 0, 0)), ("fused", (0, 0, 0)), ("fused", (64, 2, 5)),
                ("fused", (32, 1, 1)), ("fused", (128, 2, 7)), ("staged", (0, 0, 0)),
                ("staged", (64, 2, 5)), ("staged", (32, 1, 1)), ("staged", (32, 4, 3)),
                ("slab", (0, 0, 0)), ("slab", (64, 2, 5)), ("slab", (32, 1, 1)), ("slab", (128, 2, 3)),
                ("lag", (0, 0, 0)), ("lag", (256, 1, 1)),
                ("bulk", (0, 0, 0)), ("bulk", (4, 8, 7)), ("bulk", (3, 1, 32))]


@pytest.fixture(scope="module", autouse=True)
def _setup():
    import paper_1405_6162_gb300 as lbpkg
    lbpkg.build()
    oracle.build()


def _oracle_run(dims, params, f, g, nsteps):
    f2, g2 = oracle.step(dims, params, f, g, nsteps)
    return (f2, g2), oracle.moments(dims, f2, g2)


def _check_moments(got, want, tol, f_oracle):
    """rho and phi against their max-norms, u against the size of its
    summands (``u_scale``)."""
    for name, a, b in zip(("rho", "u", "phi"), got, want):
        e = rel(a, b, u_scale(f_oracle) if name == "u" else None)
        t = tol[name] if isinstance(tol, dict) else tol
        assert e <= t, f"{name}: {e:.3e} > {t:.1e}"


# ------------------------------------------------------------------ FP64

@pytest.mark.parametrize("kernel,block", KERNEL_CASES)
def test_spinodal_32cubed_fp64(kernel, block):
    """32^3, 10 steps, phi0 ~ U[-0.01, 0.01] seed 0, f and g at equilibrium."""
    dims = (32, 32, 32)
    phi0 = L.spinodal_phi0(*dims, seed=0)
    f0, g0 = oracle.init(dims, P0, phi0)
    (fo, go), mo = _oracle_run(dims, P0, f0, g0, 10)
    with gpu_lattice(dims, P0, "fp64", kernel, block) as lat:
        lat.init(phi0)
        lat.step(10)
        _check_moments(lat.moments(), mo, TOL_FP64, fo)
        f, g = lat.get_state()
    assert rel(to_oracle(f), fo) <= TOL_FP64
    assert rel(to_oracle(g), go) <= TOL_FP64


RAGGED = [(13, 7, 5), (1, 1, 9), (33, 1, 2), (5, 17, 1), (40, 9, 35), (1, 1, 1), (2, 3, 2)]


@pytest.mark.parametrize("dims", RAGGED)
@pytest.mark.parametrize("kernel,block", KERNEL_CASES)
def test_ragged_nonequilibrium_fp64(dims, kernel, block):
    from paper_1405_6162_gb300 import LBError
    p = dict(P0, tau=0.7, tau_g=0.9, kappa=0.06)
    f0, g0 = nonequilibrium_state(dims, p, seed=31)
    (fo, go), mo = _oracle_run(dims, p, f0, g0, 4)
    try:
        lat = gpu_lattice(dims, p, "fp64", kernel, block)
    except LBError:
        if kernel != "bulk":
            raise
        # rows that are not whole 16-byte units, or ny not a multiple of the
        # cluster: refused (test_gpu_bulk checks the refusals)
        pytest.skip("shape outside the bulk kernel's limits")
    with lat:
        lat.set_state(to_abi(f0), to_abi(g0))
        lat.step(4)
        _check_moments(lat.moments(), mo, TOL_FP64, fo)
        f, g = lat.get_state()
    assert rel(to_oracle(f), fo) <= TOL_FP64
    assert rel(to_oracle(g), go) <= TOL_FP64


@pytest.mark.parametrize("precision", ["fp64", "fp32_shifted"])
def test_kernels_agree(precision):
    """Every step kernel runs the same per-site arithmetic; they may differ
    only where the compiler fused a multiply and an add differently in one
    kernel's inlined copy (an ulp or two per step)."""
    dims = (48, 20, 17)
    p = dict(P0, tau=0.8)
    f0, g0 = nonequilibrium_state(dims, p, seed=41)
    out = []
    for kernel, block in (("two_pass", (0, 0, 0)), ("fused", (32, 4, 6)), ("fused", (64, 4, 32)),
                          ("staged", (32, 4, 6)), ("staged", (64, 2, 32)), ("slab", (32, 4, 6)),
                          ("slab", (64, 4, 2)), ("lag", (0, 0, 0)), ("lag", (256, 1, 3))):
        with gpu_lattice(dims, p, precision, kernel, block) as lat:
            lat.set_state(to_abi(f0), to_abi(g0))
            lat.step(6)
            out.append(lat.get_state())
    ulp = 2.0 ** -52 if precision == "fp64" else 2.0 ** -23
    for f, g in out[1:]:
        assert np.abs(f - out[0][0]).max() <= 16 * ulp * np.abs(out[0][0]).max()
        assert np.abs(g - out[0][1]).max() <= 16 * ulp * np.abs(out[0][1]).max()


@pytest.mark.parametrize("kernel,block", [("two_pass", (0, 0, 0)), ("fused", (0, 0, 0)), ("lag", (0, 0, 0))])
def test_flow_u_against_its_max_fp64(kernel, block):
    """A flow-dominated run: u ~ 1e-2 everywhere after 12 steps from a
    non-equilibrium state with a random flow; u is compared with the oracle
    against max|u| itself (not only against the size of its summands) at
    the FP64 bar."""
    dims = (20, 14, 11)
    p = dict(P0, tau=0.8, tau_g=0.7)
    f0, g0 = nonequilibrium_state(dims, p, seed=95)
    (fo, go), mo = _oracle_run(dims, p, f0, g0, 12)
    assert np.abs(mo[1]).max() > 5e-3
    with gpu_lattice(dims, p, "fp64", kernel, block) as lat:
        lat.set_state(to_abi(f0), to_abi(g0))
        lat.step(12)
        rho, u, phi = lat.moments()
    e_u = rel(u, mo[1])
    print(f"flow {kernel}: u vs max|u| = {np.abs(mo[1]).max():.3e}: {e_u:.3e}")
    assert e_u <= TOL_FP64
    assert rel(rho, mo[0]) <= TOL_FP64 and rel(phi, mo[2]) <= TOL_FP64


def test_init_with_flow_matches_oracle():
    dims = (12, 10, 8)
    n = 960
    phi0 = L.spinodal_phi0(*dims, seed=5, amp=0.4)
    u0 = 0.03 * L.uniform(6, 3 * n, -1, 1).reshape(3, n)
    fo, go = oracle.init(dims, P0, phi0, u0)
    with gpu_lattice(dims, P0, "fp64") as lat:
        lat.init(phi0, u0)
        f, g = lat.get_state()
        rho, u, phi = lat.moments()
    assert rel(to_oracle(f), fo) <= 1e-15 and rel(to_oracle(g), go) <= 1e-15
    assert np.abs(rho - 1).max() < 1e-15
    assert rel(u, u0) < 1e-14 and rel(phi, phi0) < 1e-15


def test_device_pointer_inputs_and_outputs():
    import torch
    dims = (16, 8, 4)
    phi0 = L.spinodal_phi0(*dims, seed=8, amp=0.2)
    (fo, go), mo = _oracle_run(dims, P0, *oracle.init(dims, P0, phi0), 3)
    with gpu_lattice(dims, P0, "fp64") as lat:
        lat.init(torch.from_numpy(phi0).cuda())
        lat.step(3)
        rho, u, phi = lat.moments(device=True)
        f, g = lat.get_state(device=True)
        torch.cuda.synchronize()
    _check_moments((rho.cpu().numpy(), u.cpu().numpy(), phi.cpu().numpy()), mo, TOL_FP64, fo)
    assert rel(to_oracle(f.cpu().numpy()), fo) <= TOL_FP64


def test_state_roundtrip_exact_fp64():
    dims = (7, 6, 5)
    f0, g0 = nonequilibrium_state(dims, P0, seed=50)
    with gpu_lattice(dims, P0, "fp64") as lat:
        lat.set_state(to_abi(f0), to_abi(g0))
        f, g = lat.get_state()
    assert np.array_equal(to_oracle(f), f0) and np.array_equal(to_oracle(g), g0)


def test_reductions_match_oracle_and_conserve():
    dims = (24, 20, 16)
    p = dict(P0, tau=0.75)
    f0, g0 = nonequilibrium_state(dims, p, seed=60)
    r_or = oracle.reduce(dims, f0, g0)
    with gpu_lattice(dims, p, "fp64") as lat:
        lat.set_state(to_abi(f0), to_abi(g0))
        r0 = lat.reduce()
        lat.step(200)
        r1 = lat.reduce()
        r1b = lat.reduce()
    assert np.abs(r0 - r_or).max() <= 1e-12 * abs(r_or[0])
    assert np.array_equal(r1, r1b)                      # fixed-order sums
    assert abs(r1[0] - r0[0]) <= 1e-13 * r0[0]
    assert np.abs(r1[1:] - r0[1:]).max() <= 1e-13 * r0[0]


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_nonfinite_state_is_reported(bad):
    from paper_1405_6162_gb300 import LBError
    from paper_1405_6162_gb300 import _lib as LL
    dims = (8, 8, 8)
    f0, g0 = nonequilibrium_state(dims, P0, seed=70)
    f0[3, 100] = bad
    for precision in ("fp64", "fp32_shifted", "fp64_df"):
        with gpu_lattice(dims, P0, precision) as lat:
            lat.set_state(to_abi(f0), to_abi(g0))
            with pytest.raises(LBError) as ei:
                lat.reduce()
            assert ei.value.code == LL.LB_ERR_NONFINITE
            lat.step(1)       # the context stays usable after the report


@pytest.mark.parametrize("precision", ["fp64", "fp32_shifted", "fp64_df"])
def test_reduce_exact_totals(precision):
    """A state on which every sum of stored values is exact in FP64, so the
    totals are fixed to the bit whatever the order of the additions: f =
    w_i rho0 + d with rho0 = 36/64 (w_i rho0 exact in binary) and d integer
    multiples of 2^-24, a seventh of them zero (stored as +0 in the shifted
    form); g integer multiples of 2^-140 (subnormal floats), a fifth of them
    -0.  The widening of each stored float to FP64 must be exact for every
    such class of value."""
    import math
    from paper_1405_6162_gb300 import VELOCITIES
    dims = (20, 12, 10)            # 2400 sites: a ragged last block of 256
    n = int(np.prod(dims))
    rho0 = 36.0 / 64.0
    p = dict(P0, rho0=rho0)
    c = np.asarray(VELOCITIES, dtype=float)
    w = np.where((c ** 2).sum(1) == 0, 1 / 3, np.where((c ** 2).sum(1) == 1, 1 / 18, 1 / 36))
    rng = np.random.default_rng(80)
    d = rng.integers(-2 ** 16, 2 ** 16, size=(19, n)) * 2.0 ** -24
    d[:, ::7] = 0.0
    f = w[:, None] * rho0 + d
    g = rng.integers(-2 ** 10, 2 ** 10, size=(19, n)) * 2.0 ** -140
    g[:, ::5] = -0.0
    assert np.array_equal(f - w[:, None] * rho0, d)          # the shift is exact
    fi = [math.fsum(f[i]) for i in range(19)]
    want = np.array([math.fsum(fi)] + [math.fsum(c[i, a] * fi[i] for i in range(19)) for a in range(3)]
                    + [math.fsum(g.ravel())])
    with gpu_lattice(dims, p, precision) as lat:
        lat.set_state(f, g)
        got = lat.reduce()
    assert np.array_equal(got, want), (got, want)


# ------------------------------------------------------------------ FP32 shifted

# Float rounding of the shifted values (|f - w rho0| <~ 1e-2, ulp ~ 1e-9) and
# of g (|g| <~ 0.5, ulp ~ 3e-8) per step, over 10 steps, relative to each
# field's max-norm.
TOL_FP32 = {"rho": 1e-9, "u": 1e-7, "phi": 1e-5}


@pytest.mark.parametrize("kernel,block", KERNEL_CASES[:3] + KERNEL_CASES[5:7] + KERNEL_CASES[9:11]
                         + KERNEL_CASES[13:15])
def test_spinodal_32cubed_fp32_shifted(kernel, block):
    dims = (32, 32, 32)
    phi0 = L.spinodal_phi0(*dims, seed=0)
    (fo, go), mo = _oracle_run(dims, P0, *oracle.init(dims, P0, phi0), 10)
    with gpu_lattice(dims, P0, "fp32_shifted", kernel, block) as lat:
        lat.init(phi0)
        lat.step(10)
        got = lat.moments()
    print("fp32-shifted 32^3 x 10 errors:",
          {k: rel(a, b, u_scale(fo) if k == "u" else None) for k, a, b in zip(("rho", "u", "phi"), got, mo)})
    _check_moments(got, mo, TOL_FP32, fo)


@pytest.mark.parametrize("kernel", ["fused", "staged", "slab", "lag"])
@pytest.mark.parametrize("dims", [(13, 7, 5), (40, 9, 35), (1, 1, 3)])
def test_ragged_fp32_shifted_one_step(dims, kernel):
    """One step from a float-representable state: the only difference from
    the FP64 oracle is float arithmetic within the step."""
    p = dict(P0, tau=0.7)
    f0, g0 = nonequilibrium_state(dims, p, seed=80)
    block = (0, 0, 1) if kernel == "lag" else (32, 2, 3)
    with gpu_lattice(dims, p, "fp32_shifted", kernel, block) as lat:
        lat.set_state(to_abi(f0), to_abi(g0))
        fin, gin = lat.get_state()          # float-rounded input state
        lat.step(1)
        f, g = lat.get_state()
    (fo, go), _ = _oracle_run(dims, p, to_oracle(fin), to_oracle(gin), 1)
    _, w = oracle.velocity_set()
    df = to_oracle(f) - fo
    shift = fo - w[:, None] * p["rho0"]
    # ~20 dependent float operations per value: allow 16 ulp of the largest
    # shifted value
    assert np.abs(df).max() <= 1e-6 * np.abs(shift).max()
    assert rel(to_oracle(g), go) <= 1e-6


# ------------------------------------------------------------------ bounded waits

@pytest.mark.parametrize("precision", ["fp64", "fp32_shifted"])
def test_lagged_kernel_wait_timeout_is_reported_and_recoverable(precision):
    """The lagged kernel's inter-CTA waits are time-bounded: with targets made
    unreachable (test hook) every wait gives up, the kernel returns, and the
    host sees LB_ERR_TIMEOUT; after re-initialisation the context is exact
    again."""
    from paper_1405_6162_gb300 import LBError
    from paper_1405_6162_gb300 import _lib as LL
    dims = (16, 12, 10)
    phi0 = L.spinodal_phi0(*dims, seed=11, amp=0.3)
    (fo, go), mo = _oracle_run(dims, P0, *oracle.init(dims, P0, phi0), 3)
    with gpu_lattice(dims, P0, precision, "lag", (0, 0, 0)) as lat:
        lat.set_wait_timeout(0.05)
        LL.check(LL.lib().lb_debug_wait_skew(lat.handle, 1 << 40), "skew")
        lat.init(phi0)
        lat.step(2)
        with pytest.raises(LBError) as ei:
            lat.sync()
        assert ei.value.code == LL.LB_ERR_TIMEOUT
        lat.sync()                                  # reported once, then cleared
        LL.check(LL.lib().lb_debug_wait_skew(lat.handle, 0), "skew")
        lat.init(phi0)
        lat.step(3)
        got = lat.moments()
    # phi0 amplitude 0.3 makes the stress terms O(1e-2): FP32 per-step bounds
    tol = TOL_FP64 if precision == "fp64" else {"rho": 1e-7, "u": 1e-7, "phi": 1e-6}
    _check_moments(got, mo, tol, fo)


@pytest.mark.parametrize("precision,kernel", [("fp32_shifted", "two_pass"), ("fp64", "two_pass"),
                                              ("fp64_df", "two_pass"), ("fp32_shifted", "taug1")])
def test_dependent_launch_chain_with_interleaved_work(precision, kernel):
    """The kernel pairs are chained with programmatic dependent launch.  A
    run broken up by other work on the stream between steps (state and
    moments read on the device, a torch kernel reading the state) gives the
    bits of one uninterrupted run, and both match the oracle."""
    import torch
    dims = (24, 18, 11)
    phi0 = L.spinodal_phi0(*dims, seed=77, amp=0.3)
    with gpu_lattice(dims, P0, precision, kernel) as a, gpu_lattice(dims, P0, precision, kernel) as b:
        a.init(phi0)
        b.init(phi0)
        a.step(9)
        for _ in range(9):
            b.step(1)
            f, g = b.get_state(device=True)
            assert torch.isfinite(f.sum() + g.sum()).item()
            b.moments(device=True)
        fa, ga = a.get_state()
        fb, gb = b.get_state()
        torch.cuda.synchronize()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    fo, go = oracle.step(dims, P0, *oracle.init(dims, P0, phi0), 9)
    tol = TOL_FP64 if precision != "fp32_shifted" else 2e-6
    assert rel(to_oracle(fa), fo) <= tol and rel(to_oracle(ga), go) <= tol
