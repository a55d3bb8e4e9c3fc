"""The ensemble path: many uneven lattices in one persistent, graph-captured
launch, each checked against the CPU oracle run on that lattice alone."""
import numpy as np
import pytest

import lb_inputs as L
import oracle
from tests.parity import (ENSEMBLE_STEPS, P0, TOL_FP64, ensemble_oracle, ensemble_subsample, ensemble_workload,
                          fp32_spinodal_bounds, rel, sites, spinodal_rate, u_scale)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    import paper_1405_6162_gb300 as lbpkg
    lbpkg.build()
    oracle.build()


def _small_ensemble(seed, n=6):
    specs = L.ensemble(seed, n, lo=3, hi=20)
    specs[0].update(nx=1, ny=1, nz=7)          # degenerate extents too
    specs[1].update(nx=13, ny=1, nz=2)
    return specs


def _oracle(spec, phi0, nsteps):
    dims = (spec["nx"], spec["ny"], spec["nz"])
    f, g = oracle.step(dims, spec, *oracle.init(dims, spec, phi0), nsteps)
    return oracle.moments(dims, f, g), u_scale(f)


def _phi0(spec, k, amp=0.3):
    return L.spinodal_phi0(spec["nx"], spec["ny"], spec["nz"], seed=100 + k, amp=amp)


TOL_FP32_PER_STEP = {"rho": 2.5e-8, "u": 2.5e-8, "phi": 1e-7}


@pytest.mark.parametrize("precision", ["fp64", "fp32_shifted"])
@pytest.mark.parametrize("launch", [(256, 0), (128, 1), (64, 2)])
@pytest.mark.parametrize("plan", ["lattice", "grid", 2])
def test_ensemble_matches_oracle_per_lattice(precision, launch, plan):
    from paper_1405_6162_gb300 import Batch
    specs = _small_ensemble(7)
    nsteps = 15
    with Batch(specs, precision=precision) as b:
        b.set_plan(plan)
        b.set_launch(*launch)
        assert b.groups() == {"lattice": len(specs), "grid": 1}.get(plan, plan)
        for k, d in enumerate(specs):
            b[k].init(_phi0(d, k))
        b.run(nsteps)
        b.sync()
        for k, d in enumerate(specs):
            (rho, u, phi), us = _oracle(d, _phi0(d, k), nsteps)
            got = b[k].moments()
            for name, a, ref in zip(("rho", "u", "phi"), got, (rho, u, phi)):
                e = rel(a, ref, us if name == "u" else None)
                tol = TOL_FP64 if precision == "fp64" else TOL_FP32_PER_STEP[name] * nsteps
                assert e <= tol, (k, name, e)


def test_split_runs_equal_one_run():
    """Graph per (steps, parity): 7 + 8 steps give exactly the 15-step state."""
    from paper_1405_6162_gb300 import Batch
    specs = _small_ensemble(8)
    out = []
    for plan in ((15,), (7, 8), (1, 1, 13)):
        with Batch(specs, precision="fp32_shifted") as b:
            for k, d in enumerate(specs):
                b[k].init(_phi0(d, k))
            for n in plan:
                b.run(n)
            out.append([b[k].get_state() for k in range(len(specs))])
    for other in out[1:]:
        for (f0, g0), (f1, g1) in zip(out[0], other):
            assert np.array_equal(f0, f1) and np.array_equal(g0, g1)


def test_plans_give_identical_states():
    """The CTA plan changes only which CTA runs which site: the per-lattice
    groups, the one-group grid and a switch between them mid-run give
    bit-identical states; with more lattices than CTAs (one CTA per SM)
    groups hold several lattices."""
    from paper_1405_6162_gb300 import Batch
    specs = L.ensemble(16, 200, lo=2, hi=8)
    out = []
    for plans in (("lattice",), ("grid",), (8,), ("lattice", "grid"), ("grid", 3), (5, "lattice")):
        with Batch(specs, precision="fp32_shifted") as b:
            b.set_launch(32, 0)
            for k, d in enumerate(specs):
                b[k].init(_phi0(d, k))
            for p in plans:
                b.set_plan(p)
                b.run(6 // len(plans))
            out.append([b[k].get_state() for k in range(len(specs))])
    with Batch(specs, precision="fp32_shifted") as b:
        b.set_launch(256, 1)
        ctas = b.info()[2]
        assert ctas < len(specs) and b.groups() == ctas
        for k, d in enumerate(specs):
            b[k].init(_phi0(d, k))
        b.run(6)
        out.append([b[k].get_state() for k in range(len(specs))])
    for other in out[1:]:
        for (f0, g0), (f1, g1) in zip(out[0], other):
            assert np.array_equal(f0, f1) and np.array_equal(g0, g1)


def test_members_belong_to_the_ensemble():
    from paper_1405_6162_gb300 import Batch, LBError
    from paper_1405_6162_gb300 import _lib as LL
    specs = _small_ensemble(9, n=2)
    with Batch(specs, precision="fp64") as b:
        h = b[0].handle
        assert LL.lib().lb_step(h, 1) == LL.LB_ERR_INVALID
        LL.lib().lb_destroy(h)                  # ignored: the ensemble owns it
        b[0].init(_phi0(specs[0], 0))
        b.run(2)
        b.sync()
        assert np.isfinite(b[0].reduce()).all()
        assert LL.lib().lb_batch_lattice(b.handle, 2) is None
        with pytest.raises(LBError):
            b.set_launch(48, 0)


@pytest.mark.parametrize("precision", ["fp64", "fp32_shifted"])
@pytest.mark.parametrize("plan", ["lattice", "grid"])
def test_grid_barrier_timeout_is_reported_and_recoverable(precision, plan):
    """One CTA leaves before its group's first barrier (test hook): the
    group's other CTAs' bounded waits give up, the kernel ends, the host sees
    LB_ERR_TIMEOUT, and after re-initialisation the ensemble is exact."""
    from paper_1405_6162_gb300 import Batch, LBError
    from paper_1405_6162_gb300 import _lib as LL
    specs = _small_ensemble(10, n=3)
    with Batch(specs, precision=precision) as b:
        b.set_plan(plan)
        b.set_wait_timeout(0.05)
        LL.check(LL.lib().lb_batch_debug_skip_arrival(b.handle, 1), "hook")
        for k, d in enumerate(specs):
            b[k].init(_phi0(d, k))
        b.run(3)
        with pytest.raises(LBError) as ei:
            b.sync()
        assert ei.value.code == LL.LB_ERR_TIMEOUT
        b.sync()
        LL.check(LL.lib().lb_batch_debug_skip_arrival(b.handle, 0), "hook")
        for k, d in enumerate(specs):
            b[k].init(_phi0(d, k))
        b.run(4)
        b.sync()
        for k, d in enumerate(specs):
            (rho, u, phi), us = _oracle(d, _phi0(d, k), 4)
            got = b[k].moments()
            tol = TOL_FP64 if precision == "fp64" else 1e-6
            assert rel(got[2], phi) <= tol


def test_ensemble_64_uneven_lattices_500_steps_fp32():
    """The 64-lattice workload: sides U{16..64}, tau ~ U[0.55, 1.5],
    kappa ~ U[0.01, 0.08], FP32-shifted, 500 steps in one graph replay.
    Every lattice conserves mass and phi (FP64 sums); nine lattices that
    cover the workload's extremes (the two largest, the smallest, the most
    and least unstable, the extreme taus) are compared with the oracle at
    the 1000-step spinodal bounds, scaled by each run's spinodal growth
    factor beyond that reference's."""
    from paper_1405_6162_gb300 import Batch
    specs, phis = ensemble_workload()
    nsteps = ENSEMBLE_STEPS
    with Batch(specs, precision="fp32_shifted") as b:
        for k in range(len(specs)):
            b[k].init(phis[k])
        r0 = [b[k].reduce() for k in range(len(specs))]
        b.run(nsteps)
        b.sync()
        r1 = [b[k].reduce() for k in range(len(specs))]
        for k, d in enumerate(specs):
            n = sites(d)
            assert abs(r1[k][0] - r0[k][0]) <= 1e-6 * n, (k, r1[k][0] - r0[k][0])
            assert abs(r1[k][4] - r0[k][4]) <= 1e-6 * n, (k, r1[k][4] - r0[k][4])
        got = {k: b[k].moments() for k in ensemble_subsample(specs)}
    _check_ensemble_subsample(specs, got, "general")


def _check_ensemble_subsample(specs, got, form):
    bad = []
    for k, moments in got.items():
        (rho, u, phi), us = ensemble_oracle(k)
        errs = {name: rel(a, ref, us if name == "u" else None)
                for name, a, ref in zip(("rho", "u", "phi"), moments, (rho, u, phi))}
        errs["u_vs_max_u"] = rel(moments[1], u)
        bounds = fp32_spinodal_bounds(specs[k], ENSEMBLE_STEPS)
        d = specs[k]
        print(f"{form} lattice {k} {d['nx']}x{d['ny']}x{d['nz']} tau={d['tau']:.3f} kappa={d['kappa']:.4f} "
              f"sigmaT={spinodal_rate(d) * ENSEMBLE_STEPS:.2f}:",
              {n: f"{e:.2e}" for n, e in errs.items()}, "bounds", {n: f"{e:.1e}" for n, e in bounds.items()})
        bad += [(k, n, errs[n], bounds[n]) for n in bounds if not errs[n] <= bounds[n]]
    assert not bad, bad
