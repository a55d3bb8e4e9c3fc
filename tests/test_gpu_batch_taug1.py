"""The ensemble in the tau_g = 1 reduced form (lb_batch_set_form): every
lattice against the oracle, switching forms mid-run, graph replays split
across parities, the refusal for tau_g != 1 and the bounded grid barrier."""
import numpy as np
import pytest

import lb_inputs as L
import oracle
from tests.parity import TOL_FP64, rel, u_scale

pytestmark = pytest.mark.gpu

TOL_FP32_PER_STEP = {"rho": 2.5e-8, "u": 2.5e-8, "phi": 1e-7}


@pytest.fixture(scope="module", autouse=True)
def _setup():
    import paper_1405_6162_gb300 as lbpkg
    lbpkg.build()
    oracle.build()


def _ensemble(seed, n=6):
    specs = L.ensemble(seed, n, lo=3, hi=40)
    specs[0].update(nx=1, ny=1, nz=7)          # degenerate extents too
    specs[1].update(nx=13, ny=1, nz=2)
    specs[2].update(nx=70, ny=9, nz=11)        # several x blocks of the phi tiles
    for d in specs:
        assert d["tau_g"] == 1.0
    return specs


def _phi0(spec, k, amp=0.3):
    return L.spinodal_phi0(spec["nx"], spec["ny"], spec["nz"], seed=200 + k, amp=amp)


def _oracle(spec, phi0, nsteps):
    dims = (spec["nx"], spec["ny"], spec["nz"])
    f, g = oracle.step(dims, spec, *oracle.init(dims, spec, phi0), nsteps)
    return oracle.moments(dims, f, g), u_scale(f), (f, g)


def _check(b, specs, nsteps, precision):
    for k, d in enumerate(specs):
        (rho, u, phi), us, _ = _oracle(d, _phi0(d, k), nsteps)
        got = b[k].moments()
        for name, a, ref in zip(("rho", "u", "phi"), got, (rho, u, phi)):
            e = rel(a, ref, us if name == "u" else None)
            tol = TOL_FP64 if precision == "fp64" else TOL_FP32_PER_STEP[name] * nsteps
            assert e <= tol, (k, name, e)


@pytest.mark.parametrize("precision", ["fp64", "fp32_shifted"])
@pytest.mark.parametrize("launch", [(256, 0), (128, 1), (64, 2)])
@pytest.mark.parametrize("plan", ["lattice", "grid", 3])
def test_reduced_ensemble_matches_oracle(precision, launch, plan):
    from paper_1405_6162_gb300 import Batch
    specs = _ensemble(11)
    with Batch(specs, precision=precision) as b:
        b.set_plan(plan)
        b.set_launch(*launch)
        b.set_form("taug1")
        for k, d in enumerate(specs):
            b[k].init(_phi0(d, k))
        b.run(15)
        b.sync()
        _check(b, specs, 15, precision)


def test_switching_forms_mid_run():
    from paper_1405_6162_gb300 import Batch
    specs = _ensemble(12)
    with Batch(specs, precision="fp64") as b:
        for k, d in enumerate(specs):
            b[k].init(_phi0(d, k))
        b.run(5)
        b.set_form("taug1")
        b.run(5)
        b.set_form("general")
        b.run(5)
        b.sync()
        _check(b, specs, 15, "fp64")
        # the full state too (the reduced form reports the streamed equilibria)
        for k, d in enumerate(specs):
            _, _, (fo, go) = _oracle(d, _phi0(d, k), 15)
            from tests.parity import to_oracle
            f, g = b[k].get_state()
            assert rel(to_oracle(f), fo) <= TOL_FP64 and rel(to_oracle(g), go) <= TOL_FP64


def test_split_runs_equal_one_run():
    from paper_1405_6162_gb300 import Batch
    specs = _ensemble(13)
    out = []
    for plan in ((15,), (7, 8), (1, 1, 13)):
        with Batch(specs, precision="fp32_shifted") as b:
            b.set_form("taug1")
            for k, d in enumerate(specs):
                b[k].init(_phi0(d, k))
            for n in plan:
                b.run(n)
            out.append([b[k].moments() for k in range(len(specs))])
    for other in out[1:]:
        for m0, m1 in zip(out[0], other):
            for a, c in zip(m0, m1):
                assert np.array_equal(a, c)


def test_refused_unless_tau_g_is_one():
    from paper_1405_6162_gb300 import Batch, LBError
    specs = _ensemble(14, n=3)
    specs[1]["tau_g"] = 0.9
    with Batch(specs, precision="fp32_shifted") as b:
        with pytest.raises(LBError):
            b.set_form("taug1")
        b.set_form("general")


def test_grid_barrier_timeout_in_reduced_form():
    from paper_1405_6162_gb300 import Batch, LBError
    from paper_1405_6162_gb300 import _lib as LL
    specs = _ensemble(15, n=3)
    with Batch(specs, precision="fp32_shifted") as b:
        b.set_form("taug1")
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
        _check(b, specs, 4, "fp32_shifted")


def test_reduced_ensemble_64_uneven_lattices_500_steps_fp32():
    """The 64-lattice workload in the reduced form, compared with the oracle
    on the same nine lattices and bounds as the general form."""
    from paper_1405_6162_gb300 import Batch
    from tests.parity import ensemble_subsample, ensemble_workload, sites
    from tests.test_gpu_batch import _check_ensemble_subsample
    specs, phis = ensemble_workload()
    with Batch(specs, precision="fp32_shifted") as b:
        b.set_form("taug1")
        for k in range(len(specs)):
            b[k].init(phis[k])
        r0 = [b[k].reduce() for k in range(len(specs))]
        b.run(500)
        b.sync()
        r1 = [b[k].reduce() for k in range(len(specs))]
        for k, d in enumerate(specs):
            assert abs(r1[k][4] - r0[k][4]) <= 1e-6 * sites(d), (k, r1[k][4] - r0[k][4])
        got = {k: b[k].moments() for k in ensemble_subsample(specs)}
    _check_ensemble_subsample(specs, got, "reduced")
