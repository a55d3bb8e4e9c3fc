"""Pins of the oracle's hand-written reverse mode (no GPU).

The adjoint sweep (reverse of streaming, collision, stencils, phi = sum g and
initialisation) is checked against derivatives that do not use it: the
complex-step derivative of the forward oracle (every operation is analytic,
so Im J(p + ih)/h is dJ/dp to rounding) and central finite differences.
Loss J = sum_x (phi_T - phi_target)^2 (the droplet-target workload).
"""
import numpy as np
import pytest

import lb_inputs as L
import oracle

P = dict(L.DEFAULT_PARAMS, tau=0.8, tau_g=0.9)
DIMS = (6, 5, 4)
T = 12


@pytest.fixture(scope="module")
def setup():
    oracle.build()
    n = int(np.prod(DIMS))
    phi0 = L.spinodal_phi0(*DIMS, seed=31, amp=0.4)
    xi = L.interface_width(P["A"], P["kappa"])
    tgt = L.droplet_target(*DIMS, radius=2.0, xi=xi, seed=32)
    J, gphi, gk = oracle.trajectory_gradient(DIMS, P, phi0, tgt, T)
    return n, phi0, tgt, J, gphi, gk


def test_dkappa_matches_complex_step(setup):
    n, phi0, tgt, J, gphi, gk = setup
    h = 1e-20
    pc = dict(P, kappa=P["kappa"] + 1j * h)
    Jc = oracle.trajectory_loss(DIMS, pc, phi0.astype(complex), tgt, T, kind="complex")
    assert abs(Jc.real - J) <= 1e-12 * abs(J)
    assert abs(Jc.imag / h - gk) <= 1e-10 * abs(gk)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_dphi0_matches_complex_step_directional(setup, seed):
    n, phi0, tgt, J, gphi, gk = setup
    v = L.uniform(seed, n, -1, 1)
    h = 1e-20
    Jc = oracle.trajectory_loss(DIMS, P, phi0 + 1j * h * v, tgt, T, kind="complex")
    assert abs(Jc.imag / h - gphi @ v) <= 1e-10 * np.abs(gphi).sum()


def test_central_finite_differences(setup):
    n, phi0, tgt, J, gphi, gk = setup
    hk = 1e-6
    Jp = oracle.trajectory_loss(DIMS, dict(P, kappa=P["kappa"] + hk), phi0, tgt, T)
    Jm = oracle.trajectory_loss(DIMS, dict(P, kappa=P["kappa"] - hk), phi0, tgt, T)
    assert abs((Jp - Jm) / (2 * hk) - gk) <= 1e-6 * abs(gk)
    for s in (0, 17, n - 1):
        e = np.zeros(n)
        e[s] = 1e-6
        Jp = oracle.trajectory_loss(DIMS, P, phi0 + e, tgt, T)
        Jm = oracle.trajectory_loss(DIMS, P, phi0 - e, tgt, T)
        assert abs((Jp - Jm) / 2e-6 - gphi[s]) <= 1e-6 * np.abs(gphi).max()


def test_single_step_adjoint_is_the_transpose():
    """<J v, w> = <v, J^T w> for the one-step map F(t) -> F(t+1), with the
    Jacobian-vector product taken by complex step."""
    oracle.build()
    n = int(np.prod(DIMS))
    f, g = oracle.init(DIMS, P, L.spinodal_phi0(*DIMS, seed=40, amp=0.5))
    f = f * (1 + 0.05 * L.uniform(41, 19 * n, -1, 1).reshape(19, n))
    vf = L.uniform(42, 19 * n, -1, 1).reshape(19, n)
    vg = L.uniform(43, 19 * n, -1, 1).reshape(19, n)
    wf = L.uniform(44, 19 * n, -1, 1).reshape(19, n)
    wg = L.uniform(45, 19 * n, -1, 1).reshape(19, n)
    h = 1e-20
    fc, gc = oracle.step(DIMS, P, f + 1j * h * vf, g + 1j * h * vg, 1, kind="complex")
    jv = (np.sum(fc.imag / h * wf) + np.sum(gc.imag / h * wg))
    af, ag, _ = oracle.step_adjoint(DIMS, P, f, g, wf, wg)
    vjt = np.sum(af * vf) + np.sum(ag * vg)
    assert abs(jv - vjt) <= 1e-12 * (np.abs(af).sum() + np.abs(ag).sum())
