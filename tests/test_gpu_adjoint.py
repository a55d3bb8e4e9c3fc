"""The adjoint path: liblb's reverse kernel pair and the checkpointed
autograd function, against the CPU oracle's hand-written reverse mode (itself
pinned by complex step) and against finite differences of GPU forward runs."""
import numpy as np
import pytest

import lb_inputs as L
import oracle
from tests.parity import P0, nonequilibrium_state, rel, to_abi, to_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    import paper_1405_6162_gb300 as lbpkg
    lbpkg.build()
    oracle.build()


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).cuda()


def test_one_reverse_step_matches_oracle():
    import torch
    from paper_1405_6162_gb300 import Lattice
    from paper_1405_6162_gb300 import _lib as LL
    dims = (12, 10, 8)
    n = 960
    p = dict(P0, tau=0.8, tau_g=0.9, kappa=0.05)
    f, g = nonequilibrium_state(dims, p, seed=200, amp=0.6)
    af = L.uniform(201, 19 * n, -1, 1).reshape(19, n)
    ag = L.uniform(202, 19 * n, -1, 1).reshape(19, n)
    af_o, ag_o, dk_o = oracle.step_adjoint(dims, p, f, g, af, ag)
    with Lattice.from_params(dims, p, precision="fp64") as lat:
        tf, tg, taf, tag = (_cuda(to_abi(x)) for x in (f, g, af, ag))
        oaf, oag = torch.empty_like(taf), torch.empty_like(tag)
        dk = torch.zeros(1, dtype=torch.float64, device="cuda")
        LL.check(LL.lib().lb_adjoint_step(lat.handle, tf.data_ptr(), tg.data_ptr(), taf.data_ptr(), tag.data_ptr(),
                                          oaf.data_ptr(), oag.data_ptr(), dk.data_ptr()), "adjoint")
        torch.cuda.synchronize()
    assert rel(to_oracle(oaf.cpu().numpy().reshape(19, n)), af_o) <= 1e-12
    assert rel(to_oracle(oag.cpu().numpy().reshape(19, n)), ag_o) <= 1e-12
    assert abs(dk.item() - dk_o) <= 1e-12 * abs(dk_o)


def test_init_reverse_matches_oracle():
    import torch
    from paper_1405_6162_gb300 import Lattice
    from paper_1405_6162_gb300 import _lib as LL
    dims = (9, 7, 6)
    n = 378
    p = dict(P0, kappa=0.06)
    phi0 = L.spinodal_phi0(*dims, seed=210, amp=0.5)
    af = L.uniform(211, 19 * n, -1, 1).reshape(19, n)
    ag = L.uniform(212, 19 * n, -1, 1).reshape(19, n)
    pb_o, dk_o = oracle.init_adjoint(dims, p, phi0, af, ag)
    with Lattice.from_params(dims, p, precision="fp64") as lat:
        tphi, taf, tag = _cuda(phi0), _cuda(to_abi(af)), _cuda(to_abi(ag))
        pb = torch.empty(n, dtype=torch.float64, device="cuda")
        dk = torch.zeros(1, dtype=torch.float64, device="cuda")
        LL.check(LL.lib().lb_adjoint_init(lat.handle, tphi.data_ptr(), None, taf.data_ptr(), tag.data_ptr(),
                                          pb.data_ptr(), dk.data_ptr()), "adjoint init")
        torch.cuda.synchronize()
    assert rel(pb.cpu().numpy(), pb_o) <= 1e-12
    assert abs(dk.item() - dk_o) <= 1e-12 * abs(dk_o)


@pytest.mark.parametrize("segment", [1, 5, 20])
def test_trajectory_gradient_matches_oracle_16cubed(segment):
    """16^3, T = 20: the checkpointed GPU gradient equals the oracle's
    reverse sweep (any checkpoint spacing)."""
    import torch
    from paper_1405_6162_gb300.adjoint import trajectory
    dims = (16, 16, 16)
    T = 20
    phi0 = L.spinodal_phi0(*dims, seed=220, amp=0.3)
    xi = L.interface_width(P0["A"], P0["kappa"])
    tgt = L.droplet_target(*dims, radius=4.0, xi=xi, seed=221)
    J_o, gphi_o, gk_o = oracle.trajectory_gradient(dims, P0, phi0, tgt, T)
    x = _cuda(phi0).requires_grad_(True)
    kappa = torch.tensor(P0["kappa"], dtype=torch.float64, device="cuda", requires_grad=True)
    phi_t = trajectory(x, kappa, dims, P0, T, segment=segment)
    J = ((phi_t - _cuda(tgt)) ** 2).sum()
    J.backward()
    assert abs(J.item() - J_o) <= 1e-12 * J_o
    assert rel(x.grad.cpu().numpy(), gphi_o) <= 1e-10
    assert abs(kappa.grad.item() - gk_o) <= 1e-10 * abs(gk_o)


def test_gradient_agrees_with_finite_differences_64cubed_T200():
    """The 64^3, T = 200 workload: loss sum (phi_T - phi_target)^2 with a
    seeded tanh droplet of radius 16; gradient wrt kappa and along random
    phi0 directions against central differences of GPU forward runs."""
    import torch
    from paper_1405_6162_gb300.adjoint import trajectory
    dims = (64, 64, 64)
    n = 64 ** 3
    T = 200
    phi0 = _cuda(L.spinodal_phi0(*dims, seed=4))
    xi = L.interface_width(P0["A"], P0["kappa"])
    tgt = _cuda(L.droplet_target(*dims, radius=16.0, xi=xi, seed=5))

    def phi_t(ph, kap):
        with torch.no_grad():
            return trajectory(ph, kap, dims, P0, T)

    def central(pp, pm, h):
        # J(+) - J(-) summed site by site: J is ~2.6e5 while the derivatives
        # are O(1), so differencing two rounded totals would lose ~4e-6
        return float(((pp - pm) * (pp + pm - 2 * tgt)).sum()) / (2 * h)

    x = phi0.clone().requires_grad_(True)
    kappa = torch.tensor(P0["kappa"], dtype=torch.float64, device="cuda", requires_grad=True)
    J = ((trajectory(x, kappa, dims, P0, T) - tgt) ** 2).sum()
    J.backward()
    gk = kappa.grad.item()
    # dJ/dkappa is O(1) while J'' is large: the central difference converges
    # as O(h^2) with error 1e-5 at h = 1e-5 (measured), so extrapolate
    # (Richardson) from h and h/2 to remove the h^2 term
    k0, hk = P0["kappa"], 2e-5
    d1 = central(phi_t(phi0, k0 + hk), phi_t(phi0, k0 - hk), hk)
    d2 = central(phi_t(phi0, k0 + hk / 2), phi_t(phi0, k0 - hk / 2), hk / 2)
    fd = (4 * d2 - d1) / 3
    print("dJ/dkappa adjoint", gk, "FD", d1, d2, "extrapolated", fd)
    assert abs(fd - gk) <= 1e-6 * abs(gk)
    for seed in (6, 7, 8):
        v = _cuda(L.uniform(seed, n, -1, 1))
        h = 1e-5
        fd = central(phi_t(phi0 + h * v, P0["kappa"]), phi_t(phi0 - h * v, P0["kappa"]), h)
        g = float((x.grad * v).sum())
        print("directional", seed, g, fd)
        assert abs(fd - g) <= 1e-6 * abs(g)


def test_adjoint_seed_is_the_transpose_of_the_phi_readout():
    """lb_adjoint_seed writes the adjoint of phi_T = sum_i g_i(T): f_bar = 0
    and g_bar_i(x) = dJ/dphi_T(x) for every i, bit for bit; hence
    <seed(p), (f, g)> = <p, sum_i g_i> for any state."""
    import torch
    from paper_1405_6162_gb300 import Lattice
    from paper_1405_6162_gb300 import _lib as LL
    dims = (9, 7, 5)
    n = 315
    pbar = torch.from_numpy(L.uniform(17, n, -1, 1)).cuda()
    af = torch.full((19 * n,), 7.0, dtype=torch.float64, device="cuda")
    ag = torch.empty_like(af)
    with Lattice.from_params(dims, P0, precision="fp64") as lat:
        LL.check(LL.lib().lb_adjoint_seed(lat.handle, pbar.data_ptr(), af.data_ptr(), ag.data_ptr()), "seed")
        torch.cuda.synchronize()
        assert LL.lib().lb_adjoint_seed(lat.handle, pbar.data_ptr(), af.data_ptr(), af.data_ptr()) == \
            LL.LB_ERR_INVALID
    assert bool((af == 0).all())
    assert torch.equal(ag.view(19, n), pbar.expand(19, n))
    g = torch.from_numpy(L.uniform(18, 19 * n, -1, 1)).cuda()
    lhs = float((ag * g).sum())
    rhs = float((pbar * g.view(19, n).sum(0)).sum())
    assert abs(lhs - rhs) <= 1e-13 * abs(rhs)
