"""Masked copies (lb_moments_masked, lb_get_state_masked, lb_set_state_masked)
against the oracle's select_sites / scatter_sites, through the C ABI.

Index work is bit-exact: the selected columns of the GPU's own full copies
must come back unchanged and in site order; values computed from the state
match the oracle to the FP64 bound.  Masks: empty, one site, sparse random
(bytes other than 1 included), an interface band, full; host and device.
"""
import numpy as np
import pytest

import lb_inputs as L
import oracle
from tests.parity import P0, TOL_FP64, nonequilibrium_state, rel, to_abi, to_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    import paper_1405_6162_gb300 as lbpkg
    lbpkg.build()
    oracle.build()


def _lat(dims, precision="fp64", kernel="auto", params=P0):
    from paper_1405_6162_gb300 import Lattice
    lat = Lattice.from_params(dims, params, precision=precision)
    lat.set_kernel(kernel)
    return lat


def _masks(n, phi, seed):
    m_sparse = (L.uniform(seed, n, 0, 1) < 0.07).astype(np.uint8) * (1 + L.uniform_int(seed + 1, n, 0, 254)).astype(np.uint8)
    one = np.zeros(n, np.uint8)
    one[n // 2] = 7
    return {"empty": np.zeros(n, np.uint8), "one": one, "sparse": m_sparse,
            "interface": (np.abs(phi) < 0.25 * np.abs(phi).max()).astype(np.uint8), "full": np.ones(n, np.uint8)}


@pytest.mark.parametrize("device", [False, True])
@pytest.mark.parametrize("dims", [(13, 7, 5), (40, 9, 35), (32, 32, 32)])
def test_moments_masked_fp64(dims, device):
    import torch
    n = int(np.prod(dims))
    phi0 = L.spinodal_phi0(*dims, seed=900, amp=0.5)
    fo, go = oracle.step(dims, P0, *oracle.init(dims, P0, phi0), 5)
    mo = oracle.moments(dims, fo, go)
    with _lat(dims) as lat:
        lat.init(phi0)
        lat.step(5)
        full = lat.moments()
        for name, m in _masks(n, mo[2], 901).items():
            mk = torch.from_numpy(m).cuda() if device else m
            k = lat.count_masked(mk)
            assert k == int((m != 0).sum()), name
            got = lat.moments_masked(mk)
            if device:
                got = tuple(x.cpu().numpy() for x in got)
            for a, b, c in zip(got, full, mo):
                want_gpu = oracle.select_sites(b, m)
                assert a.shape == want_gpu.shape and np.array_equal(a, want_gpu), name
                if k:
                    assert rel(a, oracle.select_sites(c, m)) <= TOL_FP64 or np.abs(a).max() < 1e-14, name


@pytest.mark.parametrize("precision", ["fp64", "fp32_shifted"])
def test_state_masked_round_trip(precision):
    dims = (16, 12, 10)
    n = 1920
    p = dict(P0, tau=0.8)
    f0, g0 = nonequilibrium_state(dims, p, seed=910)
    m = _masks(n, L.spinodal_phi0(*dims, seed=911, amp=0.5), 912)["sparse"]
    k = int((m != 0).sum())
    with _lat(dims, precision, params=p) as lat:
        lat.set_state(to_abi(f0), to_abi(g0))
        lat.step(2)
        F, G = lat.get_state()
        fm, gm = lat.get_state_masked(m)
        assert np.array_equal(fm, oracle.select_sites(F, m)) and np.array_equal(gm, oracle.select_sites(G, m))
        # overwrite the selected sites with other values
        nf = np.round(fm * 64) / 64
        ng = np.round(gm * 64) / 64
        lat.set_state_masked(m, nf, ng)
        F2, G2 = lat.get_state()
    # the same as setting the scattered full state (FP32 stores f - w rho0, so
    # a set/get round trip is exact only in FP64)
    Fs, Gs = oracle.scatter_sites(F, m, nf), oracle.scatter_sites(G, m, ng)
    with _lat(dims, precision, params=p) as ref:
        ref.set_state(Fs, Gs)
        F3, G3 = ref.get_state()
    assert np.array_equal(F2, F3) and np.array_equal(G2, G3)
    if precision == "fp64":
        assert np.array_equal(F2, Fs) and np.array_equal(G2, Gs)
    assert k > 0


def test_set_state_masked_then_step_matches_oracle():
    dims = (12, 10, 8)
    n = 960
    p = dict(P0, tau=0.7, tau_g=0.85)
    f0, g0 = nonequilibrium_state(dims, p, seed=920)
    f1, g1 = nonequilibrium_state(dims, p, seed=921)
    m = (L.uniform(922, n, 0, 1) < 0.3).astype(np.uint8)
    fs = oracle.scatter_sites(f0, m, oracle.select_sites(f1, m))
    gs = oracle.scatter_sites(g0, m, oracle.select_sites(g1, m))
    fo, go = oracle.step(dims, p, fs, gs, 4)
    import torch
    with _lat(dims, params=p) as lat:
        lat.set_state(to_abi(f0), to_abi(g0))
        md = torch.from_numpy(m).cuda()
        lat.set_state_masked(md, torch.from_numpy(to_abi(oracle.select_sites(f1, m))).cuda().contiguous(),
                             torch.from_numpy(to_abi(oracle.select_sites(g1, m))).cuda().contiguous())
        lat.step(4)
        f, g = lat.get_state()
    assert rel(to_oracle(f), fo) <= TOL_FP64 and rel(to_oracle(g), go) <= TOL_FP64


def test_reduced_form_moments_and_refusals():
    from paper_1405_6162_gb300 import LBError
    dims = (13, 7, 5)
    n = 455
    phi0 = L.spinodal_phi0(*dims, seed=930, amp=0.5)
    m = _masks(n, phi0, 931)["sparse"]
    with _lat(dims, kernel="taug1") as lat:
        lat.init(phi0)
        lat.step(3)
        full = lat.moments()
        got = lat.moments_masked(m)
        for a, b in zip(got, full):
            assert np.array_equal(a, oracle.select_sites(b, m))
        with pytest.raises(LBError):
            lat.get_state_masked(m)
        with pytest.raises(LBError):
            lat.set_state_masked(m, np.zeros(19 * int((m != 0).sum())), np.zeros(19 * int((m != 0).sum())))


def test_force_enters_masked_velocity():
    dims = (10, 9, 8)
    n = 720
    F = (1e-4, -2e-4, 5e-5)
    with _lat(dims) as lat:
        lat.set_force(*F)
        lat.init(L.spinodal_phi0(*dims, seed=940, amp=0.5))
        lat.step(2)
        m = (L.uniform(941, n, 0, 1) < 0.5).astype(np.uint8)
        assert np.array_equal(lat.moments_masked(m)[1], oracle.select_sites(lat.moments()[1], m))


@pytest.mark.parametrize("precision", ["fp32_shifted", "fp64"])
def test_interface_band_at_256cubed(precision):
    """Full-size lattice after lb_init: the state is the equilibrium of phi0,
    so the masked moments are rho0, 0 and phi0 at the selected sites."""
    import torch
    dims = (256, 256, 256)
    xi = L.interface_width(P0["A"], P0["kappa"])
    phi0 = L.flat_interface_phi0(*dims, amplitude=0.5, xi=xi)
    phi0 = phi0 + 0.01 * L.uniform(950, phi0.size, -1, 1)
    m = (np.abs(phi0) < 0.2).astype(np.uint8)
    with _lat(dims, precision) as lat:
        lat.init(phi0)
        rho, u, phi = lat.moments_masked(torch.from_numpy(m).cuda())
        k = int(m.sum())
        assert rho.shape[0] == k and k > 0
        tol = 1e-15 if precision == "fp64" else 1e-6
        assert (rho - P0["rho0"]).abs().max().item() <= tol * 2
        assert u.abs().max().item() <= tol
        assert np.abs(phi.cpu().numpy() - oracle.select_sites(phi0, m)).max() <= tol


def test_unaligned_device_mask_and_ragged_tail():
    """A device mask that does not start on a 16-byte boundary takes the
    byte-wise path; a lattice whose size is not a multiple of the 4096-site
    tile has a ragged last tile."""
    import torch
    dims = (17, 13, 11)
    n = 2431
    phi0 = L.spinodal_phi0(*dims, seed=960, amp=0.5)
    m = (L.uniform(961, n, 0, 1) < 0.3).astype(np.uint8)
    big = torch.zeros(n + 3, dtype=torch.uint8, device="cuda")
    big[1:n + 1] = torch.from_numpy(m).cuda()
    view = big[1:n + 1]
    assert view.data_ptr() % 16 != 0
    with _lat(dims) as lat:
        lat.init(phi0)
        lat.step(2)
        full = lat.moments()
        got = lat.moments_masked(view)
        assert lat.count_masked(view) == int(m.sum())
        for a, b in zip(got, full):
            assert np.array_equal(a.cpu().numpy(), oracle.select_sites(b, m))
