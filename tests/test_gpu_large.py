"""A lattice past 2^27 sites: FP32-shifted at 1024 x 1024 x 192 (201 M
sites, 61 GB of distributions).  Row offsets i*S of the SoA components reach
3.6e9 elements, past 2^31, so any 32-bit index arithmetic would show.

One step of a site depends only on its 5^3 neighbourhood, so sampled sites
(their neighbourhoods read back through the masked state copy, which is
bit-exact against the full copy) are compared with the oracle run on that
neighbourhood; the samples include the last site and sites in the last z
planes, where the offsets are largest.  The tau_g = 1 reduced form is then
compared with the default step on the same sites through the masked
moments."""
import numpy as np
import pytest

import lb_inputs as L
import oracle
from tests.parity import P0, abi_order

pytestmark = pytest.mark.gpu

DIMS = (1024, 1024, 192)


@pytest.fixture(scope="module", autouse=True)
def _setup():
    import paper_1405_6162_gb300 as lbpkg
    lbpkg.build()
    oracle.build()


def _samples():
    nx, ny, nz = DIMS
    n = nx * ny * nz
    sites = [int(s) for s in L.uniform_int(96, 12, 0, n - 1)]
    sites += [n - 1, n - nx * ny // 2 - 7, n - 3 * nx * ny + 5, n // 2, 0]
    off = np.arange(-2, 3)
    oz, oy, ox = np.meshgrid(off, off, off, indexing="ij")
    boxes = []
    for s in sites:
        x, y, z = s % nx, (s // nx) % ny, s // (nx * ny)
        boxes.append(((x + ox) % nx + nx * (((y + oy) % ny) + ny * ((z + oz) % nz))).reshape(-1))
    mask = np.zeros(n, dtype=np.uint8)
    for b in boxes:
        mask[b] = 1
    return sites, boxes, mask


def test_large_lattice_sampled_sites_and_reduced_form():
    from paper_1405_6162_gb300 import Lattice
    sites, boxes, mask = _samples()
    sel = np.flatnonzero(mask)            # site order of the masked copies
    centre = 2 + 5 * (2 + 5 * 2)
    o2a = abi_order()
    # a seeded random x-y plane, rolled differently in every z plane (every
    # plane distinct; the full-size generator would take half a minute)
    nx, ny, nz = DIMS
    plane = L.spinodal_phi0(nx, ny, 1, seed=95, amp=0.8).reshape(ny, nx)
    phi0 = np.stack([np.roll(plane, (7 * z, 13 * z), axis=(0, 1)) for z in range(nz)]).reshape(-1)
    with Lattice.from_params(DIMS, P0, precision="fp32_shifted") as lat:
        lat.init(phi0)
        lat.step(3)
        f0, g0 = lat.get_state_masked(mask)
        lat.step(1)
        f1, g1 = lat.get_state_masked(mask)
        m_general = lat.moments_masked(mask)
    for s, box in zip(sites, boxes):
        k = np.searchsorted(sel, box)
        fo, go = oracle.step((5, 5, 5), P0, f0[:, k][o2a], g0[:, k][o2a], 1)
        kc = int(np.searchsorted(sel, s))
        assert np.abs(f1[:, kc][o2a] - fo[:, centre]).max() <= 2e-8, s
        assert np.abs(g1[:, kc][o2a] - go[:, centre]).max() <= 2e-7, s
    with Lattice.from_params(DIMS, P0, precision="fp32_shifted") as lat:
        lat.set_kernel("taug1")
        lat.init(phi0)
        lat.step(4)
        m_reduced = lat.moments_masked(mask)
    # the two forms differ by float rounding only: bounds of a few ulp of the
    # O(1) rho, the O(0.1) summands of u and the O(1) phi over four steps
    for name, a, b, tol in zip(("rho", "u", "phi"), m_reduced, m_general, (1e-6, 1e-7, 1e-6)):
        assert np.abs(a - b).max() <= tol, name
