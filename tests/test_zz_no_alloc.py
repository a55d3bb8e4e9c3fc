"""The allocation-free FP64 timestep (lb_step_fp64_noalloc).

It exists for callers that cannot allocate device memory -- an application
whose device memory is all reserved by its own allocator, or a
latency-critical loop that must not enter cudaMalloc/cudaFree -- and keeps
the one scratch array it needs (phi between the two passes) in a fixed
device array inside the library.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import lb_inputs as L
from tests.parity import P0, TOL_FP64, nonequilibrium_state, rel, to_abi

pytestmark = pytest.mark.gpu

DIMS = (20, 12, 9)


def _roll(a, sign):
    """Shift each velocity row of an ABI-order [19][N] state by sign * c_i."""
    from paper_1405_6162_gb300 import VELOCITIES
    nx, ny, nz = DIMS
    a3 = a.reshape(19, nz, ny, nx)
    out = np.empty_like(a3)
    for i, c in enumerate(VELOCITIES):
        out[i] = np.roll(a3[i], shift=(sign * c[2], sign * c[1], sign * c[0]), axis=(0, 1, 2))
    return out.reshape(19, -1)


def _params():
    from paper_1405_6162_gb300 import _lib as LL
    p = dict(P0, tau=0.8, tau_g=0.9)
    return LL.lb_params(*DIMS, p["tau"], p["tau_g"], p["rho0"], p["gamma"], p["A"], p["B"], p["kappa"],
                        LL.LB_FP64), p


def test_noalloc_step_matches_lb_step_on_two_calls_in_a_row():
    import torch
    import paper_1405_6162_gb300 as lbpkg
    from paper_1405_6162_gb300 import Lattice
    from paper_1405_6162_gb300 import _lib as LL
    lbpkg.build()
    lib = LL.lib()
    prm, p = _params()
    f0, g0 = nonequilibrium_state(DIMS, p, seed=123)
    stream = torch.cuda.current_stream()
    with Lattice.from_params(DIMS, p, precision="fp64") as lat:
        lat.set_kernel("two_pass")
        lat.set_state(to_abi(f0), to_abi(g0))
        f, g = lat.get_state()
        # the entry point takes the post-collision convention: a_i(y) = f_i(y + c_i)
        fa = torch.from_numpy(np.ascontiguousarray(_roll(f, -1))).cuda()
        ga = torch.from_numpy(np.ascontiguousarray(_roll(g, -1))).cuda()
        for call in range(2):
            fb = torch.empty_like(fa)
            gb = torch.empty_like(ga)
            rc = lib.lb_step_fp64_noalloc(ctypes.byref(prm), fa.data_ptr(), ga.data_ptr(), fb.data_ptr(),
                                          gb.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
            assert rc == LL.LB_OK, lib.lb_strerror(rc)
            torch.cuda.synchronize()
            lat.step(1)
            f_ref, g_ref = lat.get_state()
            f_new = _roll(fb.cpu().numpy().reshape(19, -1), +1)
            g_new = _roll(gb.cpu().numpy().reshape(19, -1), +1)
            assert rel(f_new, f_ref) <= TOL_FP64, (call, rel(f_new, f_ref))
            assert rel(g_new, g_ref) <= TOL_FP64, (call, rel(g_new, g_ref))
            fa, ga = fb, gb


def test_noalloc_step_matches_the_oracle_and_allocates_nothing():
    """Two calls in a row against the FP64 oracle (an implementation that
    shares nothing with the library), and the device's free memory unchanged
    by calls made after the first one's set-up."""
    import torch
    import oracle
    import paper_1405_6162_gb300 as lbpkg
    from paper_1405_6162_gb300 import _lib as LL
    from tests.parity import to_oracle
    lbpkg.build()
    oracle.build()
    lib = LL.lib()
    prm, p = _params()
    f0, g0 = nonequilibrium_state(DIMS, p, seed=321)          # post-streaming state, oracle order
    fo, go = oracle.step(DIMS, p, f0, g0, 2)
    stream = torch.cuda.current_stream()
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    bufs = [cu(_roll(to_abi(f0), -1)), cu(_roll(to_abi(g0), -1))]
    bufs += [torch.empty_like(bufs[0]) for _ in range(4)]
    torch.cuda.synchronize()

    def call(src, dst):
        rc = lib.lb_step_fp64_noalloc(ctypes.byref(prm), bufs[src].data_ptr(), bufs[src + 1].data_ptr(),
                                      bufs[dst].data_ptr(), bufs[dst + 1].data_ptr(),
                                      ctypes.c_void_p(stream.cuda_stream))
        assert rc == LL.LB_OK, lib.lb_strerror(rc)

    call(0, 2)                                                # first call: set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    call(2, 4)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    f2 = to_oracle(_roll(bufs[4].cpu().numpy().reshape(19, -1), +1))
    g2 = to_oracle(_roll(bufs[5].cpu().numpy().reshape(19, -1), +1))
    assert rel(f2, fo) <= TOL_FP64, rel(f2, fo)
    assert rel(g2, go) <= TOL_FP64, rel(g2, go)


def test_noalloc_rejects_overlapping_outputs():
    """Outputs that share any byte with each other or with an input are
    refused before anything runs (the pointers below are never
    dereferenced)."""
    import paper_1405_6162_gb300 as lbpkg
    from paper_1405_6162_gb300 import _lib as LL
    lbpkg.build()
    lib = LL.lib()
    prm, _ = _params()
    nb = 19 * DIMS[0] * DIMS[1] * DIMS[2] * 8
    base = 1 << 30
    fa, ga, fb, gb = base, base + 2 * nb, base + 4 * nb, base + 6 * nb
    for args in ((fa, ga, fb, fb), (fa, ga, fb, fb + 8), (fa, ga, fa + nb - 8, gb), (fa, ga, fb, ga + 16),
                 (fa, ga, gb - nb + 8, gb), (fa, ga, fa, gb)):
        rc = lib.lb_step_fp64_noalloc(ctypes.byref(prm), *[ctypes.c_void_p(a) for a in args], None)
        assert rc == LL.LB_ERR_INVALID, args


def test_noalloc_rejects_lattices_beyond_its_scratch():
    import paper_1405_6162_gb300 as lbpkg
    from paper_1405_6162_gb300 import _lib as LL
    lbpkg.build()
    lib = LL.lib()
    prm, _ = _params()
    prm.nx, prm.ny, prm.nz = 65, 64, 64          # 266240 sites > 262144
    dummy = ctypes.c_void_p(1 << 20)              # never dereferenced: rejected first
    rc = lib.lb_step_fp64_noalloc(ctypes.byref(prm), dummy, dummy, ctypes.c_void_p(2 << 20),
                                  ctypes.c_void_p(3 << 20), None)
    assert rc == LL.LB_ERR_INVALID
    prm.nx, prm.ny, prm.nz = 8, 8, 8
    prm.precision = LL.LB_FP32_SHIFTED
    assert lib.lb_step_fp64_noalloc(ctypes.byref(prm), dummy, dummy, ctypes.c_void_p(2 << 20),
                                    ctypes.c_void_p(3 << 20), None) == LL.LB_ERR_INVALID
