"""Device-allocation failure, injected on the host.

The paper's memory calls come "with error checking" (targetMalloc,
Sec. III.B); here every device allocation of liblb goes through the
allocator installed with lb_set_allocator.  The tests install one that
fails on its k-th call, for every k an entry point reaches, and check that
the call returns LB_ERR_NOMEM, that everything it did allocate was handed
back (nothing leaked, by the allocator's own books and by torch's), and that
the process carries on normally afterwards.  No GPU fault is involved: the
failure is a NULL returned by a host callback.
"""
import ctypes

import numpy as np
import pytest

import lb_inputs as L
import oracle
from tests.parity import P0, TOL_FP64, rel

pytestmark = pytest.mark.gpu


class InjectingAllocator:
    """Allocates through torch's caching allocator and returns NULL on its
    ``fail_at``-th call (1-based; 0 = never); records what is live."""

    def __init__(self, fail_at=0):
        import torch
        from paper_1405_6162_gb300 import _lib as LL
        self.torch = torch
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}
        self.cb_alloc = LL.ALLOC_FN(self._alloc)
        self.cb_free = LL.FREE_FN(self._free)

    def _alloc(self, nbytes, stream, user):
        self.calls += 1
        if self.calls == self.fail_at:
            return None
        p = self.torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        self.live[p] = int(nbytes)
        return p

    def _free(self, ptr, nbytes, stream, user):
        assert self.live.pop(int(ptr)) == int(nbytes)
        self.torch.cuda.caching_allocator_delete(int(ptr))

    def install(self):
        from paper_1405_6162_gb300 import _lib as LL
        LL.check(LL.lib().lb_set_allocator(self.cb_alloc, self.cb_free, None), "lb_set_allocator")
        return self


@pytest.fixture()
def lib():
    import paper_1405_6162_gb300 as lbpkg
    from paper_1405_6162_gb300 import _lib as LL
    from paper_1405_6162_gb300.lattice import use_torch_allocator
    lbpkg.build()
    oracle.build()
    yield LL.lib()
    use_torch_allocator(True)          # later contexts allocate through torch again


def _params(dims, precision=0, **kw):
    from paper_1405_6162_gb300 import _lib as LL
    p = dict(P0, **kw)
    return LL.lb_params(*dims, p["tau"], p["tau_g"], p["rho0"], p["gamma"], p["A"], p["B"], p["kappa"], precision)


def _count_calls(lib, fn):
    """Allocator calls made by fn() with an allocator that never fails."""
    a = InjectingAllocator().install()
    fn(a)
    return a.calls


def _usable_afterwards():
    """A fresh lattice still steps and matches the oracle."""
    from paper_1405_6162_gb300 import Lattice
    from paper_1405_6162_gb300.lattice import use_torch_allocator
    use_torch_allocator(True)
    dims = (8, 6, 5)
    phi0 = L.spinodal_phi0(*dims, seed=3, amp=0.3)
    fo, go = oracle.step(dims, P0, *oracle.init(dims, P0, phi0), 3)
    want = oracle.moments(dims, fo, go)
    with Lattice.from_params(dims, P0, precision="fp64") as lat:
        lat.init(phi0)
        lat.step(3)
        got = lat.moments()
    assert rel(got[2], want[2]) <= TOL_FP64


@pytest.mark.parametrize("precision", [0, 1])
def test_create_fails_cleanly_at_every_allocation(lib, precision):
    import torch
    from paper_1405_6162_gb300 import _lib as LL
    dims = (10, 8, 6)
    prm = _params(dims, precision)

    def create(a):
        h = ctypes.c_void_p()
        rc = lib.lb_create(ctypes.byref(prm), None, ctypes.byref(h))
        if rc == LL.LB_OK:
            lib.lb_destroy(h)
        return rc, h

    n = _count_calls(lib, create)
    assert n >= 9                     # f, g (two levels), phi, reduction scratch, counters, error flag
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    for k in range(1, n + 1):
        a = InjectingAllocator(fail_at=k).install()
        rc, h = create(a)
        assert rc == LL.LB_ERR_NOMEM and not h.value, (k, rc)
        assert a.live == {}, (k, a.live)
        assert torch.cuda.memory_allocated() == base, k
    _usable_afterwards()


def test_ensemble_create_fails_cleanly_at_every_allocation(lib):
    import torch
    from paper_1405_6162_gb300 import _lib as LL
    specs = L.ensemble(21, 3, lo=4, hi=9)
    arr = (LL.lb_params * 3)(*[_params((d["nx"], d["ny"], d["nz"]), 1, tau=d["tau"], kappa=d["kappa"])
                               for d in specs])

    def create(a):
        h = ctypes.c_void_p()
        rc = lib.lb_batch_create(3, arr, None, ctypes.byref(h))
        if rc == LL.LB_OK:
            lib.lb_batch_destroy(h)
        return rc, h

    n = _count_calls(lib, create)
    assert n >= 27
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    for k in range(1, n + 1):
        a = InjectingAllocator(fail_at=k).install()
        rc, h = create(a)
        assert rc == LL.LB_ERR_NOMEM and not h.value, (k, rc)
        assert a.live == {}, (k, a.live)
        assert torch.cuda.memory_allocated() == base, k
    _usable_afterwards()


def test_lazy_scratch_fails_cleanly(lib):
    """The scratch allocated on first use -- the adjoint's (two buffers), the
    host-transfer staging buffer, the masked copies' compaction buffers --
    reports LB_ERR_NOMEM, keeps nothing of a half-done allocation, and the
    same call succeeds once the allocator does."""
    import torch
    from paper_1405_6162_gb300 import _lib as LL
    dims = (10, 8, 6)
    n = 480
    prm = _params(dims, 0)
    dev = dict(dtype=torch.float64, device="cuda")
    phi0 = torch.from_numpy(L.spinodal_phi0(*dims, seed=4, amp=0.3)).cuda()
    f = torch.empty(19 * n, **dev)
    g = torch.empty(19 * n, **dev)
    a_in = [torch.from_numpy(L.uniform(5 + i, 19 * n, -1, 1)).cuda() for i in range(2)]
    a_out = [torch.empty(19 * n, **dev) for _ in range(2)]
    dk = torch.zeros(1, **dev)
    host = np.empty(n)
    mask = np.zeros(n, dtype=np.uint8)
    mask[::7] = 1
    cnt = ctypes.c_longlong()

    calls = {
        "adjoint": lambda h: lib.lb_adjoint_step(h, f.data_ptr(), g.data_ptr(), a_in[0].data_ptr(),
                                                 a_in[1].data_ptr(), a_out[0].data_ptr(), a_out[1].data_ptr(),
                                                 dk.data_ptr()),
        "io": lambda h: lib.lb_moments(h, None, None, host.ctypes.data, LL.LB_HOST),
        "masked": lambda h: lib.lb_moments_masked(h, mask.ctypes.data, None, None, None, ctypes.byref(cnt),
                                                  LL.LB_HOST),
    }
    for name, call in calls.items():
        # allocations made by lb_create, then by the call's first use
        a = InjectingAllocator().install()
        h = ctypes.c_void_p()
        LL.check(lib.lb_create(ctypes.byref(prm), None, ctypes.byref(h)), "lb_create")
        n_create = a.calls
        LL.check(lib.lb_init(h, phi0.data_ptr(), None, LL.LB_DEVICE), "lb_init")
        LL.check(lib.lb_get_state(h, f.data_ptr(), g.data_ptr(), LL.LB_DEVICE), "lb_get_state")
        LL.check(call(h), name)
        n_lazy = a.calls - n_create
        lib.lb_destroy(h)
        assert a.live == {}
        assert n_lazy >= 1, name
        for k in range(1, n_lazy + 1):
            a = InjectingAllocator(fail_at=n_create + k).install()
            h = ctypes.c_void_p()
            LL.check(lib.lb_create(ctypes.byref(prm), None, ctypes.byref(h)), "lb_create")
            LL.check(lib.lb_init(h, phi0.data_ptr(), None, LL.LB_DEVICE), "lb_init")
            live0 = dict(a.live)
            torch.cuda.synchronize()
            assert call(h) == LL.LB_ERR_NOMEM, (name, k)
            assert a.live == live0, (name, k)           # nothing of the failed allocation kept
            assert call(h) == LL.LB_OK, (name, k)       # the allocator succeeds again: so does the call
            torch.cuda.synchronize()
            lib.lb_destroy(h)
            assert a.live == {}, (name, k)
    _usable_afterwards()
