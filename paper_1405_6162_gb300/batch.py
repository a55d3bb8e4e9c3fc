"""Python view of an ensemble (lb_batch): many lattices, one persistent
launch per run.  Argument marshalling only."""
from __future__ import annotations

import ctypes
import weakref

from . import _lib as L
from .lattice import PRECISIONS, Lattice, _torch, use_torch_allocator
from . import lattice as _lattice


def plan(items, ctas, bins=0):
    """The ensemble's CTA plan for lattices with ``items[k]`` work items per
    pass over ``ctas`` co-resident CTAs and ``bins`` (0: a group per lattice;
    k: k groups of whole lattices), lb_batch_plan (host only, no GPU).
    Returns (group of every lattice, [(first CTA, CTA count)] per group)."""
    n = len(items)
    it = (ctypes.c_longlong * max(n, 1))(*[int(x) for x in items])
    ng_max = max(min(n, int(ctas)), 1)
    group = (ctypes.c_int * max(n, 1))()
    cta0 = (ctypes.c_int * ng_max)()
    m = (ctypes.c_int * ng_max)()
    ng = ctypes.c_int()
    L.check(L.lib().lb_batch_plan(n, it, int(ctas), int(bins), group, cta0, m, ctypes.byref(ng)), "lb_batch_plan")
    return list(group[:n]), [(cta0[g], m[g]) for g in range(ng.value)]


def _destroy(handle):
    try:
        L.lib().lb_batch_destroy(handle)
    except Exception:
        pass


class Batch:
    """Ensemble of independent periodic lattices.

    ``lattices`` is a list of dicts with keys nx, ny, nz, tau, tau_g, rho0,
    gamma, A, B, kappa (e.g. ``lb_inputs.ensemble``); one ``precision`` for
    all.  ``batch[k]`` is lattice k as a :class:`Lattice` view (init,
    moments, reduce, get_state, set_state).
    """

    def __init__(self, lattices, precision="fp32_shifted", stream=None, torch_allocator=True):
        lib = L.lib()
        torch = _torch()
        if torch_allocator and _lattice._ALLOC_CB is None:
            use_torch_allocator(True)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        sp = self.stream.cuda_stream if hasattr(self.stream, "cuda_stream") else int(self.stream)
        self.specs = [dict(d) for d in lattices]
        self.precision = precision
        self.form = "general"
        self.plan = "lattice"
        arr = (L.lb_params * len(self.specs))()
        for k, d in enumerate(self.specs):
            arr[k] = L.lb_params(d["nx"], d["ny"], d["nz"], d["tau"], d["tau_g"], d["rho0"], d["gamma"],
                                 d["A"], d["B"], d["kappa"], PRECISIONS[precision])
        h = ctypes.c_void_p()
        L.check(lib.lb_batch_create(len(self.specs), arr, ctypes.c_void_p(sp), ctypes.byref(h)), "lb_batch_create")
        self._h = h
        self._fin = weakref.finalize(self, _destroy, h)
        self._views = {}

    def __len__(self):
        return len(self.specs)

    def __getitem__(self, k) -> Lattice:
        if k not in self._views:
            h = L.lib().lb_batch_lattice(self.handle, int(k))
            if not h:
                raise IndexError(k)
            d = self.specs[k]
            self._views[k] = Lattice._member(h, (d["nx"], d["ny"], d["nz"]), d, self.precision, self)
        return self._views[k]

    @property
    def handle(self):
        if not self._fin.alive:
            raise RuntimeError("ensemble is closed")
        return self._h

    @property
    def sites(self) -> int:
        return sum(d["nx"] * d["ny"] * d["nz"] for d in self.specs)

    def run(self, nsteps: int):
        L.check(L.lib().lb_batch_run(self.handle, int(nsteps)), "lb_batch_run")

    def sync(self):
        L.check(L.lib().lb_batch_sync(self.handle), "lb_batch_sync")

    def set_form(self, form: str = "general"):
        """"general" two-pass step or the tau_g = 1 "taug1" reduced form."""
        L.check(L.lib().lb_batch_set_form(self.handle, {"general": 0, "taug1": 1}[form]), "lb_batch_set_form")
        self.form = form

    def set_launch(self, threads: int = 256, ctas_per_sm: int = 0):
        L.check(L.lib().lb_batch_set_launch(self.handle, int(threads), int(ctas_per_sm)), "lb_batch_set_launch")

    def set_wait_timeout(self, seconds: float):
        L.check(L.lib().lb_batch_set_wait_timeout(self.handle, int(seconds * 1e9)), "lb_batch_set_wait_timeout")

    def info(self):
        """(lattices, work items per pass, CTAs in the grid, threads per CTA)."""
        v = [ctypes.c_int() for _ in range(4)]
        L.check(L.lib().lb_batch_size(self.handle, *[ctypes.byref(x) for x in v]), "lb_batch_size")
        return tuple(x.value for x in v)

    def set_plan(self, plan="lattice"):
        """"lattice": a group of CTAs per lattice (default); "grid": one group
        of all CTAs with a grid-wide barrier between the passes; an int k >= 2:
        k groups of whole lattices balanced by work (see :func:`plan`)."""
        bins = {"lattice": 0, "grid": 1}.get(plan, plan)
        L.check(L.lib().lb_batch_set_plan(self.handle, int(bins)), "lb_batch_set_plan")
        self.plan = plan

    def groups(self) -> int:
        """Number of CTA groups in the current plan (see :func:`plan`)."""
        v = ctypes.c_int()
        L.check(L.lib().lb_batch_groups(self.handle, ctypes.byref(v)), "lb_batch_groups")
        return v.value

    def close(self):
        self._views.clear()
        if self._fin.alive:
            self._fin()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
