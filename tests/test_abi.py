"""liblb loads and exports every entry point of include/lb.h; host-side
argument validation (no GPU needed: every check below returns before any
CUDA call)."""
import ctypes
import os
import re

import pytest

import paper_1405_6162_gb300 as lbpkg
from paper_1405_6162_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    lbpkg.build()
    return L.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "lb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(L.SIGNATURES)


def test_strerror(lib):
    for code in (0, -1, -2, -3, -4, -5):
        assert lib.lb_strerror(code)
    assert lib.lb_strerror(-99) == b"unknown error code"


def _params(**kw):
    d = dict(nx=8, ny=8, nz=8, tau=1.0, tau_g=1.0, rho0=1.0, gamma=0.5, A=-0.0625, B=0.0625,
             kappa=0.04, precision=0)
    d.update(kw)
    return L.lb_params(*[d[k] for k in ("nx", "ny", "nz", "tau", "tau_g", "rho0", "gamma", "A", "B",
                                        "kappa", "precision")])


@pytest.mark.parametrize("bad", [dict(nx=0), dict(ny=-1), dict(tau=0.5), dict(tau_g=0.2),
                                 dict(rho0=0.0), dict(precision=7), dict(kappa=float("nan")),
                                 dict(nx=2048, ny=2048, nz=1024)])
def test_create_rejects_invalid_params(lib, bad):
    h = ctypes.c_void_p()
    rc = lib.lb_create(ctypes.byref(_params(**bad)), None, ctypes.byref(h))
    assert rc == L.LB_ERR_INVALID and not h.value


def test_null_arguments(lib):
    assert lib.lb_create(None, None, None) == L.LB_ERR_INVALID
    assert lib.lb_step(None, 1) == L.LB_ERR_INVALID
    assert lib.lb_init(None, None, None, 0) == L.LB_ERR_INVALID
    assert lib.lb_moments(None, None, None, None, 0) == L.LB_ERR_INVALID
    assert lib.lb_reduce(None, None) == L.LB_ERR_INVALID
    assert lib.lb_set_kernel(None, 0, 0, 0, 0) == L.LB_ERR_INVALID
    assert lib.lb_set_stencil(None, 19) == L.LB_ERR_INVALID
    assert lib.lb_set_collision(None, L.LB_COLLISION_MRT, 1.0, 1.0) == L.LB_ERR_INVALID
    assert lib.lb_set_force(None, 0.0, 0.0, 1e-5) == L.LB_ERR_INVALID
    lib.lb_destroy(None)


def test_allocator_pair_must_match(lib):
    f = L.FREE_FN(lambda *a: None)
    assert lib.lb_set_allocator(L.ALLOC_FN(), f, None) == L.LB_ERR_INVALID
    assert lib.lb_set_allocator(L.ALLOC_FN(), L.FREE_FN(), None) == L.LB_OK


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(L, "_LIB", None)
    monkeypatch.setattr(L._build, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        L.lib()
