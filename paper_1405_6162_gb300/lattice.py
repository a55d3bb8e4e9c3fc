"""Python view of one lattice context of liblb.

Argument marshalling only: every step of the method runs in liblb's CUDA
kernels.  Host inputs are numpy float64 arrays (``LB_HOST``); device inputs
are CUDA torch tensors of dtype float64 (``LB_DEVICE``).  PyTorch supplies
the CUDA stream and, through ``lb_set_allocator``, the device memory (its
caching allocator).
"""
from __future__ import annotations

import ctypes
import weakref

import numpy as np

from . import _lib as L

PRECISIONS = {"fp64": L.LB_FP64, "fp32_shifted": L.LB_FP32_SHIFTED, "fp64_df": L.LB_FP64_DF}
KERNELS = {"auto": L.LB_KERNEL_AUTO, "two_pass": L.LB_KERNEL_TWO_PASS, "fused": L.LB_KERNEL_FUSED,
           "staged": L.LB_KERNEL_STAGED, "slab": L.LB_KERNEL_SLAB, "lag": L.LB_KERNEL_LAG,
           "taug1": L.LB_KERNEL_TAUG1, "bulk": L.LB_KERNEL_BULK}

_ALLOC_CB = None
_FREE_CB = None


def _torch():
    import torch
    return torch


def use_torch_allocator(enable: bool = True) -> None:
    """Route liblb's device allocations through torch's caching allocator."""
    global _ALLOC_CB, _FREE_CB
    lib = L.lib()
    if not enable:
        L.check(lib.lb_set_allocator(L.ALLOC_FN(), L.FREE_FN(), None), "lb_set_allocator")
        return
    torch = _torch()

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:  # out of memory: liblb reports LB_ERR_NOMEM
            return None

    def _free(ptr, nbytes, stream, user):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    _ALLOC_CB = L.ALLOC_FN(_alloc)
    _FREE_CB = L.FREE_FN(_free)
    L.check(lib.lb_set_allocator(_ALLOC_CB, _FREE_CB, None), "lb_set_allocator")


def _ptr_of(x, n_expected: int, name: str, writable: bool = False):
    """(pointer, kind, keepalive) of a numpy or CUDA-torch float64 array."""
    if x is None:
        return None, None, None
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags.c_contiguous:
            if writable:
                raise ValueError(f"{name} must be a C-contiguous float64 numpy array")
            x = np.ascontiguousarray(x, dtype=np.float64)
        if x.size != n_expected:
            raise ValueError(f"{name} has {x.size} values, expected {n_expected}")
        return x.ctypes.data, L.LB_HOST, x
    torch = _torch()
    if isinstance(x, torch.Tensor):
        if not x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
        if x.numel() != n_expected:
            raise ValueError(f"{name} has {x.numel()} values, expected {n_expected}")
        return x.data_ptr(), L.LB_DEVICE, x
    raise TypeError(f"{name}: expected numpy.ndarray or torch.Tensor, got {type(x)}")


def _destroy(handle):
    try:
        L.lib().lb_destroy(handle)
    except Exception:
        pass


class Lattice:
    """One periodic D3Q19 binary-fluid lattice held on the GPU.

    Parameters follow ``lb_params`` (include/lb.h): extents nx, ny, nz and
    tau, tau_g, rho0, gamma, A, B, kappa; ``precision`` is "fp64",
    "fp32_shifted" or "fp64_df" (double-float on the FP32 units).
    """

    def __init__(self, nx, ny, nz, *, tau, tau_g, rho0, gamma, A, B, kappa,
                 precision="fp64", stream=None, torch_allocator=True):
        lib = L.lib()
        torch = _torch()
        if torch_allocator and _ALLOC_CB is None:
            use_torch_allocator(True)
        self.dims = (int(nx), int(ny), int(nz))
        self.N = self.dims[0] * self.dims[1] * self.dims[2]
        self.precision = precision
        self.params = dict(tau=tau, tau_g=tau_g, rho0=rho0, gamma=gamma, A=A, B=B, kappa=kappa)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        p = L.lb_params(self.dims[0], self.dims[1], self.dims[2], tau, tau_g, rho0, gamma, A, B, kappa,
                        PRECISIONS[precision])
        h = ctypes.c_void_p()
        L.check(lib.lb_create(ctypes.byref(p), ctypes.c_void_p(sp), ctypes.byref(h)), "lb_create")
        self._h = h
        self._fin = weakref.finalize(self, _destroy, h)

    @classmethod
    def _member(cls, handle, dims, params, precision, owner):
        """A non-owning view of an ensemble member (freed by its ensemble)."""
        self = cls.__new__(cls)
        self.dims = tuple(int(d) for d in dims)
        self.N = self.dims[0] * self.dims[1] * self.dims[2]
        self.precision = precision
        self.params = {k: params[k] for k in ("tau", "tau_g", "rho0", "gamma", "A", "B", "kappa")}
        self.stream = owner.stream
        self._h = ctypes.c_void_p(handle)
        self._owner = owner
        self._fin = weakref.finalize(self, lambda: None)
        return self

    @classmethod
    def from_params(cls, dims, params, **kw):
        return cls(*dims, **{k: params[k] for k in ("tau", "tau_g", "rho0", "gamma", "A", "B", "kappa")}, **kw)

    # -------------------------------------------------------------- lifecycle
    def close(self):
        if self._fin.alive:
            self._fin()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        if not self._fin.alive:
            raise RuntimeError("lattice is closed")
        return self._h

    # -------------------------------------------------------------- calls
    def init(self, phi0, u0=None):
        pp, kind, k1 = _ptr_of(phi0, self.N, "phi0")
        up, ukind, k2 = _ptr_of(u0, 3 * self.N, "u0")
        if u0 is not None and ukind != kind:
            raise ValueError("phi0 and u0 must both be host or both be device arrays")
        L.check(L.lib().lb_init(self.handle, pp, up, kind), "lb_init")

    def step(self, nsteps: int = 1):
        L.check(L.lib().lb_step(self.handle, int(nsteps)), "lb_step")

    def set_kernel(self, kernel="auto", block_x=0, block_y=0, z_chunk=0):
        L.check(L.lib().lb_set_kernel(self.handle, KERNELS[kernel], block_x, block_y, z_chunk),
                "lb_set_kernel")

    def set_stencil(self, points: int = 7):
        """Points of the phi stencils: 7 (nearest faces), 19 or 27 (isotropic)."""
        L.check(L.lib().lb_set_stencil(self.handle, int(points)), "lb_set_stencil")

    def set_collision(self, model: str = "bgk", tau_bulk: float = 1.0, tau_ghost: float = 1.0):
        """Collision of f: "bgk", or "mrt" with the bulk and ghost relaxation
        times (shear: the lattice's tau)."""
        code = {"bgk": L.LB_COLLISION_BGK, "mrt": L.LB_COLLISION_MRT}[model]
        L.check(L.lib().lb_set_collision(self.handle, code, float(tau_bulk), float(tau_ghost)),
                "lb_set_collision")

    def set_force(self, fx: float = 0.0, fy: float = 0.0, fz: float = 0.0):
        """Uniform body force density (Guo's scheme); zero switches it off."""
        L.check(L.lib().lb_set_force(self.handle, float(fx), float(fy), float(fz)), "lb_set_force")

    def sync(self):
        """Wait for queued work; raises LBError(LB_ERR_TIMEOUT) if a bounded
        device-side wait gave up."""
        L.check(L.lib().lb_sync(self.handle), "lb_sync")

    def set_wait_timeout(self, seconds: float):
        L.check(L.lib().lb_set_wait_timeout(self.handle, int(seconds * 1e9)), "lb_set_wait_timeout")

    def moments(self, device: bool = False):
        """(rho [N], u [3,N], phi [N]) as numpy (host) or CUDA torch tensors."""
        n = self.N
        if device:
            torch = _torch()
            rho = torch.empty(n, dtype=torch.float64, device="cuda")
            u = torch.empty(3 * n, dtype=torch.float64, device="cuda")
            phi = torch.empty(n, dtype=torch.float64, device="cuda")
            L.check(L.lib().lb_moments(self.handle, rho.data_ptr(), u.data_ptr(), phi.data_ptr(),
                                       L.LB_DEVICE), "lb_moments")
            return rho, u.view(3, n), phi
        rho = np.empty(n)
        u = np.empty(3 * n)
        phi = np.empty(n)
        L.check(L.lib().lb_moments(self.handle, rho.ctypes.data, u.ctypes.data, phi.ctypes.data,
                                   L.LB_HOST), "lb_moments")
        return rho, u.reshape(3, n), phi

    def reduce(self):
        """[sum rho, sum rho u (3), sum phi] (FP64 sums on the GPU)."""
        out = np.zeros(5)
        L.check(L.lib().lb_reduce(self.handle, out.ctypes.data), "lb_reduce")
        return out

    def get_state(self, device: bool = False):
        """(f [19,N], g [19,N]) post-streaming distributions, ABI velocity order."""
        n = self.N
        if device:
            torch = _torch()
            f = torch.empty(19 * n, dtype=torch.float64, device="cuda")
            g = torch.empty(19 * n, dtype=torch.float64, device="cuda")
            L.check(L.lib().lb_get_state(self.handle, f.data_ptr(), g.data_ptr(), L.LB_DEVICE),
                    "lb_get_state")
            return f.view(19, n), g.view(19, n)
        f = np.empty(19 * n)
        g = np.empty(19 * n)
        L.check(L.lib().lb_get_state(self.handle, f.ctypes.data, g.ctypes.data, L.LB_HOST), "lb_get_state")
        return f.reshape(19, n), g.reshape(19, n)

    def set_state(self, f, g):
        fp, fk, k1 = _ptr_of(f, 19 * self.N, "f")
        gp, gk, k2 = _ptr_of(g, 19 * self.N, "g")
        if fk != gk:
            raise ValueError("f and g must both be host or both be device arrays")
        L.check(L.lib().lb_set_state(self.handle, fp, gp, fk), "lb_set_state")

    # -------------------------------------------------------------- masked copies
    def _mask(self, mask):
        """(pointer, kind, keepalive) of a uint8 mask of N sites: numpy (host)
        or a CUDA torch tensor (device)."""
        if isinstance(mask, np.ndarray):
            m = np.ascontiguousarray(mask.reshape(-1), dtype=np.uint8)
            if m.size != self.N:
                raise ValueError(f"mask has {m.size} sites, the lattice {self.N}")
            return m.ctypes.data, L.LB_HOST, m
        torch = _torch()
        if torch.is_tensor(mask) and mask.is_cuda:
            m = mask.reshape(-1).to(torch.uint8).contiguous()
            if m.numel() != self.N:
                raise ValueError(f"mask has {m.numel()} sites, the lattice {self.N}")
            return m.data_ptr(), L.LB_DEVICE, m
        raise TypeError("mask must be a numpy array or a CUDA torch tensor")

    def count_masked(self, mask) -> int:
        """Number of sites whose mask byte is non-zero."""
        mp, kind, keep = self._mask(mask)
        cnt = ctypes.c_longlong(0)
        L.check(L.lib().lb_moments_masked(self.handle, mp, None, None, None, ctypes.byref(cnt), kind),
                "lb_moments_masked")
        return int(cnt.value)

    def moments_masked(self, mask):
        """(rho [k], u [3,k], phi [k]) of the k selected sites in site order;
        numpy for a numpy mask, CUDA tensors for a CUDA mask."""
        mp, kind, keep = self._mask(mask)
        k = self.count_masked(mask)
        cnt = ctypes.c_longlong(0)
        if kind == L.LB_DEVICE:
            torch = _torch()
            rho, u, phi = (torch.empty(m * max(k, 1), dtype=torch.float64, device="cuda") for m in (1, 3, 1))
            L.check(L.lib().lb_moments_masked(self.handle, mp, rho.data_ptr(), u.data_ptr(), phi.data_ptr(),
                                              ctypes.byref(cnt), kind), "lb_moments_masked")
            return rho[:k], u[:3 * k].view(3, k), phi[:k]
        rho, u, phi = np.empty(max(k, 1)), np.empty(3 * max(k, 1)), np.empty(max(k, 1))
        L.check(L.lib().lb_moments_masked(self.handle, mp, rho.ctypes.data, u.ctypes.data, phi.ctypes.data,
                                          ctypes.byref(cnt), kind), "lb_moments_masked")
        return rho[:k], u[:3 * k].reshape(3, k), phi[:k]

    def get_state_masked(self, mask):
        """(f [19,k], g [19,k]) post-streaming distributions of the k selected
        sites in site order."""
        mp, kind, keep = self._mask(mask)
        k = self.count_masked(mask)
        cnt = ctypes.c_longlong(0)
        if kind == L.LB_DEVICE:
            torch = _torch()
            f = torch.empty(19 * max(k, 1), dtype=torch.float64, device="cuda")
            g = torch.empty_like(f)
            L.check(L.lib().lb_get_state_masked(self.handle, mp, f.data_ptr(), g.data_ptr(), ctypes.byref(cnt),
                                                kind), "lb_get_state_masked")
            return f[:19 * k].view(19, k), g[:19 * k].view(19, k)
        f, g = np.empty(19 * max(k, 1)), np.empty(19 * max(k, 1))
        L.check(L.lib().lb_get_state_masked(self.handle, mp, f.ctypes.data, g.ctypes.data, ctypes.byref(cnt),
                                            kind), "lb_get_state_masked")
        return f[:19 * k].reshape(19, k), g[:19 * k].reshape(19, k)

    def set_state_masked(self, mask, f, g):
        """Overwrite the post-streaming f, g ([19,k] each) of the k selected
        sites."""
        mp, kind, keep = self._mask(mask)
        k = self.count_masked(mask)
        fp, fk, k1 = _ptr_of(f, 19 * k, "f")
        gp, gk, k2 = _ptr_of(g, 19 * k, "g")
        if fk != kind or gk != kind:
            raise ValueError("mask, f and g must all be host or all be device arrays")
        L.check(L.lib().lb_set_state_masked(self.handle, mp, fp, gp, kind), "lb_set_state_masked")


# ABI velocity order (include/lb.h)
VELOCITIES = np.array([
    [0, 0, 0],
    [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
    [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0],
    [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1],
    [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]])
