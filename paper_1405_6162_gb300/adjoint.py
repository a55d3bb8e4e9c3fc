"""Gradients through the FP64 timestep: a torch.autograd.Function.

``trajectory(phi0, kappa, dims, params, nsteps)`` returns phi at time T
(from the equilibrium start with order parameter phi0) and back-propagates
to phi0 and kappa.  The forward keeps the state every ``segment`` steps
(default ~sqrt(T) -- square-root checkpointing); the backward, segment by
segment from the last, restores the checkpoint, recomputes and keeps that
segment's states, then sweeps them in reverse with liblb's adjoint kernel
pair (``lb_adjoint_step``, started from ``lb_adjoint_seed``, the transpose
of phi_T = sum_i g_i) and finally the initialisation's reverse
(``lb_adjoint_init``).  Memory: about 2 sqrt(T) states of 38 N doubles.
Argument marshalling only: all arithmetic is in liblb's kernels.
"""
from __future__ import annotations

import math

import torch

from . import _lib as L
from .lattice import Lattice


def _p(t):
    return t.data_ptr()


class LBTrajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi0, kappa, dims, params, nsteps, segment):
        p = dict(params)
        p["kappa"] = float(kappa)
        lat = Lattice.from_params(dims, p, precision="fp64")
        phi0 = phi0.detach().to(device="cuda", dtype=torch.float64).contiguous()
        lat.init(phi0)
        seg = int(segment) if segment else max(1, int(round(math.sqrt(nsteps))))
        ckpts = {}
        t = 0
        while t < nsteps:
            ckpts[t] = lat.get_state(device=True)
            n = min(seg, nsteps - t)
            lat.step(n)
            t += n
        _, _, phi_t = lat.moments(device=True)
        ctx.lat, ctx.ckpts, ctx.nsteps, ctx.seg, ctx.phi0 = lat, ckpts, int(nsteps), seg, phi0
        ctx.kappa_shape = kappa.shape if torch.is_tensor(kappa) else None
        return phi_t

    @staticmethod
    def backward(ctx, grad_phi_t):
        lat, lib = ctx.lat, L.lib()
        h = lat.handle
        n = lat.N
        dev = dict(device="cuda", dtype=torch.float64)
        af = torch.empty(19 * n, **dev)
        ag = torch.empty(19 * n, **dev)
        phi_bar = grad_phi_t.detach().to(**dev).contiguous()
        L.check(lib.lb_adjoint_seed(h, _p(phi_bar), _p(af), _p(ag)), "lb_adjoint_seed")
        af2 = torch.empty_like(af)
        ag2 = torch.empty_like(ag)
        dk = torch.zeros(1, **dev)
        for t0 in sorted(ctx.ckpts, reverse=True):
            t1 = min(t0 + ctx.seg, ctx.nsteps)
            lat.set_state(*ctx.ckpts[t0])
            states = [ctx.ckpts[t0]]
            for _ in range(t0 + 1, t1):
                lat.step(1)
                states.append(lat.get_state(device=True))
            for t in range(t1 - 1, t0 - 1, -1):
                f, g = states[t - t0]
                L.check(lib.lb_adjoint_step(h, _p(f), _p(g), _p(af), _p(ag), _p(af2), _p(ag2), _p(dk)),
                        "lb_adjoint_step")
                af, af2 = af2, af
                ag, ag2 = ag2, ag
        phi0_bar = torch.empty(n, **dev)
        L.check(lib.lb_adjoint_init(h, _p(ctx.phi0), None, _p(af), _p(ag), _p(phi0_bar), _p(dk)), "lb_adjoint_init")
        lat.close()
        ctx.ckpts = None
        dkappa = dk[0] if ctx.kappa_shape is None else dk.reshape(ctx.kappa_shape)
        return phi0_bar, dkappa, None, None, None, None


def trajectory(phi0, kappa, dims, params, nsteps, segment=None):
    """phi_T of the FP64 lattice started at equilibrium with order parameter
    ``phi0`` (CUDA float64 tensor [N]) and gradient coefficient ``kappa``
    (tensor, may require grad); other parameters from ``params``."""
    if not torch.is_tensor(kappa):
        kappa = torch.tensor(float(kappa), dtype=torch.float64, device="cuda")
    return LBTrajectory.apply(phi0, kappa, tuple(dims), dict(params), int(nsteps), segment)
