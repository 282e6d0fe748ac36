"""torch.autograd.Function over a checkpointed rollout of the CUDA step.

Forward: f^0 = f^eq(rho0, 0), nsteps steps through pplbm_forward_checkpointed
(checkpoints every `interval` steps, ~sqrt(nsteps)), output rho^N. Backward:
pplbm_backward_checkpointed (segment recomputation + hand-written adjoint
kernels) gives dL/df^0 and dL/d(EOS constants); the initial-density gradient is
sum_i w_i dL/df^0_i and the alpha gradient chains the constants' gradients with
their alpha-derivatives (pplbm_eos_constant_sensitivity). Argument marshalling
only: every step runs in the library's kernels.
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass, replace

from . import _lib as L
from .lattice import EOSParams, Relax, Simulation, _ptr


@dataclass
class RolloutSpec:
    nx: int
    ny: int
    bc: int
    eos: EOSParams          # alpha is taken from the Function's input
    relax: Relax
    nsteps: int
    interval: int = 0       # 0: ceil(sqrt(nsteps))
    G: float = -1.0

    def k(self):
        return self.interval if self.interval > 0 else max(1, math.ceil(math.sqrt(self.nsteps)))


def alpha_sensitivity(spec: RolloutSpec, alpha: float, h: float = 1e-4):
    """d(EOS constants)/d(alpha), PPLBM_NGRAD values (host)."""
    dc = (C.c_double * L.NGRAD)()
    p = replace(spec.eos, alpha=alpha).c()
    r = spec.relax.c()
    L.check(L.lib().pplbm_eos_constant_sensitivity(C.byref(p), spec.G, C.byref(r), 0, h, dc))
    return list(dc)


def _rollout_forward(spec: RolloutSpec, rho0, alpha: float):
    import torch

    sim = Simulation(spec.nx, spec.ny, spec.bc, replace(spec.eos, alpha=alpha), spec.relax, G=spec.G)
    sim.init_equilibrium(rho0)
    K = spec.k()
    nseg = max(1, -(-spec.nsteps // K))
    ckpt = torch.empty((nseg, 9, spec.ny, spec.nx), dtype=torch.float64, device=sim.device)
    sim._check(L.lib().pplbm_forward_checkpointed(sim.ctx, spec.nsteps, K, _ptr(ckpt)))
    rhoN = sim.fields()[0]
    return sim, ckpt, rhoN


def _rollout_backward(spec: RolloutSpec, sim: Simulation, ckpt, grad_rhoN):
    import torch

    K = spec.k()
    dev = sim.device
    lamN = grad_rhoN.to(dev, torch.float64).reshape(1, spec.ny, spec.nx).expand(9, spec.ny, spec.nx).contiguous()
    seg = torch.empty((K, 9, spec.ny, spec.nx), dtype=torch.float64, device=dev)
    lam0 = torch.empty((9, spec.ny, spec.nx), dtype=torch.float64, device=dev)
    grad = torch.zeros(L.NGRAD, dtype=torch.float64, device=dev)
    nbytes = L.lib().pplbm_adjoint_workspace_bytes(C.byref(sim.lattice))
    ws = torch.empty(nbytes // 8 + 1, dtype=torch.float64, device=dev)
    sim._check(L.lib().pplbm_backward_checkpointed(sim.ctx, spec.nsteps, K, _ptr(ckpt), _ptr(seg), _ptr(lamN),
                                                   _ptr(lam0), _ptr(grad), _ptr(ws), nbytes))
    rho0_bar = torch.empty((spec.ny, spec.nx), dtype=torch.float64, device=dev)
    sim._check(L.lib().pplbm_adjoint_initial_density(sim.ctx, _ptr(lam0), _ptr(rho0_bar)))
    sim.sync()
    return rho0_bar, grad, lam0


def _make_function():
    import torch

    class Rollout(torch.autograd.Function):
        """rho^N = rollout(rho0, alpha); gradients w.r.t. rho0 and alpha."""

        @staticmethod
        def forward(ctx, rho0, alpha, spec):
            sim, ckpt, rhoN = _rollout_forward(spec, rho0.detach(), float(alpha))
            ctx.spec, ctx.sim, ctx.ckpt, ctx.alpha = spec, sim, ckpt, float(alpha)
            return rhoN

        @staticmethod
        def backward(ctx, grad_rhoN):
            spec = ctx.spec
            rho0_bar, grad, _ = _rollout_backward(spec, ctx.sim, ctx.ckpt, grad_rhoN.contiguous())
            dc = torch.tensor(alpha_sensitivity(spec, ctx.alpha), dtype=torch.float64, device=grad.device)
            galpha = (grad * dc).sum()
            ctx.sim.close()
            return rho0_bar, galpha.to(grad_rhoN.dtype), None

    return Rollout


_FN = None


def rollout(rho0, alpha, spec: RolloutSpec):
    """Differentiable rollout: rho0 (ny, nx) CUDA float64 tensor, alpha a 0-d tensor."""
    global _FN
    if _FN is None:
        _FN = _make_function()
    return _FN.apply(rho0, alpha, spec)
