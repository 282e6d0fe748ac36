"""torch.autograd.Function over a checkpointed rollout of the CUDA step.

Forward: f^0 = f^eq(rho0, 0), nsteps steps through pplbm_forward_stored (every
step's psi and moments kept, when they fit in device memory) or
pplbm_forward_checkpointed (checkpoints every `interval` steps, ~sqrt(nsteps)),
output rho^N. Backward: pplbm_backward_stored, or pplbm_backward_checkpointed
(segment recomputation), then the hand-written adjoint kernels give dL/df^0 and
dL/d(EOS constants); the initial-density gradient is
sum_i w_i dL/df^0_i (pplbm_adjoint_initial_density) and the parameter gradient
(alpha, a_vap, a_liq or kappa, chosen by RolloutSpec.param) is the library's
chain rule: pplbm_adjoint_set_param takes dc/dtheta at the context's parameters
and selects the slots theta moves, pplbm_adjoint_param_gradient forms
sum_k grad[k] dc_k/dtheta. Argument marshalling only: every step, and every sum,
runs in the library.
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
    eos: EOSParams          # the differentiated parameter is taken from the Function's input
    relax: Relax
    nsteps: int
    interval: int = 0       # > 0: checkpoints every `interval` steps; 0: automatic (see `stored`)
    G: float = -1.0
    param: str = "alpha"    # "alpha", "a_vap", "a_liq" (EOS) or "kappa" (Relax)
    memory_fraction: float = 0.25  # automatic mode: share of free device memory the stored fields may take

    def k(self):
        return self.interval if self.interval > 0 else max(1, math.ceil(math.sqrt(self.nsteps)))

    def field_planes(self):
        """Planes a stored step keeps: psi and the moment planes (4 with unit relaxation
        times, 6 with the two-phase set)."""
        return 6 if self.relax.kind == L.RELAX_TWO_PHASE else 4

    def stored(self):
        """Keep every step's psi and moments (no recomputation) when the interval is
        automatic and field_planes() nx ny nsteps doubles fit in memory_fraction of the
        free device memory; otherwise sqrt(N) checkpointing with recomputation."""
        if self.interval > 0:
            return False
        import torch

        free, _ = torch.cuda.mem_get_info()
        return 8 * self.field_planes() * self.nx * self.ny * max(1, self.nsteps) <= self.memory_fraction * free


SENS_STEP = 1e-4  # step of the central differences behind dc/dtheta (pplbm_eos_constant_sensitivity)


def param_sensitivity(spec: RolloutSpec, value: float, h: float = SENS_STEP):
    """d(gradient constants)/d(spec.param) at spec.param = value, PPLBM_NGRAD values (host)."""
    dc = (C.c_double * L.NGRAD)()
    eos, relax = _with_param(spec, value)
    p = eos.c()
    r = relax.c()
    L.check(L.lib().pplbm_eos_constant_sensitivity(C.byref(p), spec.G, C.byref(r), L.SENS_PARAMS[spec.param], h,
                                                   dc))
    return list(dc)


def alpha_sensitivity(spec: RolloutSpec, alpha: float, h: float = SENS_STEP):
    """d(EOS constants)/d(alpha), PPLBM_NGRAD values (host)."""
    return param_sensitivity(replace(spec, param="alpha"), alpha, h)


def _with_param(spec: RolloutSpec, value: float):
    """(EOSParams, Relax) with spec.param set to value."""
    if spec.param not in L.SENS_PARAMS:
        raise ValueError(f"unknown parameter {spec.param!r}")
    if spec.param == "kappa":
        return spec.eos, replace(spec.relax, kappa=value)
    return replace(spec.eos, **{spec.param: value}), spec.relax


def _rollout_forward(spec: RolloutSpec, rho0, value: float):
    import torch

    eos, relax = _with_param(spec, value)
    sim = Simulation(spec.nx, spec.ny, spec.bc, eos, relax, G=spec.G)
    sim.init_equilibrium(rho0)
    if spec.stored():
        # ckpt holds every step's psi and moments
        ckpt = torch.empty((max(1, spec.nsteps), spec.field_planes(), spec.ny, spec.nx), dtype=torch.float64,
                           device=sim.device)
        sim._check(L.lib().pplbm_forward_stored(sim.ctx, spec.nsteps, _ptr(ckpt)))
        sim._stored = True
    else:
        K = spec.k()
        nseg = max(1, -(-spec.nsteps // K))
        ckpt = torch.empty((nseg, 9, spec.ny, spec.nx), dtype=torch.float64, device=sim.device)
        sim._check(L.lib().pplbm_forward_checkpointed(sim.ctx, spec.nsteps, K, _ptr(ckpt)))
    rhoN = sim.fields()[0]
    return sim, ckpt, rhoN


def _rollout_backward(spec: RolloutSpec, sim: Simulation, ckpt, grad_rhoN, slots=None):
    """Reverse pass; slots: the gradient slots to accumulate (bit mask), None = all."""
    import torch

    if slots is not None:
        sim._check(L.lib().pplbm_adjoint_set_slots(sim.ctx, int(slots)))
    dev = sim.device
    lamN = grad_rhoN.to(dev, torch.float64).reshape(1, spec.ny, spec.nx).expand(9, spec.ny, spec.nx).contiguous()
    lam0 = torch.empty((9, spec.ny, spec.nx), dtype=torch.float64, device=dev)
    grad = torch.zeros(L.NGRAD, dtype=torch.float64, device=dev)
    nbytes = L.lib().pplbm_adjoint_workspace_bytes(C.byref(sim.lattice))
    ws = torch.empty(nbytes // 8 + 1, dtype=torch.float64, device=dev)
    if getattr(sim, "_stored", False):   # stored fields of every step
        sim._check(L.lib().pplbm_backward_stored(sim.ctx, spec.nsteps, _ptr(ckpt), _ptr(lamN), _ptr(lam0),
                                                 _ptr(grad), _ptr(ws), nbytes))
    else:
        K = spec.k()
        seg = torch.empty((K, 9, spec.ny, spec.nx), dtype=torch.float64, device=dev)
        sim._check(L.lib().pplbm_backward_checkpointed(sim.ctx, spec.nsteps, K, _ptr(ckpt), _ptr(seg), _ptr(lamN),
                                                       _ptr(lam0), _ptr(grad), _ptr(ws), nbytes))
    rho0_bar = torch.empty((spec.ny, spec.nx), dtype=torch.float64, device=dev)
    sim._check(L.lib().pplbm_adjoint_initial_density(sim.ctx, _ptr(lam0), _ptr(rho0_bar)))
    sim.sync()
    return rho0_bar, grad, lam0


def _make_function():
    import torch

    class Rollout(torch.autograd.Function):
        """rho^N = rollout(rho0, theta); gradients w.r.t. rho0 and theta = spec.param."""

        @staticmethod
        def forward(ctx, rho0, theta, spec):
            sim, ckpt, rhoN = _rollout_forward(spec, rho0.detach(), float(theta))
            ctx.spec, ctx.sim, ctx.ckpt, ctx.theta = spec, sim, ckpt, float(theta)
            ctx.theta_device = theta.device if isinstance(theta, torch.Tensor) else torch.device("cpu")
            return rhoN

        @staticmethod
        def backward(ctx, grad_rhoN):
            spec = ctx.spec
            sim = ctx.sim
            sim._check(L.lib().pplbm_adjoint_set_param(sim.ctx, L.SENS_PARAMS[spec.param], SENS_STEP))
            rho0_bar, grad, _ = _rollout_backward(spec, sim, ctx.ckpt, grad_rhoN.contiguous())
            out = (C.c_double * 1)()
            sim._check(L.lib().pplbm_adjoint_param_gradient(sim.ctx, _ptr(grad), out))
            sim.close()
            gtheta = torch.tensor(out[0], dtype=grad_rhoN.dtype, device=ctx.theta_device)
            return rho0_bar, gtheta, None

    return Rollout


_FN = None


def rollout(rho0, theta, spec: RolloutSpec):
    """Differentiable rollout: rho0 (ny, nx) CUDA float64 tensor, theta a 0-d tensor
    holding the value of spec.param (alpha by default)."""
    global _FN
    if _FN is None:
        _FN = _make_function()
    return _FN.apply(rho0, theta, spec)
