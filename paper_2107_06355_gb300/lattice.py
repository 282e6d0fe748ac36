"""Python front end of the C ABI: parameter records and a Simulation object.

Argument marshalling only. Device buffers are torch tensors (float64, CUDA);
their pointers and the current CUDA stream are passed to the library.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

from . import _lib as L


@dataclass
class EOSParams:
    """Equation of state at one reduced temperature (Sec. III, Sec. III.D)."""
    mode: int = L.EOS_SMOOTH
    Tr: float = 0.6
    a_liq: float = 0.387
    a_vap: float = 2.0
    alpha: float = 0.834
    b: float = 4.0
    R: float = 1.0
    r_theta: float = 0.0

    def c(self):
        return L.pplbm_eos_params(self.mode, 0, self.Tr, self.a_liq, self.a_vap, self.b, self.R, self.alpha,
                                  self.r_theta)


@dataclass
class Relax:
    """Relaxation set and forcing (Eq. RelaxationMatrix, Eq. RelaxationTime, Eqs. GFS / LiFS)."""
    kind: int = L.RELAX_MRT
    forcing: int = L.FORCING_LI
    tau_rho: float = 1.0
    tau_e: float = 1.0
    tau_zeta: float = 1.0
    tau_j: float = 1.0
    tau_q: float = 1.0
    tau_nu: float = 1.0
    tau_l: float = 1.0
    visc_ratio: float = 1.0
    sigma: float = 0.0
    sigma_auto: bool = True
    kappa: float = 0.0  # surface-tension control (Sec. V's technique, Li & Luo 2013); 0 = off

    def c(self):
        return L.pplbm_relax(self.kind, self.forcing, self.tau_rho, self.tau_e, self.tau_zeta, self.tau_j,
                             self.tau_q, self.tau_nu, self.tau_l, self.visc_ratio, self.sigma,
                             1 if self.sigma_auto else 0, 0, self.kappa)


def eos_setup(params: EOSParams, G: float = -1.0) -> dict:
    """pplbm_eos_setup (host only): the derived EOS block as a dict."""
    out = L.pplbm_eos_derived()
    p = params.c()
    L.check(L.lib().pplbm_eos_setup(C.byref(p), G, C.byref(out)))
    return out.as_dict()


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


class Simulation:
    """One lattice advanced by the CUDA step (pplbm_create ... pplbm_destroy)."""

    def __init__(self, nx, ny, bc, eos: EOSParams, relax: Relax, G=-1.0, device="cuda", stream=None):
        import torch

        self.torch = torch
        self.nx, self.ny, self.bc = int(nx), int(ny), int(bc)
        self.lattice = L.pplbm_lattice(self.nx, self.ny, self.bc, 0)
        self.eos_params, self.relax, self.G = eos, relax, G
        self._eos_c, self._relax_c = eos.c(), relax.c()
        nbytes = L.lib().pplbm_workspace_bytes(C.byref(self.lattice), C.byref(self._relax_c))
        if nbytes == 0:
            raise L.PPLBMError(L.PPLBM_ERR_ARG, "invalid lattice or relaxation set")
        self.device = torch.device(device)
        self.workspace = torch.empty(nbytes // 8, dtype=torch.float64, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        ctx = C.c_void_p()
        L.check(L.lib().pplbm_create(C.byref(ctx), C.byref(self.lattice), C.byref(self._eos_c),
                                     C.byref(self._relax_c), G, _ptr(self.workspace), nbytes,
                                     C.c_void_p(self.stream.cuda_stream)))
        self.ctx = ctx

    # -- life cycle ------------------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            L.lib().pplbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, status):
        L.check(status, self.ctx)

    @property
    def n(self):
        return self.nx * self.ny

    def derived(self) -> dict:
        out = L.pplbm_eos_derived()
        self._check(L.lib().pplbm_get_derived(self.ctx, C.byref(out)))
        return out.as_dict()

    # -- state -----------------------------------------------------------------------
    def _dev(self, a):
        torch = self.torch
        if a is None:
            return None
        t = torch.as_tensor(a, dtype=torch.float64)
        if t.device != self.device:
            t = t.to(self.device)
        return t.contiguous()

    def init_equilibrium(self, rho0, ux0=None, uy0=None):
        """f = f^eq(rho0, u0); rho0/ux0/uy0 of shape (ny, nx) (numpy or torch)."""
        r, u, v = self._dev(rho0), self._dev(ux0), self._dev(uy0)
        for t in (r, u, v):
            if t is not None and t.numel() != self.n:
                raise ValueError("field has the wrong size")
        self._keep = (r, u, v)
        self._check(L.lib().pplbm_init_equilibrium(self.ctx, _ptr(r), _ptr(u), _ptr(v)))

    def step(self, nsteps=1):
        self._check(L.lib().pplbm_step(self.ctx, int(nsteps)))

    def sync(self):
        n = C.c_int64()
        self._check(L.lib().pplbm_sync(self.ctx, C.byref(n)))
        return n.value

    def fields(self):
        """(rho, ux, uy, psi) as (ny, nx) float64 CUDA tensors."""
        torch = self.torch
        out = [torch.empty((self.ny, self.nx), dtype=torch.float64, device=self.device) for _ in range(4)]
        self._check(L.lib().pplbm_get_fields(self.ctx, *[_ptr(t) for t in out]))
        return tuple(out)

    def get_f(self):
        t = self.torch.empty((9, self.ny, self.nx), dtype=self.torch.float64, device=self.device)
        self._check(L.lib().pplbm_get_f(self.ctx, _ptr(t)))
        return t

    def set_f(self, f):
        t = self._dev(f)
        if t.numel() != 9 * self.n:
            raise ValueError("f has the wrong size")
        self._check(L.lib().pplbm_set_f(self.ctx, _ptr(t)))
        self.torch.cuda.current_stream(self.device).synchronize()

    def guard(self):
        """(mass, max |u| with u = (j + F/2)/rho, bad-node count, residual
        sum |rho - rho'| / sum rho against the previous guard call, -1 if none);
        synchronises."""
        out = (C.c_double * 4)()
        self._check(L.lib().pplbm_guard(self.ctx, out))
        return out[0], out[1], int(out[2]), out[3]

    def enable_kernel_timing(self, capacity=4096):
        """Record per-launch device times of the two step kernels (capacity 0 disables)."""
        self._check(L.lib().pplbm_enable_kernel_timing(self.ctx, int(capacity)))

    def kernel_times(self):
        """((ms_rho_psi, ms_collide), (launches_rho_psi, launches_collide)) since the last call."""
        ms = (C.c_double * 2)()
        n = (C.c_int64 * 2)()
        self._check(L.lib().pplbm_kernel_times(self.ctx, ms, n))
        return (ms[0], ms[1]), (n[0], n[1])

    def run_host(self, rho0, nsteps, ux0=None, uy0=None):
        """pplbm_run_host: host arrays in, host density out (numpy float64, C-contiguous)."""
        import numpy as np
        r = np.ascontiguousarray(rho0, dtype=np.float64)
        u = None if ux0 is None else np.ascontiguousarray(ux0, dtype=np.float64)
        v = None if uy0 is None else np.ascontiguousarray(uy0, dtype=np.float64)
        out = np.empty((self.ny, self.nx), dtype=np.float64)
        p = lambda a: None if a is None else C.c_void_p(a.ctypes.data)
        self._check(L.lib().pplbm_run_host(self.ctx, p(r), p(u), p(v), int(nsteps), p(out)))
        return out
