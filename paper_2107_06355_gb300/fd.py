"""Python front end of the finite-difference solver (pplbm_fd_*): marshalling only."""
from __future__ import annotations

import ctypes as C

from . import _lib as L
from .lattice import EOSParams, _ptr


class FDSolver:
    """MacCormack solver of App. A on an nx x ny grid of spacing dx (CUDA): periodic
    (bc = BC_PERIODIC), or periodic in x with the wall layers of Eqs. B1, B2 at the
    bottom and reflexive layers at the top (bc = BC_WALLS_Y)."""

    def __init__(self, nx, ny, eos: EOSParams, tau_nu=1.0, tau_e=1.0, dx=1.0, G=-1.0, device="cuda", stream=None,
                 bc=L.BC_PERIODIC, tau_l=None, visc_ratio=None, kappa=0.0):
        import torch

        self.torch = torch
        self.nx, self.ny = int(nx), int(ny)
        self.lattice = L.pplbm_lattice(self.nx, self.ny, int(bc), 0)
        nbytes = L.lib().pplbm_fd_workspace_bytes(C.byref(self.lattice))
        if nbytes == 0:
            raise L.PPLBMError(L.PPLBM_ERR_ARG, "invalid FD grid or boundary flags")
        self.device = torch.device(device)
        self.workspace = torch.empty(nbytes // 8, dtype=torch.float64, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        p = eos.c()
        L.check(L.lib().pplbm_fd_create(C.byref(h), C.byref(self.lattice), C.byref(p), G, tau_nu, tau_e, dx,
                                        _ptr(self.workspace), nbytes, C.c_void_p(self.stream.cuda_stream)))
        self.h = h
        if tau_l is not None:   # tau_nu(rho) of Eq. RelaxationTime instead of the constant tau_nu
            L.check(L.lib().pplbm_fd_set_two_phase_viscosity(h, float(tau_l), float(visc_ratio)))
        if kappa != 0.0:        # the surface-tension control's pressure-tensor term
            L.check(L.lib().pplbm_fd_set_surface_tension(h, float(kappa)))

    def close(self):
        if getattr(self, "h", None):
            L.lib().pplbm_fd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, a):
        t = self.torch.as_tensor(a, dtype=self.torch.float64)
        return t.to(self.device).contiguous()

    def set_state(self, rho, ux, uy):
        r, u, v = self._dev(rho), self._dev(ux), self._dev(uy)
        L.check(L.lib().pplbm_fd_set_state(self.h, _ptr(r), _ptr(u), _ptr(v)))

    def get_state(self):
        out = [self.torch.empty((self.ny, self.nx), dtype=self.torch.float64, device=self.device) for _ in range(3)]
        L.check(L.lib().pplbm_fd_get_state(self.h, *[_ptr(t) for t in out]))
        return tuple(out)

    def step(self, nsteps, dt):
        L.check(L.lib().pplbm_fd_step(self.h, int(nsteps), float(dt)))

    def sync(self):
        L.check(L.lib().pplbm_fd_sync(self.h))
