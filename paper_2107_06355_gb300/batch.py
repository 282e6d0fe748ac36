"""Python front end of the batched engine (pplbm_batch_*): argument marshalling only."""
from __future__ import annotations

import ctypes as C

from . import _lib as L
from .lattice import EOSParams, Relax, _ptr


class Batch:
    """Independent lattices advanced together by one launch per pass (or one persistent
    launch per call). lattices: list of (nx, ny, bc); eos, relax: lists of the same length."""

    def __init__(self, lattices, eos, relax, G=-1.0, device="cuda", stream=None):
        import torch

        self.torch = torch
        n = len(lattices)
        if not (len(eos) == len(relax) == n and n > 0):
            raise ValueError("lattices, eos and relax must have the same, non-zero length")
        self.shapes = [(int(nx), int(ny)) for nx, ny, _ in lattices]
        self._lat = (L.pplbm_lattice * n)(*[L.pplbm_lattice(int(nx), int(ny), int(bc), 0) for nx, ny, bc in lattices])
        self._eos = (L.pplbm_eos_params * n)(*[e.c() for e in eos])
        self._relax = (L.pplbm_relax * n)(*[r.c() for r in relax])
        nbytes = L.lib().pplbm_batch_workspace_bytes(n, self._lat, self._relax)
        if nbytes == 0:
            raise L.PPLBMError(L.PPLBM_ERR_ARG, "invalid lattices or mixed collision kinds")
        self.device = torch.device(device)
        self.workspace = torch.empty(nbytes // 8 + 32, dtype=torch.float64, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        b = C.c_void_p()
        L.check(L.lib().pplbm_batch_create(C.byref(b), n, self._lat, self._eos, self._relax, G, C.c_void_p(aligned),
                                           nbytes, C.c_void_p(self.stream.cuda_stream)))
        self.b = b
        self.n = n

    def close(self):
        if getattr(self, "b", None):
            L.lib().pplbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        L.check(st, batch=self.b)

    def _dev(self, a):
        if a is None:
            return None
        t = self.torch.as_tensor(a, dtype=self.torch.float64)
        if t.device != self.device:
            t = t.to(self.device)
        return t.contiguous()

    def derived(self, i):
        out = L.pplbm_eos_derived()
        self._check(L.lib().pplbm_batch_get_derived(self.b, i, C.byref(out)))
        return out.as_dict()

    def init_equilibrium(self, i, rho0, ux0=None, uy0=None):
        r, u, v = self._dev(rho0), self._dev(ux0), self._dev(uy0)
        self._check(L.lib().pplbm_batch_init_equilibrium(self.b, i, _ptr(r), _ptr(u), _ptr(v)))

    def step(self, nsteps=1):
        self._check(L.lib().pplbm_batch_step(self.b, int(nsteps)))

    def sync(self):
        n = C.c_int64()
        self._check(L.lib().pplbm_batch_sync(self.b, C.byref(n)))
        return n.value

    def fields(self, i):
        nx, ny = self.shapes[i]
        out = [self.torch.empty((ny, nx), dtype=self.torch.float64, device=self.device) for _ in range(4)]
        self._check(L.lib().pplbm_batch_get_fields(self.b, i, *[_ptr(t) for t in out]))
        return tuple(out)

    def get_f(self, i):
        nx, ny = self.shapes[i]
        t = self.torch.empty((9, ny, nx), dtype=self.torch.float64, device=self.device)
        self._check(L.lib().pplbm_batch_get_f(self.b, i, _ptr(t)))
        return t

    def set_f(self, i, f):
        t = self._dev(f)
        self._check(L.lib().pplbm_batch_set_f(self.b, i, _ptr(t)))
        self.torch.cuda.current_stream(self.device).synchronize()

    def set_plan(self, mode, tile_width=0):
        self._check(L.lib().pplbm_batch_set_plan(self.b, int(mode), int(tile_width)))

    def plan(self):
        p = L.pplbm_batch_plan()
        self._check(L.lib().pplbm_batch_get_plan(self.b, C.byref(p)))
        return p.as_dict()

    def autotune(self, trial_steps=10):
        p = L.pplbm_batch_plan()
        self._check(L.lib().pplbm_batch_autotune(self.b, int(trial_steps), C.byref(p)))
        return p.as_dict()

    def enable_timing(self, capacity=4096):
        self._check(L.lib().pplbm_batch_enable_timing(self.b, int(capacity)))

    def times(self):
        ms = C.c_double()
        n = C.c_int64()
        self._check(L.lib().pplbm_batch_times(self.b, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def enable_pass_timing(self, capacity=4096):
        """CUDA events around each pass of every step (capacity 0 turns it off)."""
        self._check(L.lib().pplbm_batch_enable_pass_timing(self.b, int(capacity)))

    def pass_times(self):
        """((ms density/psi pass, ms collision pass), (launches, launches)) since the last call."""
        ms = (C.c_double * 2)()
        n = (C.c_int64 * 2)()
        self._check(L.lib().pplbm_batch_pass_times(self.b, ms, n))
        return (ms[0], ms[1]), (n[0], n[1])

    def set_isolation(self, on=True):
        """Let diverged instances be reported individually instead of stopping the batch."""
        self._check(L.lib().pplbm_batch_set_isolation(self.b, 1 if on else 0))

    def instance_status(self):
        """Per-instance status (0 ok, 4 diverged); synchronises."""
        st = (C.c_int32 * self.n)()
        self._check(L.lib().pplbm_batch_instance_status(self.b, st))
        return list(st)

    def run_host(self, rho0s, nsteps, outs):
        """pplbm_batch_run_host: host densities in (one contiguous float64 (ny, nx)
        array or CPU tensor per instance), nsteps, host densities out (same kind)."""
        def addr(a):
            return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data

        import numpy as np

        if len(rho0s) != self.n or len(outs) != self.n:
            raise ValueError("one input and one output array per instance")
        for k, (a, o) in enumerate(zip(rho0s, outs)):
            nx, ny = self.shapes[k]
            for t in (a, o):
                if hasattr(t, "is_cuda"):
                    ok = (not t.is_cuda) and t.dtype == self.torch.float64 and t.is_contiguous() and t.numel() == nx * ny
                else:
                    ok = isinstance(t, np.ndarray) and t.dtype == np.float64 and t.flags.c_contiguous and t.size == nx * ny
                if not ok:
                    raise ValueError(f"instance {k}: need a contiguous float64 host array of {ny} x {nx}")
        src = (C.c_void_p * self.n)(*[addr(a) for a in rho0s])
        dst = (C.c_void_p * self.n)(*[addr(a) for a in outs])
        self._check(L.lib().pplbm_batch_run_host(self.b, src, int(nsteps), dst))

    def guard(self):
        """(n, 4) array per instance: mass, max |u| with u = (j + F/2)/rho, bad-node
        count, residual against the previous guard call (-1 when there is none);
        synchronises."""
        import numpy as np

        out = np.empty(4 * self.n, dtype=np.float64)
        self._check(L.lib().pplbm_batch_guard(self.b, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out.reshape(self.n, 4)

    def barrier_selftest(self, spin_limit=1 << 14):
        """Status of the bounded-barrier self-test (expected: PPLBM_ERR_TIMEOUT = 5)."""
        return L.lib().pplbm_batch_barrier_selftest(self.b, int(spin_limit))
