"""Parameter sweeps of planar-interface equilibria on the batched engine (Sec. III).

`planar_coexistence` advances many (Nx, Ny) = (2, 200) periodic planar interfaces
(one per (EOS, relaxation) case) in one batch until the convergence criterion of
Sec. III.A holds for each, then reports the paper's observables: the vapour
density error of Eq. DensityError, the interface width (nodes with
0.01 < (rho - rho_v)/(rho_l - rho_v) < 0.99, with the simulated densities) and
the surface tension of Eq. SurfaceTension (fourth-order central differences,
Simpson's rule). Instances are isolated: one that diverges is reported as such
and the others continue. All stepping runs in the library's kernels; the host
only checks convergence and evaluates the observables on the returned fields.
"""
from __future__ import annotations

import numpy as np

from . import _lib as L
from .batch import Batch


def planar_profile(ny, rho_v, rho_l, W):
    """Eq. PlanarIntDensity along y: interfaces at 1/4 and 3/4 of the length."""
    y = np.arange(ny, dtype=np.float64)
    return rho_v + 0.5 * (rho_l - rho_v) * (np.tanh(4.6 * (y - 0.25 * ny) / W) - np.tanh(4.6 * (y - 0.75 * ny) / W))


def density_error(rho_v_sim, rho_v_maxwell):
    """Eq. DensityError, in percent."""
    return 100.0 * (rho_v_sim - rho_v_maxwell) / rho_v_maxwell


def interface_width(profile, rho_v, rho_l):
    """Nodes of the first interface with 0.01 < phi < 0.99 (Sec. III.B definition)."""
    phi = (np.asarray(profile) - rho_v) / (rho_l - rho_v)
    first = phi[: len(phi) // 2]
    return int(np.count_nonzero((first > 0.01) & (first < 0.99)))


def surface_tension(psi_profile, G=-1.0):
    """Eq. SurfaceTension on a periodic profile with two interfaces (half the period integral)."""
    p = np.asarray(psi_profile, dtype=np.float64)
    n = len(p)
    d = (p[(np.arange(n) - 2) % n] - 8 * p[(np.arange(n) - 1) % n] + 8 * p[(np.arange(n) + 1) % n]
         - p[(np.arange(n) + 2) % n]) / 12.0
    g = np.append(d * d, d[0] * d[0])
    w = np.ones(n + 1)
    w[1:-1:2] = 4.0
    w[2:-1:2] = 2.0
    return -G / 6.0 * float(np.dot(w, g) / 3.0) / 2.0


def planar_coexistence(cases, nx=2, ny=200, W=10.0, tol=1e-6, check_every=100, max_steps=300000, G=-1.0):
    """cases: list of (EOSParams, Relax). Returns one dict per case with keys
    converged, diverged, steps, rho_v, rho_l, E_percent, width, gamma."""
    import torch

    n = len(cases)
    b = Batch([(nx, ny, L.BC_PERIODIC)] * n, [c[0] for c in cases], [c[1] for c in cases], G=G)
    b.set_isolation(True)
    maxwell = []
    for i in range(n):
        d = b.derived(i)
        maxwell.append((d["rho_v"], d["rho_l"]))
        prof = planar_profile(ny, d["rho_v"], d["rho_l"], W)
        b.init_equilibrium(i, np.repeat(prof[:, None], nx, axis=1))
    b.set_plan(L.PLAN_GRAPH, 0)
    prev = [b.fields(i)[0].cpu().numpy() for i in range(n)]
    done = [False] * n
    out = [dict(converged=False, diverged=False, steps=0) for _ in range(n)]
    steps = 0
    while steps < max_steps and not all(done):
        b.step(check_every)
        steps += check_every
        status = b.instance_status()
        for i in range(n):
            if done[i]:
                continue
            if status[i] != 0:
                done[i] = True
                out[i].update(diverged=True, steps=steps)
                continue
            rho = b.fields(i)[0].cpu().numpy()
            res = float(np.abs(rho - prev[i]).sum() / np.abs(rho).sum())
            prev[i] = rho
            if not np.isfinite(res):
                done[i] = True
                out[i].update(diverged=True, steps=steps)
            elif res < tol:
                done[i] = True
                out[i].update(converged=True, steps=steps)
    for i in range(n):
        if out[i]["diverged"]:
            continue
        if not done[i]:
            out[i]["steps"] = steps
        rho, _, _, psi = [t.cpu().numpy() for t in b.fields(i)]
        col_r, col_p = rho[:, 0], psi[:, 0]
        rv, rl = float(col_r[0]), float(col_r[ny // 2])
        out[i].update(rho_v=rv, rho_l=rl, E_percent=density_error(rv, maxwell[i][0]),
                      width=interface_width(col_r, rv, rl), gamma=surface_tension(col_p, G))
    b.close()
    torch.cuda.synchronize()
    return out
