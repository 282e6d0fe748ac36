"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds no arithmetic of the lattice Boltzmann method itself: it only
builds initial density / velocity fields and workload descriptions from numbers
it is given (coexistence densities come from whichever side calls it). Shapes
follow the paper's set-ups:

* planar interface: a liquid slab between two tanh interfaces (Sec. III.A,
  Eq. PlanarIntDensity: factor 4.6/W, interfaces at 1/4 and 3/4 of the length);
* static droplet: a tanh-profiled disc (Sec. IV uses the same tanh form);
* droplet impact: a liquid film on the bottom wall and a droplet above it moving
  down with speed V_d (Sec. IV);
* a seeded batch of planar and droplet lattices of uneven size.
"""
from __future__ import annotations

import numpy as np

BATCH_SEED = 210706355


def planar(nx, ny, rho_v, rho_l, W=10.0, axis="y"):
    """Eq. PlanarIntDensity along `axis` ('y': profile varies with y; 'x': with x)."""
    n = ny if axis == "y" else nx
    s = np.arange(n, dtype=np.float64)
    s1, s2 = 0.25 * n, 0.75 * n
    prof = rho_v + 0.5 * (rho_l - rho_v) * (np.tanh(4.6 * (s - s1) / W) - np.tanh(4.6 * (s - s2) / W))
    if axis == "y":
        return np.repeat(prof[:, None], nx, axis=1)
    return np.repeat(prof[None, :], ny, axis=0)


def droplet(nx, ny, R, rho_v, rho_l, W=8.0, center=None):
    """Disc of radius R with a tanh interface of width W (0.01..0.99 span ~ W)."""
    cx, cy = (nx / 2.0, ny / 2.0) if center is None else center
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    phi = 0.5 * (1.0 - np.tanh(4.6 * (r - R) / W))
    return rho_v + (rho_l - rho_v) * phi


def impact(nx, ny, R, film_h, rho_v, rho_l, V_d, W=8.0, dx=1.0):
    """Droplet above a liquid film on the bottom wall (Sec. IV set-up).

    rho = rho_v + (rho_l - rho_v) max(phi_drop, phi_film); the drop centre is at
    (nx dx/2, film_h + R + W); the drop moves with (0, -V_d) weighted by phi_drop.
    Lengths are in lattice units; node (i, j) sits at (i dx, j dx), so dx < 1 samples
    the same field on a finer grid. Returns (rho, ux, uy)."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64) * dx
    cx, cy = nx * dx / 2.0, film_h + R + W
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    phi_d = 0.5 * (1.0 - np.tanh(4.6 * (r - R) / W))
    phi_f = 0.5 * (1.0 - np.tanh(4.6 * (y - film_h) / W))
    rho = rho_v + (rho_l - rho_v) * np.maximum(phi_d, phi_f)
    ux = np.zeros_like(rho)
    uy = -V_d * phi_d
    return rho, ux, uy


def perturbed(rho, rel_amp, seed):
    """rho * (1 + rel_amp * U(-1, 1)) with a seeded generator."""
    rng = np.random.default_rng(seed)
    return rho * (1.0 + rel_amp * rng.uniform(-1.0, 1.0, size=np.shape(rho)))


def random_velocity(shape, amp, seed):
    rng = np.random.default_rng(seed)
    return amp * rng.uniform(-1.0, 1.0, size=shape), amp * rng.uniform(-1.0, 1.0, size=shape)


def batch_specs(n=64, seed=BATCH_SEED, lmin=64, lmax=1024):
    """Batch of independent lattices: even k -> planar L x 4, odd k -> droplet L x L with
    R = L/4; L ~ U{lmin..lmax}; reduced temperature 0.35 + 0.6 k/(n-1)."""
    rng = np.random.default_rng(seed)
    L = rng.integers(lmin, lmax + 1, size=n)
    specs = []
    for k in range(n):
        Tr = 0.35 + 0.6 * k / (n - 1)
        if k % 2 == 0:
            specs.append(dict(kind="planar", nx=4, ny=int(L[k]), Tr=Tr))
        else:
            specs.append(dict(kind="droplet", nx=int(L[k]), ny=int(L[k]), R=int(L[k]) / 4.0, Tr=Tr))
    return specs
