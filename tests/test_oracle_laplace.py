"""Laplace's law pin for the oracle (CPU only): static droplets on a 64 x 64
periodic lattice, T_r = 0.6, Smooth C-S (a_l = 0.387, a_v = 2, alpha = 0.834),
tau = 1, Li forcing. The pressure jump p_EOS(rho_centre) - p_EOS(rho_corner)
times the equimolar radius approaches the planar surface tension: fitting
dp R = gamma + b/R and taking R -> infinity gives gamma within 5 % of the
surface tension the paper prints for this EOS (Table DropImpactParameters,
gamma_alpha = 6.3e-3; 2-D Laplace law dp = gamma / R)."""
import json
import os

import numpy as np

import lbm_inputs as I
from oracle import eos as E
from oracle import lbm as L

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _droplet(R, n=64):
    """(equimolar radius, dp) of a static droplet of radius R, run to the Sec. III.A
    residual 1e-7 (built here, so spawned workers can run it)."""
    e = E.make_eos(E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834)
    e.solve_eps()
    lat = L.Lattice(n, n, L.BC_PERIODIC_X | L.BC_PERIODIC_Y, e, L.Relax(sigma=e.sigma()))
    f = lat.init_equilibrium(I.droplet(n, n, R, e.rho_v, e.rho_l, W=8.0))
    prev = f.sum(0)
    for _ in range(60):
        f = lat.step(f, 100)
        rho = f.sum(0)
        r = L.convergence_residual(rho, prev)
        prev = rho
        if r < 1e-7:
            break
    rin, rout = rho[n // 2, n // 2], rho[0, 0]
    dp = float(e.pressure(rin) - e.pressure(rout))
    req = float(np.sqrt(((rho - rout) / (rin - rout)).sum() / np.pi))
    return req, dp


def test_laplace_law_extrapolates_to_planar_surface_tension():
    import multiprocessing
    from concurrent.futures import ProcessPoolExecutor

    radii = (10, 14, 20)
    # independent droplets: side by side in spawned processes
    with ProcessPoolExecutor(max_workers=3, mp_context=multiprocessing.get_context("spawn")) as ex:
        pts = list(ex.map(_droplet, radii))
    for R, (req, _) in zip(radii, pts):
        assert abs(req - R) < 0.5
    x = np.array([1.0 / r for r, _ in pts])
    y = np.array([d * r for r, d in pts])
    b, gamma = np.polyfit(x, y, 1)
    case = [c for c in GOLD["table_drop_impact_parameters"]["cases"] if c["name"] == "Smooth_alpha0.834_Tr0.6"][0]
    assert abs(gamma / (case["gamma_e3"] * 1e-3) - 1) < 0.05
    # every droplet is within 12 % of the planar value (curvature corrections shrink with R)
    assert np.all(np.abs(y / (case["gamma_e3"] * 1e-3) - 1) < 0.12)
