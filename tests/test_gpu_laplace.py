"""Static droplets at the configuration's full size on the GPU: four 512 x 512
periodic lattices (R = 32, 48, 64, 96), T_r = 0.6, Smooth C-S, tau = 1, through
the batched engine. The configuration names 50,000 steps, but the R = 96
droplet's shape oscillation (decay time ~R^2/nu ~ 5e4 steps) still shifts dp R by
40 % there; it settles by 100,000, so the test runs 150,000 steps. Laplace's law: dp R (dp = p_EOS(centre) -
p_EOS(corner)) extrapolated to R -> infinity equals the planar surface tension
the paper prints (6.3e-3) within 3 % (measured: 6.22e-3); the spurious currents
stay bounded. The
oracle pins the same law on 64 x 64 lattices (test_oracle_laplace.py)."""
import math

import numpy as np
import pytest

import lbm_inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2107_06355_gb300")


def test_laplace_law_512_droplets_150000_steps():
    radii = (32, 48, 64, 96)
    eosp = P.EOSParams(P.EOS_SMOOTH, 0.6, 0.387, 2.0, 0.834)
    b = P.Batch([(512, 512, P.BC_PERIODIC)] * 4, [eosp] * 4, [P.Relax()] * 4)
    d = b.derived(0)
    for k, R in enumerate(radii):
        b.init_equilibrium(k, I.droplet(512, 512, R, d["rho_v"], d["rho_l"], W=8.0))
    b.autotune(trial_steps=4)
    b.step(150000)
    assert b.sync() == 150000
    pts, umax = [], []
    from oracle import eos as E
    oe = E.make_eos(E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834)
    for k, R in enumerate(radii):
        rho, ux, uy, _ = [t.cpu().numpy() for t in b.fields(k)]
        rin, rout = rho[256, 256], rho[0, 0]
        dp = float(oe.pressure(rin) - oe.pressure(rout))
        req = math.sqrt(((rho - rout) / (rin - rout)).sum() / math.pi)
        assert abs(req - R) < 0.05 * R   # the droplet evaporates slightly into the large vapour region
        pts.append((req, dp))
        umax.append(float(np.sqrt(ux**2 + uy**2).max()))
    x = np.array([1.0 / r for r, _ in pts])
    y = np.array([d_ * r for r, d_ in pts])
    slope, gamma = np.polyfit(x, y, 1)
    assert abs(gamma / 6.3e-3 - 1) < 0.03, (gamma, y)
    # spurious currents (the paper prints no value; 6e-3 to 7.5e-3 measured, peaking in the vapour
    # next to the interface): a sanity bound only
    assert max(umax) < 2e-2, umax
    b.close()
