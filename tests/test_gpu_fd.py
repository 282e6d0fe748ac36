"""GPU finite-difference (MacCormack) solver against the CPU FD oracle (App. A):
same initial state, same grid and time step, normwise agreement of rho and u."""
import numpy as np
import pytest

import lbm_inputs as I
from gpu_helpers import normwise
from oracle import eos as E
from oracle import fd as F

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2107_06355_gb300")


@pytest.mark.parametrize("shape,dx,taus", [((1, 120), 0.5, (1.0, 1.0)), ((48, 40), 1.0, (0.8, 1.1)),
                                           ((37, 29), 0.5, (1.0, 1.0))])
def test_fd_matches_cpu_oracle(shape, dx, taus):
    nx, ny = shape
    tau_nu, tau_e = taus
    oe = E.make_eos(E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834)
    eps = oe.solve_eps(n=40000)
    L_ = ny * dx
    if nx == 1:
        rho = I.planar(1, ny, oe.rho_v, oe.rho_l, W=8.0 / dx)
    else:
        rho = I.droplet(nx, ny, min(nx, ny) / 4, oe.rho_v, oe.rho_l, W=6.0 / dx)
    ux, uy = I.random_velocity((ny, nx), 0.004, 3)
    dt = 0.8 * dx * dx
    cpu = F.FDSolver(oe, eps, tau_nu=tau_nu, tau_e=tau_e, dx=dx)
    r, u = cpu.run(rho.copy(), [ux.copy(), uy.copy()], 40 * dt, dt)
    gpu = P.FDSolver(nx, ny, P.EOSParams(P.EOS_SMOOTH, 0.6, 0.387, 2.0, 0.834), tau_nu=tau_nu, tau_e=tau_e, dx=dx)
    gpu.set_state(rho, ux, uy)
    gpu.step(40, dt)
    gr, gux, guy = [t.cpu().numpy() for t in gpu.get_state()]
    assert np.isfinite(r).all()
    # the oracle's eps (Simpson) differs from the library's by ~1e-11 relative
    assert normwise(gr, r) < 1e-10
    umax = max(np.abs(u[0]).max(), np.abs(u[1]).max())
    assert np.max(np.abs(gux - u[0])) < 1e-9 * umax
    assert np.max(np.abs(guy - u[1])) < 1e-9 * umax
    gpu.close()
