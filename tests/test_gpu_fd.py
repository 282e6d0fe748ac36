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


def _ellipse(n, R, eps, rv, rl, W, dx):
    y, x = np.mgrid[0:n, 0:n].astype(np.float64) * dx
    c = n * dx / 2
    a, b = R * (1 + eps), R / (1 + eps)
    r = np.sqrt(((x - c) / a) ** 2 + ((y - c) / b) ** 2) * R
    return rv + (rl - rv) * 0.5 * (1 - np.tanh(4.6 * (r - R) / W))


def _deformation(rho, rv, rl, dx):
    """(sqrt(I_xx) - sqrt(I_yy)) / (sqrt(I_xx) + sqrt(I_yy)) of the liquid fraction."""
    n = rho.shape[0]
    phi = np.clip((rho - rv) / (rl - rv), 0.0, 1.0)
    y, x = np.mgrid[0:n, 0:n].astype(np.float64) * dx
    m = phi.sum()
    cx, cy = (phi * x).sum() / m, (phi * y).sum() / m
    sx, sy = np.sqrt((phi * (x - cx) ** 2).sum() / m), np.sqrt((phi * (y - cy) ** 2).sum() / m)
    return (sx - sy) / (sx + sy)


def test_oscillating_droplet_lbm_agrees_with_fd_and_fd_refines_toward_it():
    """Nonlinear dynamics of both solvers on the same macroscopic problem (App. A: the
    FD scheme solves the equations the LBM recovers): an elliptic droplet (R = 30,
    semi-axes R(1 +- 0.15), T_r = 0.6 Smooth C-S, tau = 1) relaxing on a 128^2
    periodic domain for 4,000 time units. The deformation histories of the LBM and
    of FD at dx = 1/2 agree to 0.02 (amplitude 0.14) with zero crossings within
    200 time units, and refining FD from dx = 1 to 1/2 moves it toward the LBM."""
    L_, R, eps, W, T, every = 128, 30.0, 0.15, 8.0, 4000, 200
    eosp = P.EOSParams(P.EOS_SMOOTH, 0.6, 0.387, 2.0, 0.834)
    d = P.eos_setup(eosp)
    rv, rl = d["rho_v"], d["rho_l"]
    sim = P.Simulation(L_, L_, P.BC_PERIODIC, eosp, P.Relax())
    sim.init_equilibrium(_ellipse(L_, R, eps, rv, rl, W, 1.0))
    lbm = []
    for t in range(0, T + 1, every):
        if t:
            sim.step(every)
        lbm.append(_deformation(sim.fields()[0].cpu().numpy(), rv, rl, 1.0))
    sim.close()
    fd = {}
    for dx in (1.0, 0.5):
        n = int(L_ / dx)
        s = P.FDSolver(n, n, eosp, dx=dx, tau_nu=1.0, tau_e=1.0)
        z = np.zeros((n, n))
        s.set_state(_ellipse(n, R, eps, rv, rl, W, dx), z, z)
        dt = 0.4 * dx * dx
        hist = []
        for t in range(0, T + 1, every):
            if t:
                s.step(int(round(every / dt)), dt)
            hist.append(_deformation(s.get_state()[0].cpu().numpy(), rv, rl, dx))
        s.close()
        fd[dx] = np.array(hist)
    lbm = np.array(lbm)
    assert np.max(np.abs(lbm - fd[0.5])) < 0.02
    assert np.linalg.norm(lbm - fd[0.5]) < np.linalg.norm(lbm - fd[1.0])
    times = np.arange(0, T + 1, every, dtype=np.float64)

    def crossings(h):
        k = np.nonzero(np.sign(h[1:]) != np.sign(h[:-1]))[0]
        return times[k] + every * h[k] / (h[k] - h[k + 1])

    cl, cf = crossings(lbm), crossings(fd[0.5])
    assert len(cl) == len(cf) >= 2
    assert np.max(np.abs(cl - cf)) < 200.0


@pytest.mark.parametrize("shape,dx", [((48, 40), 1.0), ((48, 80), 0.5)])
def test_fd_with_walls_matches_cpu_oracle(shape, dx):
    """The wall layers of Eqs. B1, B2 and the reflexive top on the GPU against the CPU
    FD oracle: a drop (R = 8, W = 8 in lattice units) moving towards a liquid film of
    height 6 on the bottom wall, 40 steps, at grid spacings 1 and 1/2."""
    nx, ny = shape
    oe = E.make_eos(E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834)
    eps = oe.solve_eps(n=40000)
    rho, ux, uy = I.impact(nx, ny, 8.0, 6.0, oe.rho_v, oe.rho_l, 0.02, W=8.0, dx=dx)
    dt = 0.4 * dx * dx
    cpu = F.FDSolver(oe, eps, tau_nu=0.8, tau_e=1.0, dx=dx, walls=True)
    r, u = cpu.run(rho.copy(), [ux.copy(), uy.copy()], 40 * dt, dt)
    gpu = P.FDSolver(nx, ny, P.EOSParams(P.EOS_SMOOTH, 0.6, 0.387, 2.0, 0.834), tau_nu=0.8, tau_e=1.0, dx=dx,
                     bc=P.BC_WALLS_Y)
    gpu.set_state(rho, ux, uy)
    gpu.step(40, dt)
    gr, gux, guy = [t.cpu().numpy() for t in gpu.get_state()]
    assert np.isfinite(r).all()
    assert normwise(gr, r) < 1e-10
    umax = max(np.abs(u[0]).max(), np.abs(u[1]).max())
    assert np.max(np.abs(gux - u[0])) < 1e-9 * umax and np.max(np.abs(guy - u[1])) < 1e-9 * umax


IMPACT_CASES = {
    # T_r, a_l, alpha, W (planar width), v_r, FD dt / dx^2 (App. C: 0.8 for v_r = 1, 0.2 otherwise), t* checked
    "Tr0.5_vr1": (0.5, 0.363, 0.775, 7.0, 1.0, 0.8, (0.25, 0.5, 1.0, 1.5, 2.0)),
    "Tr0.6_vr5": (0.6, 0.387, 0.834, 8.0, 5.0, 0.2, (0.25, 0.5, 1.0, 1.5)),
}


@pytest.mark.parametrize("case", sorted(IMPACT_CASES))
def test_droplet_impact_lbm_agrees_with_the_fd_reference(case):
    """The paper's dynamic comparisons (Sec. IV.B, App. C): a drop (R = 50) hitting a
    liquid film (height 25) on a wall at Re = 112.5 (V_d = 0.075, tau_l = 0.7), Smooth
    C-S with a_v = 2, 600 x 250 lattice, at T_r = 0.5 with v_r = 1 and at T_r = 0.6
    with v_r = 5 (tau(rho) of Eq. RelaxationTime in both methods), against the FD
    scheme on the same domain at dx = 1/2 with the wall layers of Eqs. B1, B2. Up
    to t* = t V_d / D = 1.5 the liquid half-width on the row just above the film
    agrees within 2 nodes (of 60-180) and the phase fields differ by less than 3 %
    of the liquid area; at t* = 2 the phase fields still do."""
    Tr, al, alpha, W, vr, dtf, tstars = IMPACT_CASES[case]
    nx, ny, R, film, V, tau_l = 600, 250, 50.0, 25.0, 0.075, 0.7
    eosp = P.EOSParams(P.EOS_SMOOTH, Tr, al, 2.0, alpha)
    d = P.eos_setup(eosp)
    rv, rl = d["rho_v"], d["rho_l"]
    times = [int(round(ts * 2 * R / V)) for ts in tstars]

    def phase(rho, dx):
        phi = np.clip((rho - rv) / (rl - rv), 0.0, 1.0)
        return phi, (phi[int(round(30.0 / dx))] > 0.5).sum() * dx / 2.0

    sim = P.Simulation(nx, ny, P.BC_WALLS_Y, eosp, P.Relax(kind=P.RELAX_TWO_PHASE, tau_l=tau_l, visc_ratio=vr))
    sim.init_equilibrium(*I.impact(nx, ny, R, film, rv, rl, V, W=W))
    fd = P.FDSolver(2 * nx, 2 * ny, eosp, tau_e=1.0, dx=0.5, bc=P.BC_WALLS_Y, tau_l=tau_l, visc_ratio=vr)
    fd.set_state(*I.impact(2 * nx, 2 * ny, R, film, rv, rl, V, W=W, dx=0.5))
    dt, t = dtf * 0.25, 0
    for ts, T in zip(tstars, times):
        sim.step(T - t)
        fd.step(int(round((T - t) / dt)), dt)
        t = T
        phi_l, half_l = phase(sim.fields()[0].cpu().numpy(), 1.0)
        phi_f, half_f = phase(fd.get_state()[0].cpu().numpy(), 0.5)
        assert np.isfinite(phi_f).all()
        assert np.abs(phi_f[::2, ::2] - phi_l).sum() < 0.03 * phi_l.sum()
        if ts <= 1.5:
            assert abs(half_l - half_f) <= 2.0
    sim.close()
    fd.close()


def test_fd_two_phase_viscosity_with_walls_matches_cpu_oracle():
    """tau_nu(rho) of Eq. RelaxationTime (tau_l = 0.7, v_r = 5) in the FD viscosities,
    with walls, on the GPU against the CPU oracle: 40 steps at dx = 1/2, dt = 0.2 dx^2."""
    nx, ny, dx = 48, 80, 0.5
    oe = E.make_eos(E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834)
    eps = oe.solve_eps(n=40000)
    rho, ux, uy = I.impact(nx, ny, 8.0, 6.0, oe.rho_v, oe.rho_l, 0.02, W=8.0, dx=dx)
    dt = 0.2 * dx * dx
    cpu = F.FDSolver(oe, eps, tau_e=1.0, dx=dx, walls=True, tau_l=0.7, visc_ratio=5.0)
    r, u = cpu.run(rho.copy(), [ux.copy(), uy.copy()], 40 * dt, dt)
    gpu = P.FDSolver(nx, ny, P.EOSParams(P.EOS_SMOOTH, 0.6, 0.387, 2.0, 0.834), tau_e=1.0, dx=dx,
                     bc=P.BC_WALLS_Y, tau_l=0.7, visc_ratio=5.0)
    gpu.set_state(rho, ux, uy)
    gpu.step(40, dt)
    gr, gux, guy = [t.cpu().numpy() for t in gpu.get_state()]
    assert np.isfinite(r).all()
    assert normwise(gr, r) < 1e-10
    umax = max(np.abs(u[0]).max(), np.abs(u[1]).max())
    assert np.max(np.abs(gux - u[0])) < 1e-9 * umax and np.max(np.abs(guy - u[1])) < 1e-9 * umax
