"""Dynamics pin for the oracle: its lattice Boltzmann step against an independent
CPU implementation of the paper's finite-difference scheme (App. A) for the same
macroscopic equations (CPU only).

* single phase: a compressional sound wave in liquid and in vapour evolves the
  same in both (the EOS pressure, bulk viscosity and advection);
* two phases: starting from the lattice Boltzmann method's own equilibrium
  planar interface, the response of density and momentum to a velocity
  perturbation agrees with the FD response (FD grid 1/2, App. B's reference
  spacing). At T_r = 0.8 the agreement is ~1 %; at T_r = 0.6 it is ~5 %, where the
  method's higher-order terms (the paper's subject) grow.
"""
import numpy as np
import pytest

import lbm_inputs as I
from oracle import eos as E
from oracle import fd as F
from oracle import lbm as L

PER = L.BC_PERIODIC_X | L.BC_PERIODIC_Y
LY = 100


def _fd_run(e, eps, rho0, uy0, T, dx):
    n = int(round(LY / dx))
    y = np.arange(LY) * 1.0
    yy = np.arange(n) * dx
    ext = lambda a: np.interp(yy, np.concatenate([y, [LY]]), np.concatenate([a, a[:1]]))
    fds = F.FDSolver(e, eps, dx=dx)
    r, u = fds.run(ext(rho0)[:, None], [np.zeros((n, 1)), ext(uy0)[:, None]], T, 0.8 * dx * dx)
    k = int(round(1 / dx))
    return r[::k, 0], u[1][::k, 0]


@pytest.mark.parametrize("phase", ["liquid", "vapour"])
def test_sound_wave_single_phase_matches_fd(phase):
    e = E.make_eos(E.MODE_SMOOTH, 0.8, 0.5, 0.5, 0.342)
    eps = e.solve_eps()
    rho_bar = e.rho_l if phase == "liquid" else e.rho_v
    y = np.arange(LY) * 1.0
    u0 = 1e-3 * np.sin(2 * np.pi * y / LY)
    lat = L.Lattice(1, LY, PER, e, L.Relax(sigma=e.sigma()))
    f = lat.step(lat.init_equilibrium(np.full((LY, 1), rho_bar), np.zeros((LY, 1)), u0[:, None]), 100)
    rl, _, ul, *_ = lat.macroscopic(f)
    rf, uf = _fd_run(e, eps, np.full(LY, rho_bar), u0, 100, 0.5)
    drho = np.max(np.abs(rl[:, 0] - rho_bar))
    assert np.max(np.abs(rf - rl[:, 0])) < 2e-3 * drho + 1e-15
    assert np.max(np.abs(uf - ul[:, 0])) < 3e-3 * np.max(np.abs(ul))


def test_fd_uniform_rest_state_is_steady():
    e = E.make_eos(E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834)
    fds = F.FDSolver(e, e.solve_eps(), dx=0.5)
    r, u = fds.run(np.full((20, 3), e.rho_l), [np.zeros((20, 3)), np.zeros((20, 3))], 10, 0.2)
    assert np.max(np.abs(r - e.rho_l)) == 0.0 and np.max(np.abs(u[0])) == 0.0


@pytest.mark.parametrize("case,tol", [((0.8, 0.5, 0.5, 0.342), 0.03), ((0.6, 0.387, 2.0, 0.834), 0.10)],
                         ids=["Tr0.8", "Tr0.6"])
def test_interface_response_matches_fd(case, tol):
    Tr, al, av, alpha = case
    e = E.make_eos(E.MODE_SMOOTH, Tr, al, av, alpha)
    eps = e.solve_eps()
    lat = L.Lattice(1, LY, PER, e, L.Relax(sigma=e.sigma()))
    f = lat.step(lat.init_equilibrium(I.planar(1, LY, e.rho_v, e.rho_l, W=10.0)), 3000)
    rho_eq, ux_eq, uy_eq, *_ = lat.macroscopic(f)
    y = np.arange(LY) * 1.0
    du = (2e-3 * np.sin(2 * np.pi * y / LY))[:, None]
    # perturb the equilibrium part only, keeping the method's own non-equilibrium populations
    fp = f + L.equilibrium(rho_eq, ux_eq, uy_eq + du) - L.equilibrium(rho_eq, ux_eq, uy_eq)
    T = 200
    rb, _, ub, *_ = lat.macroscopic(lat.step(f, T))
    rp, _, up, *_ = lat.macroscopic(lat.step(fp, T))
    rfb, ufb = _fd_run(e, eps, rho_eq[:, 0], uy_eq[:, 0], T, 0.5)
    rfp, ufp = _fd_run(e, eps, rho_eq[:, 0], uy_eq[:, 0] + du[:, 0], T, 0.5)
    dl, df = rp[:, 0] - rb[:, 0], rfp - rfb
    ml = rho_eq[:, 0] * (up[:, 0] - ub[:, 0])
    mf = rho_eq[:, 0] * (ufp - ufb)
    assert np.max(np.abs(dl - df)) < tol * np.max(np.abs(dl))
    assert np.max(np.abs(ml - mf)) < tol * np.max(np.abs(ml))


def test_fd_walls_keep_liquid_at_rest():
    """With the wall layers of Eqs. B1, B2 and the reflexive top, uniform liquid at
    rest is a fixed point (every ghost value equals the fluid's, psi_b2 = psi_l)."""
    e = E.make_eos(E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834)
    for dx in (1.0, 0.5):
        fds = F.FDSolver(e, e.solve_eps(), dx=dx, walls=True)
        r, u = fds.run(np.full((24, 3), e.rho_l), [np.zeros((24, 3)), np.zeros((24, 3))], 5, 0.2 * dx * dx)
        assert np.max(np.abs(r - e.rho_l)) == 0.0 and np.max(np.abs(u[0])) == 0.0 and np.max(np.abs(u[1])) == 0.0


@pytest.mark.parametrize("dx", [1.0, 0.5])
def test_fd_walls_are_no_slip_shear_mode_decays_at_the_viscous_rate(dx):
    """No slip at the bottom layer b1 (y = -dx) and, through the reflexive layer, at
    (N - 1/2) dx on top: in uniform liquid the shear mode U = sin(pi (y + dx) / L),
    L = (N + 1/2) dx, decays at nu (pi / L)^2 with nu = (tau_nu - 1/2)/3 (Eq.
    DynamicViscosity). Liquid next to the walls feels no force (psi is uniform, ghost
    layers included)."""
    e = E.make_eos(E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834)
    N = int(round(32 / dx))
    y = np.arange(N) * dx
    L_ = (N + 0.5) * dx
    mode = np.sin(np.pi * (y + dx) / L_)
    fds = F.FDSolver(e, e.solve_eps(), tau_nu=1.0, dx=dx, walls=True)
    dt = 0.2 * dx * dx
    U0 = 1e-4 * np.repeat(mode[:, None], 2, axis=1)
    r, u = fds.run(np.full((N, 2), e.rho_l), [U0, np.zeros((N, 2))], 200, dt)
    amp = (u[0][:, 0] * mode).sum() / (mode * mode).sum()
    rate = -np.log(amp / 1e-4) / 200
    nu = (1.0 - 0.5) / 3.0
    assert rate == pytest.approx(nu * (np.pi / L_) ** 2, rel=5e-3)


@pytest.mark.parametrize("phase", ["liquid", "vapour"])
def test_fd_two_phase_viscosity_shear_waves_decay_at_each_phase_rate(phase):
    """tau_nu(rho) of Eq. RelaxationTime in the FD viscosities (Eq.
    FDviscosityDerivative): a periodic shear wave in uniform liquid decays at
    nu_l k^2, in uniform vapour at nu_v k^2, nu = (tau - 1/2)/3, with tau_l = 0.7
    and tau_v = 1/2 + v_r (tau_l - 1/2) for v_r = 5."""
    e = E.make_eos(E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834)
    tau_l, vr = 0.7, 5.0
    fds = F.FDSolver(e, e.solve_eps(), tau_e=1.0, dx=1.0, tau_l=tau_l, visc_ratio=vr)
    rho = e.rho_l if phase == "liquid" else e.rho_v
    tau = tau_l if phase == "liquid" else 0.5 + vr * (tau_l - 0.5)
    n, k = 64, 2 * np.pi / 64
    mode = np.sin(k * np.arange(n))
    r, u = fds.run(np.full((n, 2), rho), [1e-5 * np.repeat(mode[:, None], 2, axis=1), np.zeros((n, 2))], 100, 0.1)
    amp = (u[0][:, 0] * mode).sum() / (mode * mode).sum()
    assert -np.log(amp / 1e-5) / 100 == pytest.approx((tau - 0.5) / 3.0 * k * k, rel=2e-3)
