"""Pins for the oracle's lattice Boltzmann step (CPU only).

The step is checked against: the velocity-set definitions of the MRT moments,
an independent population-space collision with the Guo forcing written as
Eq. GFS literally, exact conservation and symmetry properties, and the
Chapman-Enskog shear viscosity nu = c_s^2 (tau_nu - 1/2) (Eq. DynamicViscosity).
"""
import numpy as np
import pytest

import lbm_inputs as I
from oracle import eos as E
from oracle import lbm as L

PER = L.BC_PERIODIC_X | L.BC_PERIODIC_Y
WALLS = L.BC_PERIODIC_X | L.BC_WALL_BOTTOM | L.BC_WALL_TOP


@pytest.fixture(scope="module")
def eos06():
    e = E.make_eos(E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834)
    e.solve_eps()
    return e


def test_mrt_rows_are_the_velocity_moments():
    cx, cy = L.C[:, 0].astype(float), L.C[:, 1].astype(float)
    c2 = cx**2 + cy**2
    rows = [np.ones(9), 3 * c2 - 4, (9 * c2**2 - 21 * c2 + 8) / 2, cx, (3 * c2 - 5) * cx, cy,
            (3 * c2 - 5) * cy, cx**2 - cy**2, cx * cy]
    assert np.array_equal(L.M, np.array(rows))
    G = L.M @ L.M.T
    assert np.allclose(G, np.diag(np.diag(G)))         # orthogonal rows
    assert np.allclose(L.MINV @ L.M, np.eye(9), atol=1e-15)
    assert np.allclose(L.W.sum(), 1.0)
    for i in range(9):
        assert np.array_equal(L.C[L.OPP[i]], -L.C[i])


def test_equilibrium_moments_closed_form():
    rng = np.random.default_rng(1)
    rho = rng.uniform(0.01, 0.5, 50)
    ux, uy = rng.uniform(-0.1, 0.1, 50), rng.uniform(-0.1, 0.1, 50)
    meq = L.M @ L.equilibrium(rho, ux, uy)
    u2 = ux**2 + uy**2
    want = np.array([rho, -2 * rho + 3 * rho * u2, rho - 3 * rho * u2, rho * ux, -rho * ux, rho * uy, -rho * uy,
                     rho * (ux**2 - uy**2), rho * ux * uy])
    assert np.allclose(meq, want, rtol=1e-13, atol=1e-16)


def guo_population_collision(f, rho, ux, uy, Fx, Fy, lam):
    """Independent population-space collision (Eqs. OperatorMRT, GFS), dense matrices."""
    Minv = np.linalg.inv(L.M)
    A = Minv @ np.diag(lam) @ L.M
    B = Minv @ (np.eye(9) - np.diag(lam) / 2) @ L.M
    feq = L.equilibrium(rho, ux, uy)
    cs2 = 1.0 / 3.0
    out = np.empty_like(f)
    for n in range(f.shape[1]):
        g = np.empty(9)
        for j in range(9):
            c = L.C[j].astype(float)
            F = np.array([Fx[n], Fy[n]])
            u = np.array([ux[n], uy[n]])
            g[j] = L.W[j] * (c @ F / cs2 + ((np.outer(c, c) - cs2 * np.eye(2)) * np.outer(F, u)).sum() / cs2**2)
        out[:, n] = f[:, n] - A @ (f[:, n] - feq[:, n]) + B @ g
    return out


@pytest.mark.parametrize("taus", [(1, 1, 1, 1, 1, 1), (1.0, 0.8, 1.1, 1.0, 1.2, 0.7), (0.9, 1.3, 0.75, 1.7, 0.6, 1.05)])
def test_collision_sigma0_equals_guo_in_population_space(eos06, taus):
    relax = L.Relax(L.RELAX_MRT, *taus, sigma=0.0)
    lat = L.Lattice(6, 5, PER, eos06, relax)
    rho0 = I.perturbed(I.droplet(6, 5, 1.5, eos06.rho_v, eos06.rho_l, W=3.0), 0.05, 3)
    ux0, uy0 = I.random_velocity((5, 6), 0.02, 4)
    f = lat.init_equilibrium(rho0, ux0, uy0) * (1 + 0.01 * np.random.default_rng(5).uniform(-1, 1, (9, 5, 6)))
    got = lat.collide(f)
    rho, ux, uy, psi, Fx, Fy = lat.macroscopic(f)
    lam = 1.0 / np.array([taus[0], taus[1], taus[2], taus[3], taus[4], taus[3], taus[4], taus[5], taus[5]])
    want = guo_population_collision(f.reshape(9, -1), rho.ravel(), ux.ravel(), uy.ravel(), Fx.ravel(), Fy.ravel(), lam)
    assert np.allclose(got.reshape(9, -1), want, rtol=1e-13, atol=1e-15)


def test_li_sigma_term_adds_only_to_energy_moments(eos06):
    relax0 = L.Relax(L.RELAX_MRT, 1.0, 0.8, 1.2, 1.0, 1.0, 1.0, sigma=0.0)
    relax1 = L.Relax(L.RELAX_MRT, 1.0, 0.8, 1.2, 1.0, 1.0, 1.0, sigma=0.11)
    rho0 = I.planar(3, 40, eos06.rho_v, eos06.rho_l, W=6.0)
    l0, l1 = L.Lattice(3, 40, PER, eos06, relax0), L.Lattice(3, 40, PER, eos06, relax1)
    f = l0.init_equilibrium(rho0)
    d = L.M @ (l1.collide(f) - l0.collide(f)).reshape(9, -1)
    rho, ux, uy, psi, Fx, Fy = l0.macroscopic(f)
    F2 = (Fx**2 + Fy**2).ravel()
    psi2 = psi.ravel() ** 2
    # (1 - 1/(2 tau)) * 12 sigma |F|^2 / (psi^2 (tau - 1/2)) = 12 sigma |F|^2 / (psi^2 tau)
    assert np.allclose(d[1], 12 * 0.11 * F2 / (psi2 * 0.8), rtol=1e-9, atol=1e-15)
    assert np.allclose(d[2], -12 * 0.11 * F2 / (psi2 * 1.2), rtol=1e-9, atol=1e-15)
    assert np.allclose(d[[0, 3, 4, 5, 6, 7, 8]], 0.0, atol=1e-15)


@pytest.mark.parametrize("bc", [PER, WALLS])
def test_mass_is_conserved_to_roundoff(eos06, bc):
    relax = L.Relax(L.RELAX_TWO_PHASE, tau_l=0.6, visc_ratio=3.0, sigma=eos06.sigma())
    lat = L.Lattice(24, 30, bc, eos06, relax)
    if bc == WALLS:
        # the bottom wall's ghost nodes are liquid, so a liquid film lies on it (Sec. IV)
        rho0, ux0, uy0 = I.impact(24, 30, 5, 5, eos06.rho_v, eos06.rho_l, 0.02, W=5.0)
    else:
        rho0 = I.droplet(24, 30, 6, eos06.rho_v, eos06.rho_l, W=5.0)
        ux0, uy0 = I.random_velocity((30, 24), 0.01, 7)
    f = lat.init_equilibrium(rho0, ux0, uy0)
    m0 = f.sum()
    f = lat.step(f, 200)
    assert abs(f.sum() - m0) < 1e-13 * m0


def test_uniform_rest_state_is_fixed_point(eos06):
    lat = L.Lattice(7, 9, PER, eos06, L.Relax(L.RELAX_MRT, 1.0, 0.9, 1.1, 1.0, 1.3, 0.8, sigma=eos06.sigma()))
    rho0 = np.full((9, 7), eos06.rho_l)
    f0 = lat.init_equilibrium(rho0)
    f = lat.step(f0, 50)
    assert np.max(np.abs(f - f0)) < 1e-13 * np.max(f0)   # fixed point up to rounding


def test_translation_invariance_periodic(eos06):
    lat = L.Lattice(16, 12, PER, eos06, L.Relax(sigma=eos06.sigma()))
    rho0 = I.perturbed(I.droplet(16, 12, 4, eos06.rho_v, eos06.rho_l, W=4.0), 0.02, 11)
    f = lat.step(lat.init_equilibrium(rho0), 20)
    g = lat.step(lat.init_equilibrium(np.roll(rho0, (3, 5), axis=(0, 1))), 20)
    assert np.array_equal(np.roll(f, (3, 5), axis=(1, 2)), g)


def test_mirror_symmetry_x(eos06):
    lat = L.Lattice(16, 24, WALLS, eos06, L.Relax(L.RELAX_TWO_PHASE, tau_l=0.7, visc_ratio=2.0, sigma=eos06.sigma()))
    rho0 = I.perturbed(I.impact(16, 24, 4, 4, eos06.rho_v, eos06.rho_l, 0.0, W=4.0)[0], 0.02, 13)
    f = lat.step(lat.init_equilibrium(rho0), 15)
    # reflect x -> -x: node x maps to (nx - 1 - x) is a reflection about a node only up
    # to a shift; use x -> (-x) mod nx, which maps the lattice onto itself
    refl = lambda a: np.roll(a[..., ::-1], 1, axis=-1)
    perm = [0, 3, 2, 1, 4, 6, 5, 8, 7]
    g = lat.step(lat.init_equilibrium(refl(rho0)), 15)
    assert np.allclose(refl(f)[perm], g, rtol=1e-13, atol=1e-17)


def test_shear_wave_decay_gives_chapman_enskog_viscosity():
    """Single phase (uniform rho, so F = 0): u_x = U sin(k y) decays as exp(-nu k^2 t)
    with nu = c_s^2 (tau_nu - 1/2) (Eq. DynamicViscosity)."""
    e = E.make_eos(E.MODE_CS, 0.8, 0.5, 0.5, 0.0)
    ny, nx, U = 64, 1, 1e-4
    for tau_nu in (0.8, 1.2):
        lat = L.Lattice(nx, ny, PER, e, L.Relax(L.RELAX_MRT, 1.0, 1.0, 1.0, 1.0, 1.0, tau_nu, sigma=0.0))
        k = 2 * np.pi / ny
        y = np.arange(ny)[:, None] * np.ones((1, nx))
        rho0 = np.full((ny, nx), e.rho_l)
        f = lat.init_equilibrium(rho0, U * np.sin(k * y), np.zeros_like(rho0))
        a0 = U
        T = 400
        f = lat.step(f, T)
        ux = lat.macroscopic(f)[1][:, 0]
        aT = 2.0 / ny * np.sum(ux * np.sin(k * np.arange(ny)))
        nu_meas = -np.log(aT / a0) / (k**2 * T)
        assert nu_meas == pytest.approx((tau_nu - 0.5) / 3.0, rel=2e-3)


def test_bounce_back_walls_hold_fluid_at_rest():
    """Liquid at rest between walls with the liquid ghost density on both sides stays at rest
    (no-slip walls, half-way bounce-back)."""
    e = E.make_eos(E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834)
    lat = L.Lattice(5, 8, WALLS, e, L.Relax(sigma=e.sigma()))
    lat.psi_ghost_top = lat.psi_ghost_bottom   # liquid on both sides for this check
    f0 = lat.init_equilibrium(np.full((8, 5), e.rho_l))
    f = lat.step(f0, 30)
    assert np.max(np.abs(f - f0)) < 1e-15


def test_two_phase_tau_endpoints():
    e = E.make_eos(E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834)
    relax = L.Relax(L.RELAX_TWO_PHASE, tau_l=0.6, visc_ratio=5.0)
    lam = L.relaxation_rates(relax, np.array([e.rho_v, e.rho_l]), e.rho_v, e.rho_l)
    assert lam[7, 0] == pytest.approx(1 / (0.5 + 5.0 * 0.1), rel=1e-14)
    assert lam[7, 1] == pytest.approx(1 / 0.6, rel=1e-14)
    assert np.all(lam[:7] == 1.0)


@pytest.mark.parametrize("i", [2, 5, 6])
def test_bounce_back_is_no_slip_for_free_streaming_packets(eos06, i):
    """Half-way bounce-back (Sec. IV) reverses the whole velocity at a wall, the
    tangential part included (no slip): a packet streaming freely between the walls
    is back at its starting node with its starting direction after 2 ny steps,
    having moved along x and back. (A specular, free-slip wall would carry a
    diagonal packet 2 ny nodes along x.)"""
    nx, ny, x0, y0 = 16, 5, 3, 1
    lat = L.Lattice(nx, ny, WALLS, eos06, L.Relax())
    f = np.zeros((9, ny, nx))
    f[i, y0, x0] = 1.0
    for _ in range(2 * ny):
        f = lat.stream(f)
        assert f.sum() == 1.0
    want = np.zeros_like(f)
    want[i, y0, x0] = 1.0
    assert np.array_equal(f, want)


def test_wall_ghosts_exert_no_force_on_their_own_phase(eos06):
    """Sec. IV: nodes inside the bottom wall carry the saturated liquid density and
    those inside the top wall the saturated vapour density. A liquid layer on the
    bottom wall and a vapour layer under the top wall then feel no Shan-Chen force
    in the rows next to the walls (their stencils see only their own phase)."""
    nx, ny = 6, 12
    lat = L.Lattice(nx, ny, WALLS, eos06, L.Relax(sigma=eos06.sigma()))
    rho = np.full((ny, nx), eos06.rho_v)
    rho[: ny // 2] = eos06.rho_l
    *_, Fx, Fy = lat.macroscopic(lat.init_equilibrium(rho))
    for row in (0, 1, ny - 2, ny - 1):
        assert np.max(np.abs(Fx[row])) == 0.0 and np.max(np.abs(Fy[row])) < 1e-15 * eos06.rho_l
    assert np.max(np.abs(Fy[ny // 2 - 1])) > 1e-3   # at the interface the force is not zero
