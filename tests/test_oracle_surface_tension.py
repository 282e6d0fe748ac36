"""Pins for the surface-tension control in the oracle (CPU only).

The paper's discussion (Sec. V) names Li & Luo's technique (Phys. Rev. E 88,
053307, 2013) as the way to keep the Weber number when lowering alpha lowers the
surface tension: a source C added to the post-collision moments,
C = [0, 1.5 l_e tr Q, -1.5 l_zeta tr Q, 0, 0, 0, 0, -l_nu (Q_xx - Q_yy), -l_nu Q_xy],
Q_ab = kappa (G/2) psi(x) sum_i w_i [psi(x + c_i) - psi(x)] c_ia c_ib.
What fixes it here, independently of how the oracle writes it:

* the stencil: for a quadratic psi the sum is exact, Q = kappa (G/12) psi
  (delta lap psi + 2 d_a d_b psi) (the weights' fourth moment is (1/3) of the
  symmetrised delta delta);
* special cases and invariants: kappa = 0 is the plain step, the change is linear
  in kappa, mass and momentum are conserved for every relaxation;
* with unit relaxation times the equilibrium shift -Q + (3/4) tr(Q) I appears in the
  post-collision second moments as it stands, and the third-order moments do not
  change;
* the normal component of that shift vanishes for any 1-D profile on the lattice
  (Q_yy = 3 Q_xx there), so a planar interface evolves identically at unit
  relaxation times (Eq. VaporLiqEq, the coexistence, is untouched);
* Laplace's law: the pressure jump of a droplet times its radius, i.e. the surface
  tension of Eq. IntegralSurfaceTension, scales by (1 - kappa);
* dynamics: the response of an equilibrium droplet to kappa agrees with the
  independent finite-difference solver (App. A) carrying the same term in its
  pressure tensor (grid 1/2, T_r = 0.8).
"""
import numpy as np
import pytest

import lbm_inputs as I
from oracle import eos as E
from oracle import fd as F
from oracle import lbm as L

PER = L.BC_PERIODIC_X | L.BC_PERIODIC_Y


def _eos06():
    e = E.make_eos(E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834)
    e.solve_eps()
    return e


def _noisy_droplet(e, n=16, seed=3):
    rng = np.random.default_rng(seed)
    rho = I.droplet(n, n, n / 4, e.rho_v, e.rho_l, W=6.0) * (1 + 0.01 * rng.standard_normal((n, n)))
    ux = 0.01 * rng.standard_normal((n, n))
    uy = 0.01 * rng.standard_normal((n, n))
    f = L.equilibrium(rho, ux, uy)
    return f * (1 + 0.002 * rng.standard_normal(f.shape))


RELAXES = {
    "unit": lambda e: L.Relax(sigma=e.sigma()),
    "mrt": lambda e: L.Relax(sigma=e.sigma(), tau_e=0.8, tau_zeta=1.1, tau_j=1.0, tau_q=1.2, tau_nu=0.9),
    "two_phase": lambda e: L.Relax(kind=L.RELAX_TWO_PHASE, tau_l=0.7, visc_ratio=5.0, sigma=e.sigma()),
}


def _with_kappa(r, kappa):
    r.kappa = kappa
    return r


def test_q_is_exact_for_a_quadratic_psi():
    n = 12
    y, x = np.mgrid[0:n, 0:n] + 0.0
    a0, bx, by, dxx, dxy, dyy = 2.0, 0.03, -0.02, 1.5e-3, -7e-4, 2.2e-3
    psi = a0 + bx * x + by * y + dxx * x * x + dxy * x * y + dyy * y * y
    G, kappa = -1.0, 0.37
    qxx, qyy, qxy = L.surface_tension_q(psi, G, kappa, PER)
    lap = 2 * dxx + 2 * dyy
    c = kappa * G / 12.0 * psi
    inner = (slice(2, -2), slice(2, -2))  # np.roll wraps at the edges, where psi is not quadratic
    assert np.allclose(qxx[inner], (c * (lap + 2 * 2 * dxx))[inner], rtol=1e-12, atol=0)
    assert np.allclose(qyy[inner], (c * (lap + 2 * 2 * dyy))[inner], rtol=1e-12, atol=0)
    assert np.allclose(qxy[inner], (c * 2 * dxy)[inner], rtol=1e-12, atol=0)


@pytest.mark.parametrize("kind", sorted(RELAXES))
def test_kappa_is_linear_zero_is_the_plain_step_and_mass_momentum_are_kept(kind):
    e = _eos06()
    f = _noisy_droplet(e)
    lat = {k: L.Lattice(16, 16, PER, e, _with_kappa(RELAXES[kind](e), k)) for k in (0.0, 0.4, 0.8)}
    base = L.Lattice(16, 16, PER, e, RELAXES[kind](e)).collide(f)
    assert np.array_equal(lat[0.0].collide(f), base)
    d4 = lat[0.4].collide(f) - base
    d8 = lat[0.8].collide(f) - base
    assert np.abs(d8).max() > 1e-3
    tol = 1e-14 * np.abs(base).max()  # rounding of M^-1 m* (measured: 1e-16)
    assert np.abs(d8 - 2 * d4).max() < tol
    assert np.abs(d8.sum(0)).max() < tol
    for a in range(2):
        assert np.abs(np.einsum("i,iyx->yx", L.C[:, a].astype(float), d8)).max() < tol


def test_unit_tau_second_moments_shift_by_minus_q_plus_three_quarters_trace():
    e = _eos06()
    f = _noisy_droplet(e)
    kappa = 0.6
    d = (L.Lattice(16, 16, PER, e, L.Relax(sigma=e.sigma(), kappa=kappa)).collide(f)
         - L.Lattice(16, 16, PER, e, L.Relax(sigma=e.sigma())).collide(f))
    rho = f.sum(0)
    qxx, qyy, qxy = L.surface_tension_q(e.psi(rho), e.G, kappa, PER)
    tr = qxx + qyy
    cx, cy = L.C[:, 0].astype(float), L.C[:, 1].astype(float)
    mom = lambda w: np.einsum("i,iyx->yx", w, d)
    tol = 1e-12 * np.abs(tr).max() + 1e-17
    assert np.abs(mom(cx * cx) - (-qxx + 0.75 * tr)).max() < tol
    assert np.abs(mom(cy * cy) - (-qyy + 0.75 * tr)).max() < tol
    assert np.abs(mom(cx * cy) - (-qxy)).max() < tol
    # third-order moments (heat-flux rows of Eq. MatrixMRT) are untouched
    assert np.abs(mom(cx * cy * cy)).max() < tol and np.abs(mom(cy * cx * cx)).max() < tol


def test_planar_interface_evolves_identically_at_unit_tau():
    e = _eos06()
    out = {}
    for kappa in (0.0, 0.5, -0.5):
        lat = L.Lattice(1, 100, PER, e, L.Relax(sigma=e.sigma(), kappa=kappa))
        out[kappa] = lat.macroscopic(lat.step(lat.init_equilibrium(I.planar(1, 100, e.rho_v, e.rho_l, W=10.0)), 500))
    for kappa in (0.5, -0.5):
        # rounding only (measured 2.5e-15 in rho ~ 0.4 and in u_y ~ 7e-3); an O(kappa) change is ~1e-4
        assert np.abs(out[kappa][0] - out[0.0][0]).max() < 1e-12
        assert np.abs(out[kappa][2] - out[0.0][2]).max() < 1e-13


def _droplet_dp_r(e, kappa, R, n=64):
    """dp R of a static droplet (dp = p_EOS(centre) - p_EOS(corner), R equimolar);
    e None: the T_r = 0.6 Smooth C-S (so spawned workers build it themselves)."""
    e = _eos06() if e is None else e
    lat = L.Lattice(n, n, PER, e, L.Relax(sigma=e.sigma(), kappa=kappa))
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
    req = float(np.sqrt(((rho - rout) / (rin - rout)).sum() / np.pi))
    return float(e.pressure(rin) - e.pressure(rout)) * req


def test_laplace_law_surface_tension_scales_by_one_minus_kappa():
    import multiprocessing
    from concurrent.futures import ProcessPoolExecutor

    kappa = 0.5
    jobs = [(k, R) for R in (10, 14) for k in (0.0, kappa)]
    # the four droplets are independent: side by side in spawned processes
    with ProcessPoolExecutor(max_workers=4, mp_context=multiprocessing.get_context("spawn")) as ex:
        dpr = dict(zip(jobs, ex.map(_droplet_dp_r, [None] * 4, [k for k, _ in jobs], [R for _, R in jobs])))
    for R in (10, 14):
        ratio = dpr[(kappa, R)] / dpr[(0.0, R)]
        assert abs(ratio / (1 - kappa) - 1) < 0.03, (R, ratio)


def _half_grid(a):
    """Periodic linear interpolation of a lattice field onto the grid of spacing 1/2."""
    n = a.shape[0]
    yy = np.arange(2 * n) * 0.5
    ext = lambda v: np.concatenate([v, v[:1]])
    a1 = np.array([np.interp(yy, np.arange(n + 1), ext(a[:, j])) for j in range(a.shape[1])]).T
    return np.array([np.interp(yy, np.arange(n + 1), ext(a1[i])) for i in range(2 * n)])


def test_droplet_response_to_kappa_matches_fd():
    e = E.make_eos(E.MODE_SMOOTH, 0.8, 0.5, 0.5, 0.342)
    eps = e.solve_eps()
    n = 32
    lat0 = L.Lattice(n, n, PER, e, L.Relax(sigma=e.sigma()))
    f = lat0.init_equilibrium(I.droplet(n, n, 9.0, e.rho_v, e.rho_l, W=8.0))
    prev = f.sum(0)
    for _ in range(100):
        f = lat0.step(f, 100)
        rho = f.sum(0)
        r = L.convergence_residual(rho, prev)
        prev = rho
        if r < 1e-10:
            break
    rho_eq, ux_eq, uy_eq, *_ = lat0.macroscopic(f)
    T, kappa = 50, 0.5
    lb, fd = {}, {}
    for k in (0.0, kappa):
        lat = L.Lattice(n, n, PER, e, L.Relax(sigma=e.sigma(), kappa=k))
        lb[k] = lat.macroscopic(lat.step(f, T))[:3]
        r, u = F.FDSolver(e, eps, dx=0.5, kappa=k).run(_half_grid(rho_eq), [_half_grid(ux_eq), _half_grid(uy_eq)],
                                                       T, 0.1)
        fd[k] = (r[::2, ::2], u[0][::2, ::2], u[1][::2, ::2])
    for c in range(3):
        dl = lb[kappa][c] - lb[0.0][c]
        df = fd[kappa][c] - fd[0.0][c]
        assert np.abs(dl).max() > 1e-4
        assert np.abs(dl - df).max() < 0.06 * np.abs(dl).max(), c
