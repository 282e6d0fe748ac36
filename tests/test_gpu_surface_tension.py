"""The surface-tension control (the technique the paper's Sec. V names for keeping
the Weber number when alpha lowers the surface tension; Li & Luo 2013's source
term, pplbm_relax.kappa) on the GPU:

* per-step parity with the oracle (1e-12 normwise) for every collision kind,
  periodic and walled, ragged and degenerate lattices;
* the batch with mixed kappa bitwise equal to single lattices, every plan;
* the FD solver's counterpart (pplbm_fd_set_surface_tension) against the CPU FD
  oracle (1e-10), periodic and walled;
* physics at sizes the oracle cannot reach: the Laplace-law surface tension
  scales by (1 - kappa) and matches the planar (1 - kappa) Eq. SurfaceTension;
  kappa chosen by the Sec. V recipe restores the C-S surface tension for a Smooth
  C-S of smaller alpha; an oscillating droplet's period grows by 1/sqrt(1 - kappa)
  and its history agrees with the FD solver carrying the same term.
"""
import numpy as np
import pytest

import lbm_inputs as I
from gpu_helpers import BC_PER, BC_WALLS, make_pair, normwise
from oracle import eos as E
from oracle import fd as F

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2107_06355_gb300")
from paper_2107_06355_gb300 import sweeps as S  # noqa: E402

SMOOTH06 = (E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834)
RELAX = {
    "unit": {},
    "shear_const": {"tau_nu": 0.7},
    "two_phase": {"kind": 1, "tau_l": 0.6, "visc_ratio": 3.0},
    "full_mrt": {"tau_rho": 1.0, "tau_e": 0.8, "tau_zeta": 1.1, "tau_j": 1.0, "tau_q": 1.2, "tau_nu": 0.7},
}


def _state(nx, ny, bc, e, seed):
    if bc == BC_WALLS:
        R = max(2.0, min(nx, ny) / 6)
        rho, ux, uy = I.impact(nx, ny, R, max(2, ny // 6), e.rho_v, e.rho_l, 0.03, W=5.0)
    else:
        rho = I.droplet(nx, ny, max(1.5, min(nx, ny) / 4), e.rho_v, e.rho_l, W=5.0)
        ux, uy = I.random_velocity((ny, nx), 0.01, seed + 1)
    return I.perturbed(rho, 0.01, seed), ux, uy


@pytest.mark.parametrize("kappa", [0.5, -0.7])
@pytest.mark.parametrize("relax", list(RELAX))
@pytest.mark.parametrize("shape,bc", [((70, 19), BC_PER), ((70, 27), BC_WALLS), ((33, 9), BC_WALLS),
                                      ((3, 3), BC_PER)])
def test_step_parity_with_kappa(kappa, relax, shape, bc):
    nx, ny = shape
    olat, sim = make_pair(nx, ny, bc, SMOOTH06, dict(RELAX[relax], kappa=kappa))
    rho, ux, uy = _state(nx, ny, bc, olat.eos, 23)
    f = olat.init_equilibrium(rho, ux, uy)
    sim.init_equilibrium(rho, ux, uy)
    f0 = f
    for nsteps in (1, 9):
        f = olat.step(f, nsteps)
        sim.step(nsteps)
        sim.sync()
        err = normwise(sim.get_f().cpu().numpy(), f)
        assert err < 1e-12 * max(1, nsteps / 2), (nsteps, err)
    # the source is active: the same run without it differs far above the tolerance
    olat.relax.kappa = 0.0
    assert normwise(olat.step(f0, 10), f) > 1e-6
    sim.close()


@pytest.mark.parametrize("relax", ["unit", "two_phase"])
def test_step_parity_with_kappa_and_guo_forcing(relax):
    """With the Guo scheme (sigma = 0) the Li term's z is zero and the source alone
    fills it. Plain C-S at T_r = 0.8, where Guo forcing is stable (Sec. III.A)."""
    cs08 = (E.MODE_CS, 0.8, 0.5, 0.5, 0.0)
    olat, sim = make_pair(40, 24, BC_PER, cs08, dict(RELAX[relax], kappa=0.4), forcing_li=False)
    rho, ux, uy = _state(40, 24, BC_PER, olat.eos, 31)
    f = olat.init_equilibrium(rho, ux, uy)
    sim.init_equilibrium(rho, ux, uy)
    f = olat.step(f, 8)
    sim.step(8)
    sim.sync()
    assert normwise(sim.get_f().cpu().numpy(), f) < 4e-12
    sim.close()


@pytest.mark.parametrize("mode,width", [(0, 0), (0, 8), (1, 0), (2, 0), (3, 0)])
def test_batch_with_mixed_kappa_bitwise_equals_single_lattices(mode, width):
    inst = [(4, 90, BC_PER, 0.8, 0.0), (70, 45, BC_PER, 0.6, 0.5), (33, 33, BC_PER, 0.5, -0.4),
            (48, 40, BC_WALLS, 0.6, 0.3), (3, 5, BC_PER, 0.6, 0.0), (130, 9, BC_WALLS, 0.5, 0.0)]
    eos = [P.EOSParams(P.EOS_SMOOTH, Tr, 0.363, 2.0, 0.775) for (_, _, _, Tr, _) in inst]
    relax = [P.Relax(kappa=k) for (*_, k) in inst]
    b = P.Batch([(nx, ny, bc) for (nx, ny, bc, _, _) in inst], eos, relax)
    sims = []
    for k, (nx, ny, bc, Tr, kap) in enumerate(inst):
        s = P.Simulation(nx, ny, bc, eos[k], relax[k])
        d = s.derived()
        if bc == BC_WALLS:
            rho, ux, uy = I.impact(nx, ny, max(2.0, min(nx, ny) / 6), max(2, ny // 6), d["rho_v"], d["rho_l"], 0.03,
                                   W=5.0)
        else:
            rho = I.perturbed(I.droplet(nx, ny, max(1.0, min(nx, ny) / 4), d["rho_v"], d["rho_l"], W=5.0), 0.01, k)
            ux, uy = I.random_velocity((ny, nx), 0.01, k + 1)
        s.init_equilibrium(rho, ux, uy)
        b.init_equilibrium(k, rho, ux, uy)
        sims.append(s)
    b.set_plan(mode, width)
    for nsteps in (1, 6, 7):
        b.step(nsteps)
        for s in sims:
            s.step(nsteps)
        assert b.sync() > 0
        for k, s in enumerate(sims):
            assert torch.equal(b.get_f(k), s.get_f()), (k, nsteps)
    b.close()
    for s in sims:
        s.close()


@pytest.mark.parametrize("shape,dx,walls", [((48, 40), 1.0, False), ((37, 29), 0.5, False), ((48, 80), 0.5, True)])
def test_fd_with_kappa_matches_cpu_oracle(shape, dx, walls):
    nx, ny = shape
    kappa = 0.5
    oe = E.make_eos(E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834)
    eps = oe.solve_eps(n=40000)
    if walls:
        rho, ux, uy = I.impact(nx, ny, 8.0, 6.0, oe.rho_v, oe.rho_l, 0.02, W=8.0, dx=dx)
    else:
        rho = I.droplet(nx, ny, min(nx, ny) / 4, oe.rho_v, oe.rho_l, W=6.0 / dx)
        ux, uy = I.random_velocity((ny, nx), 0.004, 3)
    dt = 0.4 * dx * dx
    cpu = F.FDSolver(oe, eps, tau_nu=0.8, tau_e=1.0, dx=dx, walls=walls, kappa=kappa)
    r, u = cpu.run(rho.copy(), [ux.copy(), uy.copy()], 40 * dt, dt)
    gpu = P.FDSolver(nx, ny, P.EOSParams(P.EOS_SMOOTH, 0.6, 0.387, 2.0, 0.834), tau_nu=0.8, tau_e=1.0, dx=dx,
                     bc=P.BC_WALLS_Y if walls else P.BC_PERIODIC, kappa=kappa)
    gpu.set_state(rho, ux, uy)
    gpu.step(40, dt)
    gr, gux, guy = [t.cpu().numpy() for t in gpu.get_state()]
    assert np.isfinite(r).all()
    assert normwise(gr, r) < 1e-10
    umax = max(np.abs(u[0]).max(), np.abs(u[1]).max())
    assert np.max(np.abs(gux - u[0])) < 1e-9 * umax and np.max(np.abs(guy - u[1])) < 1e-9 * umax
    # the term is active: without it the FD state differs well above the tolerance
    r0, _ = F.FDSolver(oe, eps, tau_nu=0.8, tau_e=1.0, dx=dx, walls=walls).run(rho.copy(), [ux.copy(), uy.copy()],
                                                                               40 * dt, dt)
    assert normwise(r0, r) > 1e-7
    gpu.close()


RADII = (24.0, 32.0, 48.0)


def test_laplace_law_surface_tension_scales_by_one_minus_kappa():
    """Droplets R = 24, 32, 48 on 192^2 (T_r = 0.6 Smooth C-S, alpha = 0.834), 60,000
    steps: the Laplace-law fit with kappa = 0.5 is half the kappa = 0 one (within 2 %),
    every radius within 3 %, and each agrees with the planar (1 - kappa) Eq.
    SurfaceTension within 4 %."""
    eosp = P.EOSParams(P.EOS_SMOOTH, 0.6, 0.387, 2.0, 0.834)
    kappa = 0.5
    cases = [(eosp, P.Relax()), (eosp, P.Relax(kappa=kappa))]
    lap = S.laplace_law(cases, RADII, n=192, steps=60000)
    planar = S.planar_coexistence(cases)
    assert not any(c["diverged"] for c in lap)
    g0, gk = lap[0]["gamma"], lap[1]["gamma"]
    assert abs(gk / g0 / (1 - kappa) - 1) < 0.02, (g0, gk)
    for a, c in zip(lap[0]["dpR"], lap[1]["dpR"]):
        assert abs(c / a / (1 - kappa) - 1) < 0.03
    # the planar profile is the same (Q_yy = 3 Q_xx for a 1-D profile): only the factor differs
    assert planar[1]["gamma"] == pytest.approx((1 - kappa) * planar[0]["gamma"], rel=1e-7)
    for c, p in zip(lap, planar):
        assert abs(c["gamma"] / p["gamma"] - 1) < 0.04, (c["gamma"], p["gamma"])


def test_kappa_restores_the_cs_surface_tension_for_a_smaller_alpha():
    """Sec. V's proposal: lowering alpha lowers the Smooth C-S surface tension (and so
    changes the Weber number); kappa = 1 - gamma_CS / gamma_alpha (planar values)
    restores it. T_r = 0.6: C-S a = 0.387 against Smooth C-S alpha = 0.5 (a_l = 0.387,
    a_v = 2; planar gamma 4.9e-3 against 6.3e-3 in the oracle, so kappa ~ -0.3); the
    droplets' Laplace fits then agree within 3 %, against a 15 % mismatch or more
    without the control."""
    cs = (P.EOSParams(P.EOS_CS, 0.6, 0.387, 0.387, 0.5), P.Relax())
    sm = (P.EOSParams(P.EOS_SMOOTH, 0.6, 0.387, 2.0, 0.5), P.Relax())
    planar = S.planar_coexistence([cs, sm])
    g_cs, g_sm = planar[0]["gamma"], planar[1]["gamma"]
    assert g_sm < 0.85 * g_cs
    kappa = S.kappa_for_surface_tension(g_cs, g_sm)
    assert kappa < 0
    sm_k = (sm[0], P.Relax(kappa=kappa))
    lap = S.laplace_law([cs, sm, sm_k], RADII, n=192, steps=60000)
    assert not any(c["diverged"] for c in lap)
    assert lap[1]["gamma"] < 0.85 * lap[0]["gamma"]
    assert abs(lap[2]["gamma"] / lap[0]["gamma"] - 1) < 0.03, (lap[0]["gamma"], lap[2]["gamma"])


def _ellipse(n, R, eps, rv, rl, W, dx):
    y, x = np.mgrid[0:n, 0:n].astype(np.float64) * dx
    c = n * dx / 2
    a, b = R * (1 + eps), R / (1 + eps)
    r = np.sqrt(((x - c) / a) ** 2 + ((y - c) / b) ** 2) * R
    return rv + (rl - rv) * 0.5 * (1 - np.tanh(4.6 * (r - R) / W))


def _deformation(rho, rv, rl, dx):
    n = rho.shape[0]
    phi = np.clip((rho - rv) / (rl - rv), 0.0, 1.0)
    y, x = np.mgrid[0:n, 0:n].astype(np.float64) * dx
    m = phi.sum()
    cx, cy = (phi * x).sum() / m, (phi * y).sum() / m
    sx, sy = np.sqrt((phi * (x - cx) ** 2).sum() / m), np.sqrt((phi * (y - cy) ** 2).sum() / m)
    return (sx - sy) / (sx + sy)


def _crossings(h, times):
    k = np.nonzero(np.sign(h[1:]) != np.sign(h[:-1]))[0]
    return times[k] + (times[1] - times[0]) * h[k] / (h[k] - h[k + 1])


def test_oscillating_droplet_period_and_fd_agreement_with_kappa():
    """An elliptic droplet (R = 30, semi-axes R (1 +- 0.15), T_r = 0.6 Smooth C-S,
    tau = 1, 128^2) oscillates with an undamped frequency ~ sqrt(gamma / (rho R^3)):
    with kappa = 0.5 it falls by sqrt(1 - kappa). Viscous damping (beta, the same for
    both) lowers the observed frequency sqrt(w0^2 - beta^2) more for the slower
    oscillation, so the half period between zero crossings grows by at least
    1/sqrt(1 - kappa) = 1.414 (measured 1.50); the test takes that bound and at most
    10 % above it. The LBM history agrees with the FD solver (dx = 1/2) carrying the
    same term to 0.02 in deformation (amplitude 0.14; measured 0.015)."""
    L_, R, ecc, W, T, every = 128, 30.0, 0.15, 8.0, 6000, 100
    eosp = P.EOSParams(P.EOS_SMOOTH, 0.6, 0.387, 2.0, 0.834)
    d = P.eos_setup(eosp)
    rv, rl = d["rho_v"], d["rho_l"]
    times = np.arange(0, T + 1, every, dtype=np.float64)
    hist = {}
    for kappa in (0.0, 0.5):
        sim = P.Simulation(L_, L_, P.BC_PERIODIC, eosp, P.Relax(kappa=kappa))
        sim.init_equilibrium(_ellipse(L_, R, ecc, rv, rl, W, 1.0))
        h = []
        for t in times:
            if t:
                sim.step(every)
            h.append(_deformation(sim.fields()[0].cpu().numpy(), rv, rl, 1.0))
        sim.close()
        hist[kappa] = np.array(h)
    dx = 0.5
    n = int(L_ / dx)
    s = P.FDSolver(n, n, eosp, dx=dx, tau_nu=1.0, tau_e=1.0, kappa=0.5)
    z = np.zeros((n, n))
    s.set_state(_ellipse(n, R, ecc, rv, rl, W, dx), z, z)
    dt = 0.4 * dx * dx
    fd = []
    for t in times:
        if t:
            s.step(int(round(every / dt)), dt)
        fd.append(_deformation(s.get_state()[0].cpu().numpy(), rv, rl, dx))
    s.close()
    fd = np.array(fd)
    assert np.max(np.abs(hist[0.5] - fd)) < 0.02
    c0, ck = _crossings(hist[0.0], times), _crossings(hist[0.5], times)
    assert len(c0) >= 3 and len(ck) >= 2
    half0 = np.mean(np.diff(c0[:3]))
    halfk = np.mean(np.diff(ck[:2])) if len(ck) < 3 else np.mean(np.diff(ck[:3]))
    r = halfk / half0 * np.sqrt(1 - 0.5)
    assert 1.0 <= r < 1.1, (half0, halfk)


def test_weber_matching_keeps_the_cs_surface_tension_at_the_cs_width():
    """Sec. V across T_r (sweeps.weber_matching): the Smooth C-S set to the C-S
    interface width (a = 0.363, alpha tuned as in the stability study) has a lower
    surface tension (Table DropImpactParameters at T_r = 0.5: 8.3e-3 against 8.9e-3);
    kappa = 1 - gamma_CS / gamma_alpha restores it, checked on static droplets
    (Laplace fits within 3 % of C-S at T_r = 0.5 and 0.6)."""
    res = S.weber_matching((0.5, 0.6))
    assert set(res) == {0.5, 0.6}
    assert res[0.5]["gamma_alpha"] < 0.96 * res[0.5]["gamma_cs"]
    for Tr, v in res.items():
        assert v["kappa"] < 0
        assert v["laplace_cs"] and v["laplace_matched"], (Tr, v)
        assert abs(v["laplace_matched"] / v["laplace_cs"] - 1) < 0.03, (Tr, v)


@pytest.mark.parametrize("kappa", [0.5, -0.5])
def test_droplet_impact_with_kappa_lbm_agrees_with_the_fd_reference(kappa):
    """The paper's impact comparison (Sec. IV.B, App. C: R = 50 drop on a film of
    height 25, 600 x 250, Re = 112.5, Smooth C-S at T_r = 0.5, v_r = 1) with the
    surface-tension control in both the LBM and the FD reference (dx = 1/2): the
    phase fields stay within 3 % of the liquid area of each other up to t* = 3 and
    the half-widths on the row above the film within 2 nodes up to t* = 1.5
    (measured: 0.8-2.3 % and <= 1.25 nodes), while the control itself changes the
    LBM phase field by more than 5 % from t* = 1.5 on (measured 7-12 % at
    kappa = -0.5 and 12-30 % at kappa = 0.5, where the lower surface tension lets the
    crown rise higher)."""
    Tr, al, alpha, W, vr, dtf = 0.5, 0.363, 0.775, 7.0, 1.0, 0.8
    tstars = (0.25, 0.5, 1.0, 1.5, 2.0, 3.0)
    nx, ny, R, film, V, tau_l = 600, 250, 50.0, 25.0, 0.075, 0.7
    eosp = P.EOSParams(P.EOS_SMOOTH, Tr, al, 2.0, alpha)
    d = P.eos_setup(eosp)
    rv, rl = d["rho_v"], d["rho_l"]

    def phase(rho, dx):
        phi = np.clip((rho - rv) / (rl - rv), 0.0, 1.0)
        return phi, (phi[int(round(30.0 / dx))] > 0.5).sum() * dx / 2.0

    def relax(k):
        return P.Relax(kind=P.RELAX_TWO_PHASE, tau_l=tau_l, visc_ratio=vr, kappa=k)

    sim, sim0 = (P.Simulation(nx, ny, P.BC_WALLS_Y, eosp, relax(k)) for k in (kappa, 0.0))
    for s in (sim, sim0):
        s.init_equilibrium(*I.impact(nx, ny, R, film, rv, rl, V, W=W))
    fd = P.FDSolver(2 * nx, 2 * ny, eosp, tau_e=1.0, dx=0.5, bc=P.BC_WALLS_Y, tau_l=tau_l, visc_ratio=vr,
                    kappa=kappa)
    fd.set_state(*I.impact(2 * nx, 2 * ny, R, film, rv, rl, V, W=W, dx=0.5))
    dt, t = dtf * 0.25, 0
    for ts in tstars:
        T = int(round(ts * 2 * R / V))
        sim.step(T - t)
        sim0.step(T - t)
        fd.step(int(round((T - t) / dt)), dt)
        t = T
        phi_l, half_l = phase(sim.fields()[0].cpu().numpy(), 1.0)
        phi_0, _ = phase(sim0.fields()[0].cpu().numpy(), 1.0)
        phi_f, half_f = phase(fd.get_state()[0].cpu().numpy(), 0.5)
        assert np.isfinite(phi_f).all()
        assert np.abs(phi_f[::2, ::2] - phi_l).sum() < 0.03 * phi_l.sum(), ts
        if ts <= 1.5:
            assert abs(half_l - half_f) <= 2.0, (ts, half_l, half_f)
        if ts >= 1.5:
            assert np.abs(phi_l - phi_0).sum() > 0.05 * phi_l.sum(), ts
    for o in (sim, sim0, fd):
        o.close()
