"""The per-M-step guards (single lattice: pplbm_guard; batch: pplbm_batch_guard)
against the oracle stepped from the same seeded state.

Each guard reports the total mass, the largest fluid speed |u| with
u = (j + F/2)/rho (Eq. Momentum), the number of non-finite or non-positive
densities and the residual sum |rho(t) - rho(t')| / sum |rho(t)| against the
density at its previous call; called every 100 steps that residual is the
convergence criterion of Sec. III.A (paragraph after Eq. PlanarIntDensity). The
expected values come from oracle.lbm: Lattice.macroscopic for rho and u,
convergence_residual for the residual.

Tolerances (derived from the per-step parity bound, normwise 1e-12 on f):
  mass: a sum of densities each within ~1e-12 relative, so rel 1e-12;
  max |u|: |du| <= (|dj| + |dF|/2)/rho + |u| |drho|/rho; with errors of a few 1e-13
    of max f and rho >= rho_v (about 0.3 max rho at these temperatures... down to
    1e-2 of it) this stays below 1e-10 absolute;
  residual: |d res| <= 2 max|drho| / mean(rho) + res max|drho|/rho, below 1e-10
    absolute for these states.
"""
import numpy as np
import pytest

import lbm_inputs as I
from gpu_helpers import BC_PER, BC_WALLS, make_pair
from oracle import eos as E
from oracle import lbm as OL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SMOOTH06 = (E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834)
SMOOTH05 = (E.MODE_SMOOTH, 0.5, 0.363, 2.0, 0.775)
CS07 = (E.MODE_CS, 0.7, 0.387, 0.387, 0.0)

MASS_REL = 1e-12
U_ABS = 1e-10
RES_ABS = 1e-10


def _oracle_guard(olat, f, rho_prev):
    rho, ux, uy, _, _, _ = olat.macroscopic(f)
    res = -1.0 if rho_prev is None else OL.convergence_residual(rho, rho_prev)
    return float(rho.sum()), float(np.hypot(ux, uy).max()), res, rho


def _initial(kind, nx, ny, e, seed):
    if kind == "planar":
        rho = I.perturbed(I.planar(nx, ny, e.rho_v, e.rho_l, W=8.0), 1e-3, seed)
        return rho, None, None
    if kind == "droplet":
        rho = I.perturbed(I.droplet(nx, ny, min(nx, ny) / 4.0, e.rho_v, e.rho_l, W=7.0), 1e-3, seed)
        ux, uy = I.random_velocity((ny, nx), 1e-3, seed + 1)
        return rho, ux, uy
    return I.impact(nx, ny, 7, 6, e.rho_v, e.rho_l, 0.04, W=6.0)


def _check(got, want, what):
    mass, umax, bad, res = got
    wm, wu, wr = want
    assert bad == 0, what
    assert mass == pytest.approx(wm, rel=MASS_REL), what
    assert abs(umax - wu) <= U_ABS, (what, umax, wu)
    if wr < 0:
        assert res == -1.0, what
    else:
        assert abs(res - wr) <= RES_ABS, (what, res, wr)


CASES = [
    ("droplet", 64, 56, BC_PER, SMOOTH06, {}),
    ("planar", 4, 200, BC_PER, SMOOTH05, {"tau_e": 0.9, "tau_nu": 0.8, "tau_q": 1.1}),
    ("impact", 72, 40, BC_WALLS, SMOOTH06, {"kind": 1, "tau_l": 0.6, "visc_ratio": 3.0}),
    ("impact", 48, 36, BC_WALLS, CS07, {}),
]


@pytest.mark.parametrize("case", CASES, ids=["droplet_unit", "planar_mrt", "impact_two_phase", "impact_cs_walls"])
def test_single_lattice_guard_matches_oracle(case):
    kind, nx, ny, bc, eos_case, relax = case
    olat, sim = make_pair(nx, ny, bc, eos_case, relax)
    rho0, ux0, uy0 = _initial(kind, nx, ny, olat.eos, 11)
    f = olat.init_equilibrium(rho0, ux0, uy0)
    sim.init_equilibrium(rho0, ux0, uy0)
    prev = None
    # the Sec. III.A rhythm: a guard every 100 steps, then a short interval
    for nsteps in (0, 100, 100, 7):
        if nsteps:
            f = olat.step(f, nsteps)
            sim.step(nsteps)
        wm, wu, wr, prev = _oracle_guard(olat, f, prev)
        _check(sim.guard(), (wm, wu, wr), (kind, nsteps))
    # set_f restarts the residual; planted non-physical nodes are counted, left out of
    # the mass, and make the call return PPLBM_ERR_DIVERGED (the outputs are written)
    import ctypes as C
    from paper_2107_06355_gb300 import _lib as L

    fb = f.copy()
    fb[:, 3, 1] = -1.0
    fb[:, ny - 1, 0] = np.nan
    sim.set_f(fb)
    rho = fb.sum(axis=0)
    good = np.isfinite(rho) & (rho > 0)
    out = (C.c_double * 4)()
    assert L.lib().pplbm_guard(sim.ctx, out) == L.PPLBM_ERR_DIVERGED
    assert out[2] == 2 and out[3] == -1.0
    assert out[0] == pytest.approx(float(rho[good].sum()), rel=MASS_REL)
    sim.close()


def test_single_lattice_guard_is_deterministic_and_residual_zero_at_rest_point():
    olat, sim = make_pair(40, 24, BC_PER, SMOOTH06, {})
    rho0, ux0, uy0 = _initial("droplet", 40, 24, olat.eos, 5)
    sim.init_equilibrium(rho0, ux0, uy0)
    sim.step(13)
    a = sim.guard()
    b = sim.guard()
    assert a[:3] == b[:3]
    assert b[3] == 0.0
    sim.close()


def _batch_case():
    """Instances of one collision kind (unit relaxation times), periodic and walled."""
    import paper_2107_06355_gb300 as P

    inst = [("planar", 4, 160, BC_PER, SMOOTH05), ("droplet", 48, 48, BC_PER, SMOOTH06),
            ("impact", 56, 40, BC_WALLS, SMOOTH06), ("droplet", 33, 27, BC_PER, CS07),
            ("impact", 40, 30, BC_WALLS, SMOOTH05)]
    olats, inits = [], []
    for k, (kind, nx, ny, bc, ec) in enumerate(inst):
        olat, sim = make_pair(nx, ny, bc, ec, {})
        sim.close()
        olats.append(olat)
        inits.append(_initial(kind, nx, ny, olat.eos, 40 + k))
    eos = []
    for (_, _, _, _, ec) in inst:
        mode, Tr, a_l, a_v, alpha = ec
        eos.append(P.EOSParams(mode, Tr, a_l, a_v if mode == E.MODE_SMOOTH else a_l, alpha if alpha > 0 else 0.5))
    b = P.Batch([(nx, ny, bc) for (_, nx, ny, bc, _) in inst], eos, [P.Relax() for _ in inst])
    for k, (rho, ux, uy) in enumerate(inits):
        b.init_equilibrium(k, rho, ux, uy)
    return b, olats, inits


@pytest.mark.parametrize("plan", [0, 1, 2, 3], ids=["launches", "graph", "persistent", "pipelined"])
def test_batch_guard_matches_oracle(plan):
    b, olats, inits = _batch_case()
    b.set_plan(plan, 0)
    fs = [o.init_equilibrium(*init) for o, init in zip(olats, inits)]
    prev = [None] * b.n
    for nsteps in (0, 100, 100, 9):
        if nsteps:
            fs = [o.step(f, nsteps) for o, f in zip(olats, fs)]
            b.step(nsteps)
        g = b.guard()
        for i, (o, f) in enumerate(zip(olats, fs)):
            wm, wu, wr, prev[i] = _oracle_guard(o, f, prev[i])
            _check((g[i, 0], g[i, 1], int(g[i, 2]), g[i, 3]), (wm, wu, wr), (i, nsteps, plan))
    # planted non-physical densities: counted, left out of the mass, and (with
    # isolation) they mark only their own instance diverged
    b.set_isolation(True)
    f = fs[1].copy()
    f[:, 2, 3] = -1.0
    f[:, 4, 5] = np.inf
    rho = f.sum(axis=0)
    good = np.isfinite(rho) & (rho > 0)
    b.set_f(1, torch.as_tensor(f, device="cuda"))
    g = b.guard()
    assert g[1, 2] == 2 and g[1, 3] == -1.0
    assert g[1, 0] == pytest.approx(float(rho[good].sum()), rel=MASS_REL)
    assert b.instance_status()[1] == 4
    b.close()
