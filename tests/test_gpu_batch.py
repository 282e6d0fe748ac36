"""Batched engine: many uneven lattices advanced by one launch per pass (or one
persistent cooperative launch). The per-node arithmetic is the single-lattice
step's, so every plan must give distributions bitwise equal to stepping each
lattice alone through pplbm_create/pplbm_step; that path in turn matches the
oracle (test_gpu_parity.py), and one batch instance is checked against the
oracle directly here."""
import numpy as np
import pytest

import lbm_inputs as I
from gpu_helpers import BC_PER, BC_WALLS, make_pair, normwise
from oracle import eos as E

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2107_06355_gb300")
from paper_2107_06355_gb300 import _lib as L  # noqa: E402


def _instances():
    # (nx, ny, bc, Tr, init kind)
    return [(4, 90, BC_PER, 0.8, "planar"), (70, 45, BC_PER, 0.6, "droplet"), (4, 37, BC_PER, 0.5, "planar"),
            (33, 33, BC_PER, 0.35, "droplet"), (48, 40, BC_WALLS, 0.6, "impact"), (3, 5, BC_PER, 0.6, "droplet"),
            (1, 1, BC_PER, 0.7, "uniform"), (130, 9, BC_WALLS, 0.5, "impact")]


def _init_fields(kind, nx, ny, d, seed):
    if kind == "planar":
        return I.planar(nx, ny, d["rho_v"], d["rho_l"], W=6.0), None, None
    if kind == "droplet":
        rho = I.perturbed(I.droplet(nx, ny, max(1.0, min(nx, ny) / 4), d["rho_v"], d["rho_l"], W=5.0), 0.01, seed)
        ux, uy = I.random_velocity((ny, nx), 0.01, seed + 1)
        return rho, ux, uy
    if kind == "impact":
        return I.impact(nx, ny, max(2.0, min(nx, ny) / 6), max(2, ny // 6), d["rho_v"], d["rho_l"], 0.03, W=5.0)
    return np.full((ny, nx), d["rho_l"]), None, None


def _build(relax_kw):
    inst = _instances()
    eos = [P.EOSParams(P.EOS_SMOOTH, Tr, 0.363, 2.0, 0.775) for (_, _, _, Tr, _) in inst]
    relax = [P.Relax(**relax_kw) for _ in inst]
    b = P.Batch([(nx, ny, bc) for (nx, ny, bc, _, _) in inst], eos, relax)
    sims = []
    for k, (nx, ny, bc, Tr, kind) in enumerate(inst):
        s = P.Simulation(nx, ny, bc, eos[k], relax[k])
        rho, ux, uy = _init_fields(kind, nx, ny, s.derived(), 100 + k)
        s.init_equilibrium(rho, ux, uy)
        b.init_equilibrium(k, rho, ux, uy)
        sims.append(s)
    return b, sims


@pytest.mark.parametrize("relax_kw", [{}, {"kind": 1, "tau_l": 0.6, "visc_ratio": 2.0},
                                      {"tau_e": 0.8, "tau_zeta": 1.1, "tau_q": 1.2, "tau_nu": 0.9}],
                         ids=["unit", "two_phase", "full_mrt"])
@pytest.mark.parametrize("mode,width", [(0, 0), (0, 4), (0, 32), (0, 256), (1, 0), (2, 0), (2, 8), (3, 0), (3, 32)])
def test_batch_bitwise_equals_single_lattice(relax_kw, mode, width):
    b, sims = _build(relax_kw)
    b.set_plan(mode, width)
    for nsteps in (1, 6, 7):
        b.step(nsteps)
        for s in sims:
            s.step(nsteps)
        assert b.sync() > 0
        for k, s in enumerate(sims):
            assert torch.equal(b.get_f(k), s.get_f()), (k, nsteps)
    for k, s in enumerate(sims):
        rb = b.fields(k)
        rs = s.fields()
        for x, y in zip(rb, rs):
            assert torch.equal(x, y)
    b.close()


def test_batch_instance_matches_oracle():
    inst = [(4, 64, BC_PER, 0.5), (40, 24, BC_WALLS, 0.6)]
    eos = [P.EOSParams(P.EOS_SMOOTH, Tr, 0.363, 2.0, 0.775) for (_, _, _, Tr) in inst]
    relax = [P.Relax(kind=1, tau_l=0.6, visc_ratio=2.0) for _ in inst]
    b = P.Batch([(nx, ny, bc) for (nx, ny, bc, _) in inst], eos, relax)
    b.set_plan(P.PLAN_PERSISTENT, 0)
    olat, _ = make_pair(40, 24, BC_WALLS, (E.MODE_SMOOTH, 0.6, 0.363, 2.0, 0.775),
                        {"kind": 1, "tau_l": 0.6, "visc_ratio": 2.0})
    e = olat.eos
    rho, ux, uy = I.impact(40, 24, 4, 4, e.rho_v, e.rho_l, 0.03, W=5.0)
    d0 = b.derived(0)
    b.init_equilibrium(0, I.planar(4, 64, d0["rho_v"], d0["rho_l"], W=6.0))
    b.init_equilibrium(1, rho, ux, uy)
    f = olat.init_equilibrium(rho, ux, uy)
    f = olat.step(f, 12)
    b.step(12)
    assert normwise(b.get_f(1).cpu().numpy(), f) < 1e-11


def test_autotune_keeps_state_and_reports_plan():
    b, sims = _build({})
    b.step(3)
    before = [b.get_f(k).clone() for k in range(len(sims))]
    plan = b.autotune(trial_steps=6)
    assert plan["mode"] in (0, 1, 2, 3)
    assert plan["ms_launches"] > 0 and plan["ms_graph"] > 0 and plan["ms_persistent"] > 0
    assert plan["ms_pipelined"] > 0
    for k in range(len(sims)):
        assert torch.equal(b.get_f(k), before[k])
    # stepping after tuning still matches the single-lattice path
    b.step(5)
    for s in sims:
        s.step(8)
    for k, s in enumerate(sims):
        assert torch.equal(b.get_f(k), s.get_f())


def test_persistent_barrier_wait_runs_out_and_is_reported():
    """Failure detection without a GPU fault: one block leaves without arriving,
    the others' bounded waits run out, the status is PPLBM_ERR_TIMEOUT, and the
    batch (whose distributions the test run did not touch) keeps working."""
    b, sims = _build({})
    b.set_plan(P.PLAN_PERSISTENT, 0)
    b.step(2)
    for s in sims:
        s.step(2)
    assert b.barrier_selftest(spin_limit=1 << 12) == 5
    b.step(3)
    for s in sims:
        s.step(3)
    assert b.sync() == 5
    for k, s in enumerate(sims):
        assert torch.equal(b.get_f(k), s.get_f())


def test_sweep_64_instances_full_size_sampled():
    """The 64-lattice sweep (seed 210706355, planar L x 4 and droplets L x L, L in
    64..1024, T_r 0.35..0.95; ~12.9 M nodes) in the autotuned plan: sampled small
    instances against the oracle, large ones bitwise against single-lattice steps."""
    specs = I.batch_specs()
    eos = [P.EOSParams(P.EOS_SMOOTH, s["Tr"], 0.363, 2.0, 0.775) for s in specs]
    relax = [P.Relax() for _ in specs]
    b = P.Batch([(s["nx"], s["ny"], BC_PER) for s in specs], eos, relax)
    inits = []
    for k, s in enumerate(specs):
        d = b.derived(k)
        if s["kind"] == "planar":
            rho = I.planar(s["nx"], s["ny"], d["rho_v"], d["rho_l"], W=8.0)
        else:
            rho = I.droplet(s["nx"], s["ny"], s["R"], d["rho_v"], d["rho_l"], W=8.0)
        b.init_equilibrium(k, rho)
        inits.append(rho)
    plan = b.autotune(trial_steps=4)
    b.step(5)
    b.sync()
    # small planar instances against the oracle
    for k in (0, 6, 62):
        s = specs[k]
        olat, _ = make_pair(s["nx"], s["ny"], BC_PER, (E.MODE_SMOOTH, s["Tr"], 0.363, 2.0, 0.775), {})
        f = olat.step(olat.init_equilibrium(inits[k]), 5)
        assert normwise(b.get_f(k).cpu().numpy(), f) < 1e-12, (k, plan)
    # large droplets bitwise against the single-lattice path
    for k in (1, 33, 63):
        s = specs[k]
        sim = P.Simulation(s["nx"], s["ny"], BC_PER, eos[k], relax[k])
        sim.init_equilibrium(inits[k])
        sim.step(5)
        assert torch.equal(b.get_f(k), sim.get_f()), (k, plan)
        sim.close()
    b.close()


def _host_guard(b, i, prev_rho):
    """mass, max |u|, bad count, residual on the host from the library's fields
    (rho, and u = (j + F/2)/rho as the collision pass computes it)."""
    rho, ux, uy, _ = [t.cpu().numpy() for t in b.fields(i)]
    good = np.isfinite(rho) & (rho > 0)
    mass = rho[good].sum()
    umax = np.hypot(ux, uy)[good].max() if good.any() else 0.0
    res = -1.0 if prev_rho is None else np.abs(rho - prev_rho)[good].sum() / mass
    return np.array([mass, umax, float((~good).sum()), res]), rho


def test_batch_guard_matches_host_reduction():
    b, sims = _build({"kind": 1, "tau_l": 0.6, "visc_ratio": 2.0})
    for s in sims:
        s.close()
    b.set_plan(1, 0)
    prev = [None] * b.n
    for nsteps in (3, 10, 1):
        g = b.guard()
        for i in range(b.n):
            want, prev[i] = _host_guard(b, i, prev[i])
            assert g[i, 2] == want[2] == 0
            assert g[i, 0] == pytest.approx(want[0], rel=1e-13)
            assert g[i, 1] == pytest.approx(want[1], rel=1e-12, abs=1e-300)
            if want[3] < 0:
                assert g[i, 3] == -1.0
            else:
                assert g[i, 3] == pytest.approx(want[3], rel=1e-9, abs=1e-17)
        b.step(nsteps)
    # deterministic: the same state gives the same bits
    a1 = b.guard()
    a2 = b.guard()
    assert np.array_equal(a1[:, :3], a2[:, :3]) and np.all(a2[:, 3] == 0.0)
    # set_f restarts the residual; non-positive nodes are counted, not summed, and
    # (with isolation) mark only their own instance diverged
    b.set_isolation(True)
    nx, ny = b.shapes[1]
    f = b.get_f(1).cpu().numpy()
    f[:, 2, 3] = -1.0
    f[:, 4, 5] = -2.0
    good_mass = np.delete(f.sum(axis=0).reshape(-1), [2 * nx + 3, 4 * nx + 5]).sum()
    b.set_f(1, torch.as_tensor(f, device="cuda"))
    g = b.guard()
    assert g[1, 2] == 2 and g[1, 3] == -1.0
    assert g[1, 0] == pytest.approx(good_mass, rel=1e-13)
    assert g[0, 3] == 0.0
    assert b.instance_status()[1] == L.PPLBM_ERR_DIVERGED
    assert [st for k, st in enumerate(b.instance_status()) if k != 1] == [0] * (b.n - 1)
    b.close()


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_batch_run_host_equals_init_step_fields(mode):
    """pplbm_batch_run_host (host in, nsteps, host out) gives the densities of
    init_equilibrium + step + get_fields, bit for bit, in every plan."""
    inst = _instances()
    eos = [P.EOSParams(P.EOS_SMOOTH, Tr, 0.363, 2.0, 0.775) for (_, _, _, Tr, _) in inst]
    lats = [(nx, ny, bc) for (nx, ny, bc, _, _) in inst]
    relax = [P.Relax() for _ in inst]
    b1 = P.Batch(lats, eos, relax)
    b2 = P.Batch(lats, eos, relax)
    b1.set_plan(mode, 0)
    b2.set_plan(mode, 0)
    rho0s = []
    for k, (nx, ny, bc, Tr, kind) in enumerate(inst):
        rho, _, _ = _init_fields(kind, nx, ny, b1.derived(k), 300 + k)
        rho0s.append(np.ascontiguousarray(rho, dtype=np.float64))
        b2.init_equilibrium(k, rho)
    outs = [np.empty_like(r) for r in rho0s]
    b1.run_host(rho0s, 9, outs)
    b2.step(9)
    for k in range(len(inst)):
        assert np.array_equal(outs[k], b2.fields(k)[0].cpu().numpy())
    with pytest.raises(ValueError):
        b1.run_host(rho0s[:-1], 1, outs)
    b1.close()
    b2.close()


def test_one_call_batch_init_equals_create_then_init():
    import ctypes as C

    inst = _instances()
    eos = [P.EOSParams(P.EOS_SMOOTH, Tr, 0.363, 2.0, 0.775) for (_, _, _, Tr, _) in inst]
    relax = [P.Relax() for _ in inst]
    ref = P.Batch([(nx, ny, bc) for (nx, ny, bc, _, _) in inst], eos, relax)
    fields = []
    for k, (nx, ny, bc, Tr, kind) in enumerate(inst):
        rho, ux, uy = _init_fields(kind, nx, ny, ref.derived(k), 500 + k)
        fields.append(tuple(None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux, uy)))
        ref.init_equilibrium(k, *fields[-1])
    n = len(inst)
    ptrs = [(C.c_void_p * n)(*[None if f[j] is None else f[j].ctypes.data for f in fields]) for j in range(3)]
    ws = torch.empty(ref.workspace.numel(), dtype=torch.float64, device="cuda")
    base = (ws.data_ptr() + 255) // 256 * 256
    nbytes = L.lib().pplbm_batch_workspace_bytes(n, ref._lat, ref._relax)
    b = C.c_void_p()
    st = L.lib().pplbm_batch_init(C.byref(b), n, ref._lat, ref._eos, ref._relax, -1.0, *ptrs, C.c_void_p(base),
                                  nbytes, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == L.PPLBM_OK
    L.check(L.lib().pplbm_batch_step(b, 4), batch=b)
    ref.step(4)
    for k, (nx, ny, _, _, _) in enumerate(inst):
        f = torch.empty((9, ny, nx), dtype=torch.float64, device="cuda")
        L.check(L.lib().pplbm_batch_get_f(b, k, C.c_void_p(f.data_ptr())), batch=b)
        torch.cuda.synchronize()
        assert torch.equal(f, ref.get_f(k))
    L.lib().pplbm_batch_destroy(b)
    ref.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_pass_timing_counts_launches_and_keeps_results(mode):
    """pplbm_batch_enable_pass_timing brackets each pass with CUDA events; the steps it
    issues are the same arithmetic (bitwise) and every launch is counted."""
    b, sims = _build({})
    for s in sims:
        s.close()
    ref, _ = _build({})
    b.set_plan(mode, 0)
    ref.set_plan(mode, 0)
    b.enable_pass_timing(3)
    b.step(7)
    (m0, m1), (n0, n1) = b.pass_times()
    assert (n0, n1) == (7, 7) and m0 > 0 and m1 > 0
    b.step(2)
    assert b.pass_times()[1] == (2, 2)
    with pytest.raises(P.PPLBMError):
        b.set_plan(2, 0)   # the persistent plan has a single launch
    with pytest.raises(P.PPLBMError):
        b.set_plan(3, 0)   # the pipelined plan's launches mix the passes
    b.enable_pass_timing(0)
    ref.step(9)
    for k in range(b.n):
        assert torch.equal(b.get_f(k), ref.get_f(k))
    b.close()
    ref.close()


def test_sweep_64_lattices_full_length_stable():
    """The 64-lattice sweep the benchmark times (seed 210706355, T_r 0.35..0.95, Smooth
    C-S a_l = 0.363, a_v = 2, alpha = 0.775, tau = 1, Li forcing), run for its full
    20,000 steps: no non-physical node, mass conserved to round-off, speeds bounded, and
    the small instances still equal to the oracle's state stepped alongside for the
    first 200 steps (the large ones are covered by bitwise equality with the single-
    lattice path, itself checked against the oracle)."""
    specs = I.batch_specs()
    eos = [P.EOSParams(P.EOS_SMOOTH, s["Tr"], 0.363, 2.0, 0.775) for s in specs]
    b = P.Batch([(s["nx"], s["ny"], BC_PER) for s in specs], eos, [P.Relax() for _ in specs])
    inits = []
    for k, s in enumerate(specs):
        d = b.derived(k)
        rho = (I.planar(s["nx"], s["ny"], d["rho_v"], d["rho_l"], W=8.0) if s["kind"] == "planar"
               else I.droplet(s["nx"], s["ny"], s["R"], d["rho_v"], d["rho_l"], W=8.0))
        b.init_equilibrium(k, rho)
        inits.append(rho)
    b.autotune(trial_steps=4)
    g0 = b.guard()
    small = [k for k, s in enumerate(specs) if s["nx"] * s["ny"] <= 1200][:3]
    oracles = {}
    for k in small:
        s = specs[k]
        olat, _ = make_pair(s["nx"], s["ny"], BC_PER, (E.MODE_SMOOTH, s["Tr"], 0.363, 2.0, 0.775), {})
        oracles[k] = (olat, olat.step(olat.init_equilibrium(inits[k]), 200))
    b.step(200)
    for k, (olat, f) in oracles.items():
        assert normwise(b.get_f(k).cpu().numpy(), f) < 1e-10, k
    b.step(20000 - 200)
    g = b.guard()
    assert (g[:, 2] == 0).all()
    np.testing.assert_allclose(g[:, 0], g0[:, 0], rtol=1e-10)
    assert (g[:, 1] < 0.3).all()
    b.close()


@pytest.mark.parametrize("count", [1, 2, 3])
def test_pipelined_plan_small_batches_bitwise(count):
    """The pipelined plan with one instance (the second group empty: prologue, the
    first group's passes in turn, an empty epilogue), two and three (groups of
    unequal node counts), over call lengths 1, 2, 5: bitwise the single-lattice step,
    and every instance at the same step after each call."""
    inst = [(70, 45, BC_PER, 0.6, "droplet"), (48, 40, BC_WALLS, 0.6, "impact"), (4, 90, BC_PER, 0.8, "planar")]
    inst = inst[:count]
    eos = [P.EOSParams(P.EOS_SMOOTH, Tr, 0.363, 2.0, 0.775) for (_, _, _, Tr, _) in inst]
    relax = [P.Relax() for _ in inst]
    b = P.Batch([(nx, ny, bc) for (nx, ny, bc, _, _) in inst], eos, relax)
    sims = []
    for k, (nx, ny, bc, Tr, kind) in enumerate(inst):
        s = P.Simulation(nx, ny, bc, eos[k], relax[k])
        rho, ux, uy = _init_fields(kind, nx, ny, s.derived(), 300 + k)
        s.init_equilibrium(rho, ux, uy)
        b.init_equilibrium(k, rho, ux, uy)
        sims.append(s)
    b.set_plan(P.PLAN_PIPELINED, 0)
    done = 0
    for nsteps in (1, 2, 5):
        b.step(nsteps)
        done += nsteps
        for s in sims:
            s.step(nsteps)
        assert b.sync() == done
        for k, s in enumerate(sims):
            assert torch.equal(b.get_f(k), s.get_f()), (count, k, nsteps)
    b.close()
    for s in sims:
        s.close()
