"""GPU adjoint: one adjoint step against the oracle's reverse-mode autograd, a
small checkpointed rollout against the oracle, and the 256 x 256 droplet
rollout of 2,000 steps (R = 48, T_r = 0.5, sqrt(N) checkpoints) against central
finite differences (h = 1e-6) in alpha and in the initial density."""
import ctypes as C
import math

import numpy as np
import pytest

import lbm_inputs as I
from gpu_helpers import BC_PER, BC_WALLS, make_pair, normwise
from oracle import adjoint as A
from oracle import eos as E

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2107_06355_gb300")
from paper_2107_06355_gb300 import _lib as L  # noqa: E402
from paper_2107_06355_gb300 import adjoint as AD  # noqa: E402

CASE = (E.MODE_SMOOTH, 0.5, 0.363, 2.0, 0.775)


def _state(olat, nx, ny, bc):
    e = olat.eos
    if bc == BC_WALLS:
        rho, ux, uy = I.impact(nx, ny, 3, 4, e.rho_v, e.rho_l, 0.01, W=6.0)
    else:
        rho = I.perturbed(I.droplet(nx, ny, min(nx, ny) / 4, e.rho_v, e.rho_l, W=5.0), 0.01, 5)
        ux, uy = I.random_velocity((ny, nx), 0.005, 6)
    return olat.step(olat.init_equilibrium(rho, ux, uy), 3)


def _gpu_param_grad(sim, grad, which=0):
    """dL/dtheta through the library's chain rule (pplbm_adjoint_set_param at the
    context's parameters, then pplbm_adjoint_param_gradient over grad on the device)."""
    assert L.lib().pplbm_adjoint_set_param(sim.ctx, which, 1e-4) == 0
    out = (C.c_double * 1)()
    assert L.lib().pplbm_adjoint_param_gradient(sim.ctx, C.c_void_p(grad.data_ptr()), out) == 0
    return out[0]


@pytest.mark.parametrize("kappa", [0.0, 0.6])
@pytest.mark.parametrize("shape,bc", [((40, 18), BC_PER), ((37, 22), BC_WALLS)], ids=["periodic", "walls"])
def test_adjoint_step_matches_oracle_autograd(shape, bc, kappa):
    """One adjoint step against reverse mode through the oracle's torch restatement;
    kappa != 0 includes the surface-tension source (its stencil sums' transposes)."""
    nx, ny = shape
    olat, sim = make_pair(nx, ny, bc, CASE, {"kappa": kappa})
    f = _state(olat, nx, ny, bc)
    lam1 = np.random.default_rng(11).standard_normal((9, ny, nx))
    # oracle: reverse mode through the torch restatement
    c = A.constants_as_tensors(olat.eos)
    c["kappa"] = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
    x = torch.tensor(f, requires_grad=True)
    (A.step(x, olat, c) * torch.tensor(lam1)).sum().backward()
    dc_cpu = A.constants_derivative(*CASE[:4], CASE[4])
    galpha_cpu = sum(float(c[k].grad) * dc_cpu[k] for k in A.CONST_NAMES)
    # GPU
    fd = torch.tensor(f, device="cuda")
    l1 = torch.tensor(lam1, device="cuda")
    l0 = torch.empty_like(l1)
    grad = torch.zeros(L.NGRAD, dtype=torch.float64, device="cuda")
    nbytes = L.lib().pplbm_adjoint_workspace_bytes(C.byref(sim.lattice))
    ws = torch.empty(nbytes // 8 + 1, dtype=torch.float64, device="cuda")
    p = lambda t: C.c_void_p(t.data_ptr())
    assert L.lib().pplbm_adjoint_step(sim.ctx, p(fd), p(l1), p(l0), p(grad), p(ws), nbytes) == 0
    torch.cuda.synchronize()
    assert normwise(l0.cpu().numpy(), x.grad.numpy()) < 1e-12
    # dL/dkappa: its own slot (computed at kappa = 0 too, the default slots including it)
    assert float(c["kappa"].grad) != 0.0
    assert float(grad[L.GRAD_NAMES.index("kappa")]) == pytest.approx(float(c["kappa"].grad), rel=1e-9)
    out = (C.c_double * 1)()
    assert L.lib().pplbm_adjoint_param_gradient(sim.ctx, C.c_void_p(grad.data_ptr()), out) == L.PPLBM_ERR_STATE
    galpha_gpu = _gpu_param_grad(sim, grad, 0)
    assert galpha_gpu == pytest.approx(galpha_cpu, rel=1e-6)
    # the branch parameters: the GPU's k1, k2, k4 slots against the oracle's a, T, Delta P
    for wrt, which in (("a_v", 1), ("a_l", 2)):
        dc_w = A.constants_derivative(*CASE[:4], CASE[4], wrt=wrt)
        g_cpu = sum(float(c[k].grad) * dc_w[k] for k in A.CONST_NAMES)
        g_gpu = _gpu_param_grad(sim, grad, which)
        assert g_cpu != 0.0
        assert g_gpu == pytest.approx(g_cpu, rel=1e-6), wrt


@pytest.mark.parametrize("kappa", [0.0, 0.6])
def test_small_rollout_matches_oracle_reference_adjoint(kappa):
    nx, ny, nsteps = 24, 24, 30
    olat, _ = make_pair(nx, ny, BC_PER, CASE, {"kappa": kappa})
    e = olat.eos
    rho0 = I.droplet(nx, ny, 6.0, e.rho_v, e.rho_l, W=5.0)
    # oracle reference adjoint
    c = A.constants_as_tensors(e)
    r0 = torch.tensor(rho0, requires_grad=True)
    g = torch.stack([float(w) * r0 for w in A._W])
    for _ in range(nsteps):
        g = A.step(g, olat, c)
    loss = A.droplet_loss(g.sum(0), e.rho_v, e.rho_l, 6.0)
    loss.backward()
    dc_cpu = A.constants_derivative(*CASE[:4], CASE[4])
    galpha_cpu = sum(float(c[k].grad) * dc_cpu[k] for k in A.CONST_NAMES)
    # GPU rollout through the autograd Function
    spec = AD.RolloutSpec(nx, ny, P.BC_PERIODIC, P.EOSParams(P.EOS_SMOOTH, 0.5, 0.363, 2.0, 0.775),
                          P.Relax(kappa=kappa), nsteps, interval=7)
    rho0_t = torch.tensor(rho0, device="cuda", requires_grad=True)
    alpha = torch.tensor(0.775, dtype=torch.float64, requires_grad=True)
    rhoN = AD.rollout(rho0_t, alpha, spec)
    lg = A.droplet_loss(rhoN, e.rho_v, e.rho_l, 6.0)
    lg.backward()
    # the vapour term divides by rho_v ~ 6e-4, which amplifies 1e-13 differences in rho
    assert float(lg.detach()) == pytest.approx(float(loss.detach()), rel=1e-8)
    assert normwise(rho0_t.grad.cpu().numpy(), r0.grad.numpy()) < 1e-8
    assert float(alpha.grad) == pytest.approx(galpha_cpu, rel=1e-6)


def test_droplet_256_rollout_2000_steps_against_finite_differences():
    """The adjoint configuration: 256 x 256 periodic droplet, R = 48, T_r = 0.5
    (a_l = 0.363, a_v = 2, alpha = 0.775), tau = 1, 2,000 steps, checkpoint every
    45 steps; loss = squared vapour-density error vs Maxwell + radius mismatch."""
    nx = ny = 256
    nsteps, R0 = 2000, 48.0
    eosp = P.EOSParams(P.EOS_SMOOTH, 0.5, 0.363, 2.0, 0.775)
    d = P.eos_setup(eosp)
    rv, rl = d["rho_v"], d["rho_l"]
    rho0 = torch.tensor(I.droplet(nx, ny, R0, rv, rl, W=7.0), device="cuda")
    spec = AD.RolloutSpec(nx, ny, P.BC_PERIODIC, eosp, P.Relax(), nsteps, interval=45)

    def loss_of(rho):
        phi = (rho - rv) / (rl - rv)
        reff = torch.sqrt(phi.sum() / math.pi)
        return ((rho[0, 0] - rv) / rv) ** 2 + ((reff - R0) / R0) ** 2

    r0 = rho0.clone().requires_grad_(True)
    alpha = torch.tensor(0.775, dtype=torch.float64, requires_grad=True)
    L0 = loss_of(AD.rollout(r0, alpha, spec))
    L0.backward()

    def loss_at(al, rho):
        with torch.no_grad():
            return float(loss_of(AD.rollout(rho, torch.tensor(al, dtype=torch.float64), spec)))

    h = 1e-6
    fd_alpha = (loss_at(0.775 + h, rho0) - loss_at(0.775 - h, rho0)) / (2 * h)
    assert float(alpha.grad) == pytest.approx(fd_alpha, rel=1e-6)
    v = torch.tensor(np.random.default_rng(7).standard_normal((ny, nx)), device="cuda") * rho0
    hv = 1e-6
    fd_rho = (loss_at(0.775, rho0 + hv * v) - loss_at(0.775, rho0 - hv * v)) / (2 * hv)
    assert float((r0.grad * v).sum()) == pytest.approx(fd_rho, rel=1e-6)


def test_rollout_gradients_do_not_depend_on_the_checkpoint_interval():
    """Intervals below 4 store the recomputed states, longer ones keep only psi and
    the moments of each state: both feed the adjoint kernels the same values in the
    same order, so the gradients are bitwise equal across intervals."""
    nx, ny, nsteps = 40, 36, 30
    eosp = P.EOSParams(P.EOS_SMOOTH, 0.5, 0.363, 2.0, 0.775)
    d = P.eos_setup(eosp)
    rho0 = I.perturbed(I.droplet(nx, ny, 10.0, d["rho_v"], d["rho_l"], W=6.0), 0.002, 11)
    grads = []
    for interval in (1, 2, 3, 7, 30):
        spec = AD.RolloutSpec(nx, ny, P.BC_PERIODIC, eosp, P.Relax(), nsteps, interval=interval)
        r0 = torch.tensor(rho0, device="cuda", requires_grad=True)
        alpha = torch.tensor(0.775, dtype=torch.float64, requires_grad=True)
        rhoN = AD.rollout(r0, alpha, spec)
        (rhoN ** 2).sum().backward()
        grads.append((r0.grad.cpu().numpy(), float(alpha.grad)))
    for g in grads[1:]:
        assert np.array_equal(g[0], grads[0][0])
        assert g[1] == grads[0][1]


def test_adjoint_segment_equals_one_segment_backward():
    """pplbm_adjoint_segment(f_start, n) = pplbm_backward_checkpointed with interval n."""
    nx, ny, nsteps = 40, 36, 12
    eosp = P.EOSParams(P.EOS_SMOOTH, 0.5, 0.363, 2.0, 0.775)
    sim = P.Simulation(nx, ny, P.BC_PERIODIC, eosp, P.Relax())
    d = sim.derived()
    sim.init_equilibrium(I.perturbed(I.droplet(nx, ny, 10.0, d["rho_v"], d["rho_l"], W=6.0), 0.002, 5))
    f0 = sim.get_f().clone()
    lam = torch.as_tensor(np.random.default_rng(3).standard_normal((9, ny, nx)), device="cuda")
    nb = L.lib().pplbm_adjoint_workspace_bytes(C.byref(sim.lattice))
    out = []
    for which in range(2):
        ws = torch.zeros(nb // 8 + 1, dtype=torch.float64, device="cuda")
        states = torch.empty((nsteps, 9, ny, nx), dtype=torch.float64, device="cuda")
        lam0 = torch.empty_like(lam)
        grad = torch.zeros(L.NGRAD, dtype=torch.float64, device="cuda")
        p = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
        if which == 0:
            st = L.lib().pplbm_adjoint_segment(sim.ctx, p(f0), nsteps, p(states), p(lam), p(lam0), p(grad), p(ws), nb)
        else:
            st = L.lib().pplbm_backward_checkpointed(sim.ctx, nsteps, nsteps, p(f0), p(states), p(lam), p(lam0),
                                                     p(grad), p(ws), nb)
        L.check(st, sim.ctx)
        torch.cuda.synchronize()
        out.append((lam0.cpu(), grad.cpu()))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    sim.close()


@pytest.mark.parametrize("param", ["alpha", "a_vap", "a_liq"])
def test_planar_vapour_density_error_gradient_against_finite_differences(param):
    """The planar-interface loss: E^2 with E = (rho_v(sim) - rho_v^M)/rho_v^M the
    vapour-density error of Eq. DensityError, after 3,000 steps of the (4, 200)
    planar interface at T_r = 0.5 (Smooth C-S, a = 0.5, a_v = 0.5, alpha = 0.610,
    the w = 7 row of Table ParamSmooth; tau = 1, Li forcing). d(E^2)/d theta for
    theta = alpha, a_vap, a_liq from the adjoint (sqrt(N) checkpoints) against
    central differences, h = 1e-6."""
    nx, ny, nsteps = 4, 200, 3000
    eosp = P.EOSParams(P.EOS_SMOOTH, 0.5, 0.5, 0.5, 0.610)
    th0 = getattr(eosp, param)
    d = P.eos_setup(eosp)
    rv, rl = d["rho_v"], d["rho_l"]   # the Maxwell densities do not depend on theta (fixed T_r)
    rho0 = torch.tensor(I.planar(nx, ny, rv, rl, W=10.0), device="cuda")
    spec = AD.RolloutSpec(nx, ny, P.BC_PERIODIC, eosp, P.Relax(), nsteps, param=param)

    def loss_of(rho):
        return ((rho[0, :].mean() - rv) / rv) ** 2

    theta = torch.tensor(th0, dtype=torch.float64, requires_grad=True)
    L0 = loss_of(AD.rollout(rho0, theta, spec))
    L0.backward()

    def loss_at(v):
        with torch.no_grad():
            return float(loss_of(AD.rollout(rho0, torch.tensor(v, dtype=torch.float64), spec)))

    h = 1e-6
    fd = (loss_at(th0 + h) - loss_at(th0 - h)) / (2 * h)
    assert abs(float(theta.grad)) > 0
    assert float(theta.grad) == pytest.approx(fd, rel=1e-6)


def test_slot_mask_skips_only_the_deselected_gradients():
    """pplbm_adjoint_set_slots: the selected slots are bitwise those of the full
    computation, the others stay 0; lambda does not depend on the mask."""
    nx, ny = 40, 18
    olat, sim = make_pair(nx, ny, BC_PER, CASE, {})
    f = torch.tensor(_state(olat, nx, ny, BC_PER), device="cuda")
    l1 = torch.tensor(np.random.default_rng(12).standard_normal((9, ny, nx)), device="cuda")
    nbytes = L.lib().pplbm_adjoint_workspace_bytes(C.byref(sim.lattice))
    p = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    alpha_slots = sum(1 << k for k in range(9))
    res = []
    for mask in ((1 << L.NGRAD) - 1, alpha_slots):
        assert L.lib().pplbm_adjoint_set_slots(sim.ctx, mask) == 0
        l0 = torch.empty_like(l1)
        grad = torch.zeros(L.NGRAD, dtype=torch.float64, device="cuda")
        ws = torch.empty(nbytes // 8 + 1, dtype=torch.float64, device="cuda")
        assert L.lib().pplbm_adjoint_step(sim.ctx, p(f), p(l1), p(l0), p(grad), p(ws), nbytes) == 0
        torch.cuda.synchronize()
        res.append((l0.cpu(), grad.cpu()))
    assert torch.equal(res[0][0], res[1][0])
    assert torch.equal(res[0][1][:9], res[1][1][:9])
    assert torch.all(res[1][1][9:] == 0) and torch.any(res[0][1][9:] != 0)
    assert L.lib().pplbm_adjoint_set_slots(sim.ctx, 1 << L.NGRAD) == L.PPLBM_ERR_ARG


@pytest.mark.parametrize("kappa", [0.0, 0.6])
def test_stored_rollout_equals_checkpointed_rollout_bitwise(kappa):
    """pplbm_forward_stored / pplbm_backward_stored keep every step's psi and
    moments instead of recomputing them: the gradients are bitwise those of the
    sqrt(N)-checkpointed pair (the Python rollout picks the stored mode when the
    interval is automatic and the fields fit)."""
    nx, ny, nsteps = 40, 36, 30
    eosp = P.EOSParams(P.EOS_SMOOTH, 0.5, 0.363, 2.0, 0.775)
    d = P.eos_setup(eosp)
    rho0 = I.perturbed(I.droplet(nx, ny, 10.0, d["rho_v"], d["rho_l"], W=6.0), 0.002, 21)
    out = []
    for interval in (0, 6):
        spec = AD.RolloutSpec(nx, ny, P.BC_PERIODIC, eosp, P.Relax(kappa=kappa), nsteps, interval=interval)
        assert spec.stored() == (interval == 0)
        r0 = torch.tensor(rho0, device="cuda", requires_grad=True)
        alpha = torch.tensor(0.775, dtype=torch.float64, requires_grad=True)
        rhoN = AD.rollout(r0, alpha, spec)
        (rhoN ** 2).sum().backward()
        out.append((rhoN.detach().cpu(), r0.grad.cpu(), float(alpha.grad)))
    assert torch.equal(out[0][0], out[1][0])
    assert torch.equal(out[0][1], out[1][1]) and out[0][2] == out[1][2]


@pytest.mark.parametrize("kappa", [0.0, 0.4])
def test_rollout_gradient_wrt_kappa_matches_finite_differences(kappa):
    """dL/dkappa of a checkpointed rollout (the surface-tension control, its own
    gradient slot) against central differences of the forward rollout: a 48^2
    droplet (T_r = 0.5, Smooth C-S), 300 steps, loss = droplet-shape mismatch (the
    oracle's reverse mode on the same case gives 0.64268440237 at kappa = 0.4, the
    GPU adjoint 0.64268440234)."""
    nx = ny = 48
    eosp = P.EOSParams(P.EOS_SMOOTH, 0.5, 0.363, 2.0, 0.775)
    d = P.eos_setup(eosp)
    rho0 = I.perturbed(I.droplet(nx, ny, 12.0, d["rho_v"], d["rho_l"], W=6.0), 0.002, 5)
    spec = AD.RolloutSpec(nx, ny, P.BC_PERIODIC, eosp, P.Relax(), 300, interval=20, param="kappa")

    def loss(rhoN):
        return A.droplet_loss(rhoN, d["rho_v"], d["rho_l"], 12.0)

    r0 = torch.tensor(rho0, device="cuda", requires_grad=True)
    k = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
    loss(AD.rollout(r0, k, spec)).backward()
    h = 1e-4
    with torch.no_grad():
        # float64: a float32 theta would round kappa +- h by ~1e-8, 1e-4 of the step
        lp = float(loss(AD.rollout(torch.tensor(rho0, device="cuda"), torch.tensor(kappa + h, dtype=torch.float64),
                                   spec)))
        lm = float(loss(AD.rollout(torch.tensor(rho0, device="cuda"), torch.tensor(kappa - h, dtype=torch.float64),
                                   spec)))
    fd = (lp - lm) / (2 * h)
    assert abs(fd) > 1e-8
    assert float(k.grad) == pytest.approx(fd, rel=1e-6)
