"""The hand-written adjoint with the two-phase relaxation of the dynamic runs (Sec. IV:
Lambda = diag(1, ..., 1, 1/tau(rho), 1/tau(rho)), tau(rho) of Eq. RelaxationTime),
periodic and walled, with and without the surface-tension control.

References: reverse mode through the oracle's torch restatement (oracle/adjoint.py,
itself pinned to the numpy oracle and to finite differences in
tests/test_oracle_adjoint.py) and central differences of the GPU forward rollout.
Tolerances as for unit relaxation times: lambda 1e-12 normwise per step (the step's
parity bound), parameter gradients 1e-6 relative (the chain rule's dc/dtheta and
the oracle's are central-difference estimates good to ~1e-8 relative)."""
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
TWO_PHASE = {"kind": 1, "tau_l": 0.6, "visc_ratio": 3.0}


def _state(olat, nx, ny, bc):
    e = olat.eos
    if bc == BC_WALLS:
        rho, ux, uy = I.impact(nx, ny, 3, 4, e.rho_v, e.rho_l, 0.01, W=6.0)
    else:
        rho = I.perturbed(I.droplet(nx, ny, min(nx, ny) / 4, e.rho_v, e.rho_l, W=5.0), 0.01, 5)
        ux, uy = I.random_velocity((ny, nx), 0.005, 6)
    return olat.step(olat.init_equilibrium(rho, ux, uy), 3)


def _param_grad(sim, grad, which):
    assert L.lib().pplbm_adjoint_set_param(sim.ctx, which, 1e-4) == 0
    out = (C.c_double * 1)()
    assert L.lib().pplbm_adjoint_param_gradient(sim.ctx, C.c_void_p(grad.data_ptr()), out) == 0
    return out[0]


@pytest.mark.parametrize("kappa", [0.0, 0.6])
@pytest.mark.parametrize("shape,bc", [((40, 18), BC_PER), ((37, 22), BC_WALLS)], ids=["periodic", "walls"])
def test_two_phase_adjoint_step_matches_oracle_autograd(shape, bc, kappa):
    nx, ny = shape
    olat, sim = make_pair(nx, ny, bc, CASE, dict(TWO_PHASE, kappa=kappa))
    f = _state(olat, nx, ny, bc)
    lam1 = np.random.default_rng(13).standard_normal((9, ny, nx))
    c = A.constants_as_tensors(olat.eos)
    c["kappa"] = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
    x = torch.tensor(f, requires_grad=True)
    (A.step(x, olat, c) * torch.tensor(lam1)).sum().backward()
    fd = torch.tensor(f, device="cuda")
    l1 = torch.tensor(lam1, device="cuda")
    l0 = torch.empty_like(l1)
    grad = torch.zeros(L.NGRAD, dtype=torch.float64, device="cuda")
    nbytes = L.lib().pplbm_adjoint_workspace_bytes(C.byref(sim.lattice))
    ws = torch.empty(nbytes // 8 + 1, dtype=torch.float64, device="cuda")
    p = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    assert L.lib().pplbm_adjoint_step(sim.ctx, p(fd), p(l1), p(l0), p(grad), p(ws), nbytes) == 0
    torch.cuda.synchronize()
    assert normwise(l0.cpu().numpy(), x.grad.numpy()) < 1e-12
    assert float(grad[L.GRAD_NAMES.index("kappa")]) == pytest.approx(float(c["kappa"].grad), rel=1e-9)
    for wrt, which in (("alpha", 0), ("a_v", 1), ("a_l", 2)):
        dc = A.constants_derivative(*CASE[:4], CASE[4], wrt=wrt)
        g_cpu = sum(float(c[k].grad) * dc[k] for k in A.CONST_NAMES)
        assert g_cpu != 0.0
        assert _param_grad(sim, grad, which) == pytest.approx(g_cpu, rel=1e-6), wrt
    sim.close()


def test_general_mrt_adjoint_is_refused():
    """The six-time MRT set has no adjoint: PPLBM_ERR_STATE, not a wrong gradient."""
    nx, ny = 24, 16
    olat, sim = make_pair(nx, ny, BC_PER, CASE, {"tau_e": 0.8, "tau_nu": 0.9})
    f = torch.tensor(_state(olat, nx, ny, BC_PER), device="cuda")
    l1 = torch.ones_like(f)
    l0 = torch.empty_like(f)
    grad = torch.zeros(L.NGRAD, dtype=torch.float64, device="cuda")
    nbytes = L.lib().pplbm_adjoint_workspace_bytes(C.byref(sim.lattice))
    ws = torch.empty(nbytes // 8 + 1, dtype=torch.float64, device="cuda")
    p = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    assert L.lib().pplbm_adjoint_step(sim.ctx, p(f), p(l1), p(l0), p(grad), p(ws), nbytes) == L.PPLBM_ERR_STATE
    sim.close()


@pytest.mark.parametrize("bc", [BC_PER, BC_WALLS], ids=["periodic", "walls"])
def test_two_phase_rollout_matches_oracle_reference_adjoint(bc):
    nx, ny, nsteps = 24, 24, 30
    olat, _ = make_pair(nx, ny, bc, CASE, TWO_PHASE)
    e = olat.eos
    if bc == BC_WALLS:
        # a film on the bottom wall under a drop (the walled set-up of Sec. IV); the
        # vapour term of the loss is read at the top wall's corner
        rho0 = I.impact(nx, ny, 5.0, 4, e.rho_v, e.rho_l, 0.0, W=5.0)[0]
    else:
        rho0 = I.droplet(nx, ny, 6.0, e.rho_v, e.rho_l, W=5.0)

    def loss_fn(rho):
        phi = (rho - e.rho_v) / (e.rho_l - e.rho_v)
        reff = torch.sqrt(phi.sum() / math.pi)
        return ((rho[ny - 1, 0] - e.rho_v) / e.rho_v) ** 2 + ((reff - 6.0) / 6.0) ** 2

    c = A.constants_as_tensors(e)
    r0 = torch.tensor(rho0, requires_grad=True)
    g = torch.stack([float(w) * r0 for w in A._W])
    for _ in range(nsteps):
        g = A.step(g, olat, c)
    loss = loss_fn(g.sum(0))
    loss.backward()
    dc = A.constants_derivative(*CASE[:4], CASE[4])
    galpha_cpu = sum(float(c[k].grad) * dc[k] for k in A.CONST_NAMES)
    spec = AD.RolloutSpec(nx, ny, bc, P.EOSParams(P.EOS_SMOOTH, 0.5, 0.363, 2.0, 0.775),
                          P.Relax(kind=P.RELAX_TWO_PHASE, tau_l=0.6, visc_ratio=3.0), nsteps, interval=7)
    rho0_t = torch.tensor(rho0, device="cuda", requires_grad=True)
    alpha = torch.tensor(0.775, dtype=torch.float64, requires_grad=True)
    rhoN = AD.rollout(rho0_t, alpha, spec)
    lg = loss_fn(rhoN)
    lg.backward()
    assert float(lg.detach()) == pytest.approx(float(loss.detach()), rel=1e-8)
    assert normwise(rho0_t.grad.cpu().numpy(), r0.grad.numpy()) < 1e-8
    assert float(alpha.grad) == pytest.approx(galpha_cpu, rel=1e-6)


def test_two_phase_walled_rollout_300_steps_against_finite_differences():
    """A drop resting above a liquid film between walls (96 x 64, T_r = 0.5, Smooth
    C-S, tau_l = 0.6, v_r = 3), 300 steps with sqrt(N) checkpoints; loss = squared
    vapour-density error at the top wall's corner + radius mismatch of the liquid
    content. dL/dalpha and the derivative along a random direction of rho0 against
    central differences of the forward rollout, h = 1e-6."""
    nx, ny, nsteps, R0 = 96, 64, 300, 12.0
    eosp = P.EOSParams(P.EOS_SMOOTH, 0.5, 0.363, 2.0, 0.775)
    relax = P.Relax(kind=P.RELAX_TWO_PHASE, tau_l=0.6, visc_ratio=3.0)
    d = P.eos_setup(eosp)
    rv, rl = d["rho_v"], d["rho_l"]
    rho_np, _, _ = I.impact(nx, ny, R0, 10, rv, rl, 0.0, W=6.0)
    rho0 = torch.tensor(rho_np, device="cuda")
    spec = AD.RolloutSpec(nx, ny, P.BC_WALLS_Y, eosp, relax, nsteps, interval=17)

    def loss_of(rho):
        phi = (rho - rv) / (rl - rv)
        reff = torch.sqrt(phi.sum() / math.pi)
        return ((rho[ny - 1, 0] - rv) / rv) ** 2 + ((reff - 30.0) / 30.0) ** 2

    r0 = rho0.clone().requires_grad_(True)
    alpha = torch.tensor(0.775, dtype=torch.float64, requires_grad=True)
    loss_of(AD.rollout(r0, alpha, spec)).backward()

    def loss_at(al, rho):
        with torch.no_grad():
            return float(loss_of(AD.rollout(rho, torch.tensor(al, dtype=torch.float64), spec)))

    h = 1e-6
    fd_alpha = (loss_at(0.775 + h, rho0) - loss_at(0.775 - h, rho0)) / (2 * h)
    assert abs(fd_alpha) > 0
    assert float(alpha.grad) == pytest.approx(fd_alpha, rel=1e-6)
    v = torch.tensor(np.random.default_rng(9).standard_normal((ny, nx)), device="cuda") * rho0
    fd_rho = (loss_at(0.775, rho0 + h * v) - loss_at(0.775, rho0 - h * v)) / (2 * h)
    assert float((r0.grad * v).sum()) == pytest.approx(fd_rho, rel=1e-6)


def test_two_phase_stored_and_checkpointed_rollouts_are_bitwise_equal():
    """Six stored planes per step (psi, rho, j, the stress moments) feed the adjoint the
    values the checkpointed recomputation does, for every interval."""
    nx, ny, nsteps = 40, 36, 30
    eosp = P.EOSParams(P.EOS_SMOOTH, 0.5, 0.363, 2.0, 0.775)
    relax = P.Relax(kind=P.RELAX_TWO_PHASE, tau_l=0.6, visc_ratio=3.0, kappa=0.3)
    d = P.eos_setup(eosp)
    # a drop above a film on the bottom wall (the walled set-up of Sec. IV), perturbed
    rho0 = I.perturbed(I.impact(nx, ny, 7.0, 6, d["rho_v"], d["rho_l"], 0.0, W=6.0)[0], 0.002, 31)
    out = []
    for interval in (0, 1, 3, 6):
        spec = AD.RolloutSpec(nx, ny, P.BC_WALLS_Y, eosp, relax, nsteps, interval=interval)
        assert spec.stored() == (interval == 0)
        r0 = torch.tensor(rho0, device="cuda", requires_grad=True)
        alpha = torch.tensor(0.775, dtype=torch.float64, requires_grad=True)
        rhoN = AD.rollout(r0, alpha, spec)
        (rhoN ** 2).sum().backward()
        out.append((rhoN.detach().cpu(), r0.grad.cpu(), float(alpha.grad)))
    for o in out[1:]:
        assert torch.equal(o[0], out[0][0])
        assert torch.equal(o[1], out[0][1]) and o[2] == out[0][2]
