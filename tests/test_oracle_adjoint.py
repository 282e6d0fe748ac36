"""Pins for the oracle's reference adjoint (CPU only): the torch restatement of
the step equals the numpy oracle step, and its reverse-mode gradients agree with
central finite differences of the numpy oracle (w.r.t. the initial field and the
shaping parameter alpha), also with the surface-tension control on (kappa)."""
import numpy as np
import pytest

import lbm_inputs as I
from oracle import adjoint as A
from oracle import eos as E
from oracle import lbm as L

torch = pytest.importorskip("torch")

CASE = (E.MODE_SMOOTH, 0.5, 0.363, 2.0, 0.775)
PER = L.BC_PERIODIC_X | L.BC_PERIODIC_Y
WALLS = L.BC_PERIODIC_X | L.BC_WALL_BOTTOM | L.BC_WALL_TOP


def lattice(nx, ny, bc, alpha=CASE[4], kappa=0.0):
    e = E.make_eos(CASE[0], CASE[1], CASE[2], CASE[3], alpha)
    e.solve_eps(n=40000)
    return L.Lattice(nx, ny, bc, e, L.Relax(sigma=e.sigma(), kappa=kappa))


def initial(lat, nx, ny, bc):
    e = lat.eos
    if bc == WALLS:
        rho, ux, uy = I.impact(nx, ny, 3, 4, e.rho_v, e.rho_l, 0.01, W=6.0)
    else:
        rho = I.perturbed(I.droplet(nx, ny, min(nx, ny) / 4, e.rho_v, e.rho_l, W=4.0), 0.01, 1)
        ux, uy = I.random_velocity((ny, nx), 0.005, 2)
    return lat.init_equilibrium(rho, ux, uy)


@pytest.mark.parametrize("kappa", [0.0, 0.6])
@pytest.mark.parametrize("bc", [PER, WALLS], ids=["periodic", "walls"])
def test_torch_step_equals_numpy_oracle(bc, kappa):
    lat = lattice(12, 10, bc, kappa=kappa)
    f = initial(lat, 12, 10, bc)
    c = A.constants_as_tensors(lat.eos, requires_grad=False)
    g = torch.tensor(f)
    for _ in range(4):
        f = lat.step(f, 1)
        g = A.step(g, lat, c)
    assert np.max(np.abs(g.numpy() - f)) < 1e-14 * np.max(np.abs(f))


@pytest.mark.parametrize("kappa", [0.0, 0.6])
@pytest.mark.parametrize("bc", [PER, WALLS], ids=["periodic", "walls"])
def test_gradient_wrt_initial_field_matches_finite_differences(bc, kappa):
    nx, ny, steps = 10, 12, 5
    lat = lattice(nx, ny, bc, kappa=kappa)
    e = lat.eos
    f0 = initial(lat, nx, ny, bc)
    c = A.constants_as_tensors(e, requires_grad=False)
    x = torch.tensor(f0, requires_grad=True)
    g = x
    for _ in range(steps):
        g = A.step(g, lat, c)
    loss = A.droplet_loss(g.sum(0), e.rho_v, e.rho_l, 2.5)
    loss.backward()
    v = np.random.default_rng(3).standard_normal(f0.shape) * f0
    h = 1e-6

    def Lnp(f):
        rho = lat.step(f, steps).sum(0)
        return float(A.droplet_loss(torch.tensor(rho), e.rho_v, e.rho_l, 2.5))

    fd = (Lnp(f0 + h * v) - Lnp(f0 - h * v)) / (2 * h)
    ad = float((x.grad.numpy() * v).sum())
    assert ad == pytest.approx(fd, rel=1e-6)


def test_gradient_wrt_alpha_matches_finite_differences():
    nx, ny, steps = 12, 12, 6
    alpha = CASE[4]
    lat = lattice(nx, ny, PER, alpha)
    e = lat.eos
    rho0 = I.droplet(nx, ny, 3.0, e.rho_v, e.rho_l, W=4.0)
    c = A.constants_as_tensors(e)
    g = torch.tensor(lat.init_equilibrium(rho0))
    for _ in range(steps):
        g = A.step(g, lat, c)
    loss = A.droplet_loss(g.sum(0), e.rho_v, e.rho_l, 3.0)
    loss.backward()
    dc = A.constants_derivative(*CASE[:4], alpha)
    ad = sum(float(c[k].grad) * dc[k] for k in A.CONST_NAMES)

    def Lalpha(al):
        lt = lattice(nx, ny, PER, al)
        rho = lt.step(lt.init_equilibrium(rho0), steps).sum(0)
        return float(A.droplet_loss(torch.tensor(rho), e.rho_v, e.rho_l, 3.0))

    h = 1e-4
    fd = (Lalpha(alpha + h) - Lalpha(alpha - h)) / (2 * h)
    assert ad == pytest.approx(fd, rel=1e-5)


@pytest.mark.parametrize("wrt", ["a_v", "a_l"])
def test_gradient_wrt_branch_parameters_matches_finite_differences(wrt):
    """d loss / d a_v and d a_l: the vapour branch C-S(a_v, T_v), the liquid branch
    C-S(a_l, T_l) + Delta P and the shaped loop all move with them (Sec. III.D, the
    higher vapour sound speed variant); the Maxwell densities do not (fixed T_r)."""
    nx, ny, steps = 12, 12, 6
    base = {"a_l": CASE[2], "a_v": CASE[3]}

    def make(v):
        args = dict(base)
        args[wrt] = v
        e = E.make_eos(CASE[0], CASE[1], args["a_l"], args["a_v"], CASE[4])
        e.solve_eps(n=40000)
        return L.Lattice(nx, ny, PER, e, L.Relax(sigma=e.sigma()))

    lat = make(base[wrt])
    e = lat.eos
    rho0 = I.perturbed(I.droplet(nx, ny, 3.0, e.rho_v, e.rho_l, W=4.0), 0.01, 4)
    c = A.constants_as_tensors(e)
    g = torch.tensor(lat.init_equilibrium(rho0))
    for _ in range(steps):
        g = A.step(g, lat, c)
    loss = A.droplet_loss(g.sum(0), e.rho_v, e.rho_l, 3.0)
    loss.backward()
    dc = A.constants_derivative(CASE[0], CASE[1], base["a_l"], base["a_v"], CASE[4], wrt=wrt)
    ad = sum(float(c[k].grad) * dc[k] for k in A.CONST_NAMES)

    def Lv(v):
        lt = make(v)
        assert lt.eos.rho_v == pytest.approx(e.rho_v, rel=1e-12)
        rho = lt.step(lt.init_equilibrium(rho0), steps).sum(0)
        return float(A.droplet_loss(torch.tensor(rho), e.rho_v, e.rho_l, 3.0))

    h = 1e-4
    fd = (Lv(base[wrt] + h) - Lv(base[wrt] - h)) / (2 * h)
    assert ad != 0.0
    assert ad == pytest.approx(fd, rel=1e-5)


@pytest.mark.parametrize("kappa", [0.0, 0.4])
@pytest.mark.parametrize("bc", [PER, WALLS], ids=["periodic", "walls"])
def test_gradient_wrt_kappa_matches_finite_differences(bc, kappa):
    """dL/dkappa of the surface-tension control through the torch restatement
    (kappa as a tensor in the constants) against central differences of the numpy
    oracle over 5 steps, L = sum rho^2 (a loss of moderate size, so the differences
    are not lost to rounding)."""
    nx, ny, steps = 12, 10, 5
    lat = lattice(nx, ny, bc, kappa=kappa)
    e = lat.eos
    f0 = initial(lat, nx, ny, bc)
    c = A.constants_as_tensors(e, requires_grad=False)
    c["kappa"] = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
    g = torch.tensor(f0)
    for _ in range(steps):
        g = A.step(g, lat, c)
    (g.sum(0) ** 2).sum().backward()
    h = 1e-5

    def Lnp(k):
        rho = L.Lattice(nx, ny, bc, e, L.Relax(sigma=e.sigma(), kappa=k)).step(f0, steps).sum(0)
        return float((rho ** 2).sum())

    fd = (Lnp(kappa + h) - Lnp(kappa - h)) / (2 * h)
    assert abs(fd) > 1e-8
    assert float(c["kappa"].grad) == pytest.approx(fd, rel=1e-6)


# ---- the two-phase relaxation of the dynamic runs (Sec. IV, Eq. RelaxationTime) ----

def lattice_two_phase(nx, ny, bc, alpha=CASE[4], kappa=0.0, tau_l=0.6, visc_ratio=3.0):
    e = E.make_eos(CASE[0], CASE[1], CASE[2], CASE[3], alpha)
    e.solve_eps(n=40000)
    return L.Lattice(nx, ny, bc, e, L.Relax(kind=L.RELAX_TWO_PHASE, tau_l=tau_l, visc_ratio=visc_ratio,
                                            sigma=e.sigma(), kappa=kappa))


@pytest.mark.parametrize("kappa", [0.0, 0.6])
@pytest.mark.parametrize("bc", [PER, WALLS], ids=["periodic", "walls"])
def test_two_phase_torch_step_equals_numpy_oracle(bc, kappa):
    """The restatement with Lambda = diag(1, ..., 1, 1/tau(rho), 1/tau(rho)) equals the
    numpy oracle's step (whose tau(rho) end points are pinned in test_oracle_lbm)."""
    lat = lattice_two_phase(12, 10, bc, kappa=kappa)
    f = initial(lat, 12, 10, bc)
    c = A.constants_as_tensors(lat.eos, requires_grad=False)
    g = torch.tensor(f)
    for _ in range(4):
        f = lat.step(f, 1)
        g = A.step(g, lat, c)
    assert np.max(np.abs(g.numpy() - f)) < 1e-14 * np.max(np.abs(f))


@pytest.mark.parametrize("bc", [PER, WALLS], ids=["periodic", "walls"])
def test_two_phase_gradient_wrt_initial_field_matches_finite_differences(bc):
    """Reverse mode through tau(rho) as well: the derivative of the droplet loss after 5
    steps along a random direction equals central differences (h = 1e-6) of the numpy
    oracle."""
    nx, ny, steps = 10, 12, 5
    lat = lattice_two_phase(nx, ny, bc)
    e = lat.eos
    f0 = initial(lat, nx, ny, bc)
    c = A.constants_as_tensors(e, requires_grad=False)
    x = torch.tensor(f0, requires_grad=True)
    g = x
    for _ in range(steps):
        g = A.step(g, lat, c)
    loss = A.droplet_loss(g.sum(0), e.rho_v, e.rho_l, 2.5)
    loss.backward()
    v = np.random.default_rng(4).standard_normal(f0.shape) * f0
    h = 1e-6

    def Lnp(f):
        rho = lat.step(f, steps).sum(0)
        return float(A.droplet_loss(torch.tensor(rho), e.rho_v, e.rho_l, 2.5))

    fd = (Lnp(f0 + h * v) - Lnp(f0 - h * v)) / (2 * h)
    ad = float((x.grad.numpy() * v).sum())
    assert ad == pytest.approx(fd, rel=1e-6)


def test_two_phase_gradient_wrt_alpha_matches_finite_differences():
    """dL/dalpha through the constants with the two-phase relaxation, walls: autograd
    of the restatement chained with constants_derivative against central differences
    of the numpy oracle rebuilt at alpha +- h."""
    nx, ny, steps = 12, 12, 6
    alpha = CASE[4]
    lat = lattice_two_phase(nx, ny, WALLS, alpha)
    e = lat.eos
    rho0, ux0, uy0 = I.impact(nx, ny, 3, 4, e.rho_v, e.rho_l, 0.01, W=6.0)
    c = A.constants_as_tensors(e)
    g = A.step(torch.tensor(lat.init_equilibrium(rho0, ux0, uy0)), lat, c)
    for _ in range(steps - 1):
        g = A.step(g, lat, c)
    A.droplet_loss(g.sum(0), e.rho_v, e.rho_l, 3.0).backward()
    dc = A.constants_derivative(*CASE[:4], alpha)
    ad = sum(float(c[k].grad) * dc[k] for k in A.CONST_NAMES)
    h = 1e-5

    def Lnp(a):
        la = lattice_two_phase(nx, ny, WALLS, a)
        # the same initial field (the Maxwell densities do not depend on alpha)
        rho = la.step(la.init_equilibrium(rho0, ux0, uy0), steps).sum(0)
        return float(A.droplet_loss(torch.tensor(rho), e.rho_v, e.rho_l, 3.0))

    fd = (Lnp(alpha + h) - Lnp(alpha - h)) / (2 * h)
    assert ad == pytest.approx(fd, rel=1e-6)
