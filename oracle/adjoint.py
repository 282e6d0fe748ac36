"""Oracle: reference adjoint (reverse-mode gradients) of the lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). The step of
``oracle/lbm.py`` is restated with plain PyTorch CPU float64 tensor operations,
in the same order (rho, psi, Shan-Chen force, u, m = M f, m_eq, Li source S,
m* = m - Lambda (m - m_eq) + (I - Lambda/2) S, f* = M^-1 m*, streaming with
half-way bounce-back), and torch.autograd supplies the exact reverse-mode
derivatives of that arithmetic. The EOS enters through its derived constants
(p_max, b1, a1^2, p_min, b3, a3^2 of Sec. III.D, sigma, and the C-S parameters
a, T of the vapour and liquid branches with the liquid shift Delta P), which are
inputs here; their dependence on a parameter (alpha, a_v or a_l) is taken from the
numpy oracle by central differences with Richardson extrapolation.

Two relaxation sets are restated: unit relaxation times (Lambda = I, Sec. III.A)
and the two-phase set of the dynamic runs (Sec. IV): Lambda = diag(1, ..., 1,
1/tau, 1/tau) with tau(rho) linear between tau_v at rho_v and tau_l at rho_l
(Eq. RelaxationTime), so that autograd also differentiates through tau(rho). Both
carry the optional surface-tension source of ``oracle/lbm.py`` (``Relax.kappa``;
the technique the paper's Sec. V names, Li & Luo 2013), whose moment vector is
C = [0, 1.5 l_e tr Q, -1.5 l_zeta tr Q, 0, 0, 0, 0, -l_nu (Q_xx - Q_yy), -l_nu Q_xy]
with l the diagonal of Lambda.
"""
from __future__ import annotations

import numpy as np
import torch

from . import eos as E
from . import lbm as L

CONST_NAMES = ("p_max", "b1", "a1sq", "p_min", "b3", "a3sq", "sigma", "a_v", "T_v", "a_l", "T_l", "dP")

_C = torch.tensor(L.C, dtype=torch.float64)
_W = torch.tensor(L.W, dtype=torch.float64)
_M = torch.tensor(L.M, dtype=torch.float64)
_MINV = torch.tensor(L.MINV, dtype=torch.float64)
_WSC = torch.tensor(L.W_SC, dtype=torch.float64)


def eos_constants(eos):
    """The constants of a Smooth C-S oracle EOS that its parameters move: those of
    the shaped branches, sigma, and the C-S parameters of both bulk branches."""
    return {"p_max": eos.p_max, "b1": eos.b1, "a1sq": eos.a1sq, "p_min": eos.p_min, "b3": eos.b3,
            "a3sq": eos.a3sq, "sigma": eos.sigma(), "a_v": eos.a_v, "T_v": eos.T_v, "a_l": eos.a_l,
            "T_l": eos.T_l, "dP": eos.dP}


def constants_derivative(mode, Tr, a_l, a_v, alpha, h=1e-3, wrt="alpha"):
    """d(constant)/d(theta), theta = alpha, a_v or a_l (`wrt`), for each of CONST_NAMES:
    central differences of the oracle's set-up at steps h and h/2 combined by
    Richardson extrapolation."""
    def at(v):
        args = {"alpha": alpha, "a_v": a_v, "a_l": a_l}
        args[wrt] = v
        e = E.make_eos(mode, Tr, args["a_l"], args["a_v"], args["alpha"])
        e.solve_eps(n=40000)
        return np.array([eos_constants(e)[k] for k in CONST_NAMES])

    x = {"alpha": alpha, "a_v": a_v, "a_l": a_l}[wrt]
    d1 = (at(x + h) - at(x - h)) / (2 * h)
    d2 = (at(x + h / 2) - at(x - h / 2)) / h
    return dict(zip(CONST_NAMES, (4 * d2 - d1) / 3))


def _cs_pressure(rho, a, b, R, T):
    eta = b * rho / 4.0
    return rho * R * T * (1.0 + eta + eta**2 - eta**3) / (1.0 - eta) ** 3 - a * rho**2


def pressure(rho, eos, c):
    """Smooth C-S p(rho) (Sec. III.D) with the alpha-dependent constants c as tensors."""
    p = torch.zeros_like(rho)
    m1 = rho <= eos.rho_v
    m2 = (rho > eos.rho_v) & (rho <= eos.rho_max)
    m3 = (rho > eos.rho_max) & (rho < eos.rho_min)
    m4 = (rho >= eos.rho_min) & (rho < eos.rho_l)
    m5 = rho >= eos.rho_l
    p = p.index_put((m1,), _cs_pressure(rho[m1], c["a_v"], eos.b, eos.R, c["T_v"]))
    x = rho[m2]
    p = p.index_put((m2,), c["p_max"] - c["b1"] + c["b1"] * torch.sqrt(1.0 - (x - eos.rho_max) ** 2 / c["a1sq"]))
    t = (rho[m3] - eos.rho_max) / (eos.rho_min - eos.rho_max)
    a2 = 2.0 * (c["p_max"] - c["p_min"])
    b2 = 3.0 * (c["p_min"] - c["p_max"])
    p = p.index_put((m3,), a2 * t**3 + b2 * t**2 + c["p_max"])
    x = rho[m4]
    p = p.index_put((m4,), c["p_min"] + c["b3"] - c["b3"] * torch.sqrt(1.0 - (x - eos.rho_min) ** 2 / c["a3sq"]))
    p = p.index_put((m5,), _cs_pressure(rho[m5], c["a_l"], eos.b, eos.R, c["T_l"]) + c["dP"])
    return p


def _roll(a, dy, dx):
    return torch.roll(a, shifts=(dy, dx), dims=(-2, -1))


def _surface_tension_source(qxx, qyy, qxy, z, lam):
    """The surface-tension source's moment vector (Li & Luo 2013):
    [0, 1.5 l_1 tr Q, -1.5 l_2 tr Q, 0, 0, 0, 0, -l_7 (Q_xx - Q_yy), -l_8 Q_xy], l = lam the
    diagonal of Lambda (l_1 = l_2 = 1 in both restated sets); z a zero plane."""
    return torch.stack([z, 1.5 * lam[1] * (qxx + qyy), -1.5 * lam[2] * (qxx + qyy), z, z, z, z,
                        -lam[7] * (qxx - qyy), -lam[8] * qxy])


def relaxation_diagonal(lat: L.Lattice, rho):
    """Diagonal of Lambda per node, shape (9,) + rho.shape: all ones for unit relaxation
    times (Sec. III.A); for the two-phase set (Sec. IV) rows 7, 8 are 1/tau(rho) with
    tau(rho) = tau_l (rho - rho_v)/(rho_l - rho_v) + tau_v (rho - rho_l)/(rho_v - rho_l),
    tau_v = 1/2 + v_r (tau_l - 1/2) (Eq. RelaxationTime). Other sets are not restated."""
    r = lat.relax
    one = torch.ones_like(rho)
    if r.kind == L.RELAX_TWO_PHASE:
        e = lat.eos
        tau_v = 0.5 + r.visc_ratio * (r.tau_l - 0.5)
        tau = r.tau_l * (rho - e.rho_v) / (e.rho_l - e.rho_v) + tau_v * (rho - e.rho_l) / (e.rho_v - e.rho_l)
        return torch.stack([one] * 7 + [1.0 / tau, 1.0 / tau])
    if r.kind == L.RELAX_MRT and all(t == 1.0 for t in (r.tau_rho, r.tau_e, r.tau_zeta, r.tau_j, r.tau_q, r.tau_nu)):
        return torch.stack([one] * 9)
    raise ValueError("the torch restatement covers unit relaxation times and the two-phase set only")


def step(f, lat: L.Lattice, c):
    """One step, f of shape (9, ny, nx) (torch float64); c: dict of constant tensors."""
    eos = lat.eos
    G = eos.G
    rho = f.sum(dim=0)
    psi = torch.sqrt(2.0 * (pressure(rho, eos, c) - rho / 3.0) / G)
    walls = not (lat.bc & L.BC_PERIODIC_Y)
    ny = lat.ny
    sx = torch.zeros_like(psi)
    sy = torch.zeros_like(psi)
    for i in range(1, 9):
        cx, cy = int(L.C[i, 0]), int(L.C[i, 1])
        nb = _roll(psi, -cy, -cx)
        if walls:
            rows = torch.arange(ny).reshape(ny, 1).expand_as(psi)
            if cy == 1:
                nb = torch.where(rows == ny - 1, torch.full_like(nb, lat.psi_ghost_top), nb)
            elif cy == -1:
                nb = torch.where(rows == 0, torch.full_like(nb, lat.psi_ghost_bottom), nb)
        sx = sx + _WSC[i] * nb * cx
        sy = sy + _WSC[i] * nb * cy
    Fx, Fy = -G * psi * sx, -G * psi * sy
    # kappa: a tensor in c (to differentiate by it) or the lattice's Relax.kappa
    kappa = c["kappa"] if "kappa" in c else lat.relax.kappa
    with_st = torch.is_tensor(kappa) or kappa != 0.0
    if with_st:
        # Q_ab = kappa (G/2) psi(x) sum_i w_i [psi(x + c_i) - psi(x)] c_ia c_ib (same ghosts)
        qxx = torch.zeros_like(psi)
        qyy = torch.zeros_like(psi)
        qxy = torch.zeros_like(psi)
        for i in range(1, 9):
            cx, cy = int(L.C[i, 0]), int(L.C[i, 1])
            nb = _roll(psi, -cy, -cx)
            if walls:
                rows = torch.arange(ny).reshape(ny, 1).expand_as(psi)
                if cy == 1:
                    nb = torch.where(rows == ny - 1, torch.full_like(nb, lat.psi_ghost_top), nb)
                elif cy == -1:
                    nb = torch.where(rows == 0, torch.full_like(nb, lat.psi_ghost_bottom), nb)
            d = nb - psi
            qxx = qxx + _WSC[i] * d * cx * cx
            qyy = qyy + _WSC[i] * d * cy * cy
            qxy = qxy + _WSC[i] * d * cx * cy
        kq = kappa * G / 2.0 * psi
        qxx, qyy, qxy = kq * qxx, kq * qyy, kq * qxy
    jx = torch.einsum("i,iyx->yx", _C[:, 0], f)
    jy = torch.einsum("i,iyx->yx", _C[:, 1], f)
    ux = (jx + Fx / 2.0) / rho
    uy = (jy + Fy / 2.0) / rho
    feq = torch.stack([_W[i] * (rho + 3.0 * (_C[i, 0] * ux + _C[i, 1] * uy) * rho
                                + 4.5 * (_C[i, 0] * ux + _C[i, 1] * uy) ** 2 * rho - 1.5 * (ux**2 + uy**2) * rho)
                       for i in range(9)])
    m = torch.einsum("ki,iyx->kyx", _M, f)
    meq = torch.einsum("ki,iyx->kyx", _M, feq)
    uF = ux * Fx + uy * Fy
    F2 = Fx * Fx + Fy * Fy
    sigma = c["sigma"]
    S = torch.stack([torch.zeros_like(rho), 6.0 * uF + 12.0 * sigma * F2 / (psi**2 * 0.5),
                     -6.0 * uF - 12.0 * sigma * F2 / (psi**2 * 0.5), Fx, -Fx, Fy, -Fy,
                     2.0 * (ux * Fx - uy * Fy), ux * Fy + uy * Fx])
    lam = relaxation_diagonal(lat, rho)
    mstar = m - lam * (m - meq) + (1.0 - lam / 2.0) * S
    if with_st:
        z = torch.zeros_like(rho)
        mstar = mstar + _surface_tension_source(qxx, qyy, qxy, z, lam)
    fstar = torch.einsum("ik,kyx->iyx", _MINV, mstar)
    out = []
    for i in range(9):
        cx, cy = int(L.C[i, 0]), int(L.C[i, 1])
        fi = _roll(fstar[i], cy, cx)
        if walls:
            rows = torch.arange(ny).reshape(ny, 1).expand_as(fi)
            if cy == 1:
                fi = torch.where(rows == 0, fstar[L.OPP[i]], fi)
            elif cy == -1:
                fi = torch.where(rows == ny - 1, fstar[L.OPP[i]], fi)
        out.append(fi)
    return torch.stack(out)


def constants_as_tensors(eos, requires_grad=True):
    return {k: torch.tensor(v, dtype=torch.float64, requires_grad=requires_grad) for k, v in eos_constants(eos).items()}


def droplet_loss(rho, rho_v, rho_l, R0):
    """((rho(0,0) - rho_v)/rho_v)^2 + ((R_eff - R0)/R0)^2, R_eff = sqrt(sum phi / pi),
    phi = (rho - rho_v)/(rho_l - rho_v) (the corner node is farthest from a centred droplet)."""
    phi = (rho - rho_v) / (rho_l - rho_v)
    reff = torch.sqrt(phi.sum() / np.pi)
    return ((rho[0, 0] - rho_v) / rho_v) ** 2 + ((reff - R0) / R0) ** 2
