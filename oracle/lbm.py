"""Oracle: one time step of the pseudopotential D2Q9 lattice Boltzmann method.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). Plain numpy in float64,
vectorised over lattice nodes only; per node the arithmetic follows the paper's
equations in the paper's order:

1. density and pseudopotential: rho = sum_i f_i (Eq. Density), p = p_EOS(rho),
   psi(rho) (Eq. InteractionPotential);
2. Shan-Chen force F = -G psi(x) sum_i w(|c_i|^2) psi(x + c_i) c_i with
   w(1) = 1/3, w(2) = 1/12 (Eq. ShanChenForce); walls use ghost nodes of density
   rho_l (bottom) and rho_v (top) (Sec. IV);
3. velocity rho u = sum_i f_i c_i + F/2 (Eq. Momentum);
4. MRT collision with forcing in moment space: m = M f (Eq. MatrixMRT),
   m_eq = M f_eq (Eq. EquilibriumDistribution), source S of the Li scheme
   (Eq. LiFS; sigma = 0 gives the Guo scheme, Eq. GFS),
   m* = m - Lambda (m - m_eq) + (I - Lambda/2) S (Eqs. LBE, OperatorMRT, GFS),
   f* = M^-1 m*;
5. streaming f_i(x + c_i, t + 1) = f*_i(x, t) (Eq. LBE), periodic, or half-way
   bounce-back at the walls (Sec. IV, App. B).

Optional surface-tension control (``Relax.kappa``, 0 = off): the technique the
paper's discussion (Sec. V) names for keeping the Weber number when alpha lowers
the surface tension, Li & Luo's source term (Phys. Rev. E 88, 053307, 2013),
added to m* in step 4; see ``surface_tension_source``.

Array layout: f has shape (9, ny, nx); index [i, y, x]; x is the fastest axis.
Relaxation: ``Relax`` holds either six constant relaxation times (Eq.
RelaxationMatrix) or the density-dependent two-phase form of Sec. IV
(Eq. RelaxationTime).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# D2Q9 velocity set, Eq. VelocitySet (Sec. II.A)
C = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]], dtype=np.int64)
# weights below Eq. EquilibriumDistribution
W = np.array([4 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 36, 1 / 36, 1 / 36, 1 / 36])
CS2 = 1.0 / 3.0
# opposite direction of each velocity
OPP = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6])
# MRT transformation matrix, Eq. MatrixMRT
M = np.array(
    [
        [1, 1, 1, 1, 1, 1, 1, 1, 1],
        [-4, -1, -1, -1, -1, 2, 2, 2, 2],
        [4, -2, -2, -2, -2, 1, 1, 1, 1],
        [0, 1, 0, -1, 0, 1, -1, -1, 1],
        [0, -2, 0, 2, 0, 1, -1, -1, 1],
        [0, 0, 1, 0, -1, 1, 1, -1, -1],
        [0, 0, -2, 0, 2, 1, 1, -1, -1],
        [0, 1, -1, 1, -1, 0, 0, 0, 0],
        [0, 0, 0, 0, 0, 1, -1, 1, -1],
    ],
    dtype=np.float64,
)
MINV = np.linalg.inv(M)
# Shan-Chen interaction weights w(|c|^2), below Eq. ShanChenForce
W_SC = np.array([0.0, 1 / 3, 1 / 3, 1 / 3, 1 / 3, 1 / 12, 1 / 12, 1 / 12, 1 / 12])

# boundary flags
BC_PERIODIC_X = 1
BC_PERIODIC_Y = 2
BC_WALL_BOTTOM = 4
BC_WALL_TOP = 8

RELAX_MRT = 0        # six constant relaxation times, Eq. RelaxationMatrix
RELAX_TWO_PHASE = 1  # diag(1,1,1,1,1,1,1,1/tau,1/tau), tau(rho) of Eq. RelaxationTime


@dataclass
class Relax:
    kind: int = RELAX_MRT
    tau_rho: float = 1.0
    tau_e: float = 1.0
    tau_zeta: float = 1.0
    tau_j: float = 1.0
    tau_q: float = 1.0
    tau_nu: float = 1.0
    tau_l: float = 1.0
    visc_ratio: float = 1.0
    sigma: float = 0.0   # Li forcing parameter; 0 = Guo forcing
    kappa: float = 0.0   # surface-tension control (Sec. V; Li & Luo 2013); 0 = off


def equilibrium(rho, ux, uy):
    """f_eq_i = w_i (rho + c.(rho u)/cs^2 + (c c - cs^2 I):(rho u u)/(2 cs^4)), Eq. EquilibriumDistribution."""
    feq = np.empty((9,) + np.shape(rho))
    for i in range(9):
        cu = C[i, 0] * ux + C[i, 1] * uy
        uu = ux * ux + uy * uy
        feq[i] = W[i] * (rho + cu * rho / CS2 + (cu * cu - CS2 * uu) * rho / (2.0 * CS2 * CS2))
    return feq


def _neighbour(field, dx, dy, bc, ghost_bottom, ghost_top):
    """field(x + dx, y + dy): periodic in x; periodic in y, or a ghost row beyond a wall."""
    ny = field.shape[0]
    out = np.roll(field, shift=(-dy, -dx), axis=(0, 1))
    if not (bc & BC_PERIODIC_Y):
        if dy == 1:
            out[ny - 1, :] = ghost_top
        elif dy == -1:
            out[0, :] = ghost_bottom
    return out


def shan_chen_force(psi, G, bc, psi_ghost_bottom=0.0, psi_ghost_top=0.0):
    """Eq. ShanChenForce: F = -G psi(x) sum_i w(|c_i|^2) psi(x + c_i) c_i."""
    sx = np.zeros_like(psi)
    sy = np.zeros_like(psi)
    for i in range(1, 9):
        nb = _neighbour(psi, C[i, 0], C[i, 1], bc, psi_ghost_bottom, psi_ghost_top)
        sx += W_SC[i] * nb * C[i, 0]
        sy += W_SC[i] * nb * C[i, 1]
    return -G * psi * sx, -G * psi * sy


def relaxation_rates(relax: Relax, rho, rho_v, rho_l):
    """Diagonal of Lambda per node, shape (9,) + rho.shape (Eq. RelaxationMatrix / Sec. IV)."""
    lam = np.empty((9,) + rho.shape)
    if relax.kind == RELAX_MRT:
        taus = [relax.tau_rho, relax.tau_e, relax.tau_zeta, relax.tau_j, relax.tau_q,
                relax.tau_j, relax.tau_q, relax.tau_nu, relax.tau_nu]
        for k in range(9):
            lam[k] = 1.0 / taus[k]
    elif relax.kind == RELAX_TWO_PHASE:
        tau_v = 0.5 + relax.visc_ratio * (relax.tau_l - 0.5)
        tau = relax.tau_l * (rho - rho_v) / (rho_l - rho_v) + tau_v * (rho - rho_l) / (rho_v - rho_l)
        lam[:7] = 1.0
        lam[7] = 1.0 / tau
        lam[8] = 1.0 / tau
    else:
        raise ValueError("unknown relaxation kind")
    return lam


def tau_e_zeta(relax: Relax):
    if relax.kind == RELAX_MRT:
        return relax.tau_e, relax.tau_zeta
    return 1.0, 1.0


def li_source(ux, uy, Fx, Fy, psi, sigma, tau_e, tau_zeta):
    """Moment-space forcing vector of Eq. LiFS (sigma = 0: the Guo scheme's M F')."""
    uF = ux * Fx + uy * Fy
    F2 = Fx * Fx + Fy * Fy
    S = np.empty((9,) + ux.shape)
    S[0] = 0.0
    S[1] = 6.0 * uF + 12.0 * sigma * F2 / (psi**2 * (tau_e - 0.5))
    S[2] = -6.0 * uF - 12.0 * sigma * F2 / (psi**2 * (tau_zeta - 0.5))
    S[3] = Fx
    S[4] = -Fx
    S[5] = Fy
    S[6] = -Fy
    S[7] = 2.0 * (ux * Fx - uy * Fy)
    S[8] = ux * Fy + uy * Fx
    return S


def surface_tension_q(psi, G, kappa, bc, psi_ghost_bottom=0.0, psi_ghost_top=0.0):
    """Q_ab = kappa (G/2) psi(x) sum_i w(|c_i|^2) [psi(x + c_i) - psi(x)] c_ia c_ib, the
    tensor of the surface-tension control the paper's Sec. V names (Li & Luo 2013),
    with the Shan-Chen weights of Eq. ShanChenForce and the same wall ghosts.
    Returns Q_xx, Q_yy, Q_xy."""
    qxx = np.zeros_like(psi)
    qyy = np.zeros_like(psi)
    qxy = np.zeros_like(psi)
    for i in range(1, 9):
        d = _neighbour(psi, C[i, 0], C[i, 1], bc, psi_ghost_bottom, psi_ghost_top) - psi
        qxx += W_SC[i] * d * C[i, 0] * C[i, 0]
        qyy += W_SC[i] * d * C[i, 1] * C[i, 1]
        qxy += W_SC[i] * d * C[i, 0] * C[i, 1]
    k = kappa * G / 2.0 * psi
    return k * qxx, k * qyy, k * qxy


def surface_tension_source(qxx, qyy, qxy, lam):
    """Moment-space source added to m* by the surface-tension control (Li & Luo 2013):
    C = [0, 1.5 l_e (Q_xx + Q_yy), -1.5 l_zeta (Q_xx + Q_yy), 0, 0, 0, 0,
    -l_nu (Q_xx - Q_yy), -l_nu Q_xy] with l_k the diagonal of Lambda (Eq. RelaxationMatrix)
    for the rows of Eq. MatrixMRT."""
    Cs = np.zeros((9,) + qxx.shape)
    Cs[1] = 1.5 * lam[1] * (qxx + qyy)
    Cs[2] = -1.5 * lam[2] * (qxx + qyy)
    Cs[7] = -lam[7] * (qxx - qyy)
    Cs[8] = -lam[8] * qxy
    return Cs


@dataclass
class Lattice:
    nx: int
    ny: int
    bc: int          # BC_* flags
    eos: object      # oracle.eos.EOS
    relax: Relax

    def __post_init__(self):
        if not (self.bc & BC_PERIODIC_X):
            raise ValueError("x must be periodic")
        walls = self.bc & (BC_WALL_BOTTOM | BC_WALL_TOP)
        if self.bc & BC_PERIODIC_Y:
            if walls:
                raise ValueError("y is either periodic or walled")
        elif walls != (BC_WALL_BOTTOM | BC_WALL_TOP):
            raise ValueError("walled y needs both walls")
        # ghost densities inside the walls (Sec. IV): liquid below, vapour above
        self.psi_ghost_bottom = float(self.eos.psi(self.eos.rho_l))
        self.psi_ghost_top = float(self.eos.psi(self.eos.rho_v))

    # -- step pieces ----------------------------------------------------------------
    def macroscopic(self, f):
        """rho, ux, uy, psi, Fx, Fy at the state f (Eqs. Density, Momentum, ShanChenForce)."""
        rho = f.sum(axis=0)
        psi = self.eos.psi(rho)
        Fx, Fy = shan_chen_force(psi, self.eos.G, self.bc, self.psi_ghost_bottom, self.psi_ghost_top)
        jx = np.einsum("i,iyx->yx", C[:, 0].astype(np.float64), f)
        jy = np.einsum("i,iyx->yx", C[:, 1].astype(np.float64), f)
        ux = (jx + Fx / 2.0) / rho
        uy = (jy + Fy / 2.0) / rho
        return rho, ux, uy, psi, Fx, Fy

    def collide(self, f):
        rho, ux, uy, psi, Fx, Fy = self.macroscopic(f)
        m = np.einsum("ki,iyx->kyx", M, f)
        meq = np.einsum("ki,iyx->kyx", M, equilibrium(rho, ux, uy))
        te, tz = tau_e_zeta(self.relax)
        S = li_source(ux, uy, Fx, Fy, psi, self.relax.sigma, te, tz)
        lam = relaxation_rates(self.relax, rho, self.eos.rho_v, self.eos.rho_l)
        mstar = m - lam * (m - meq) + (1.0 - lam / 2.0) * S
        if self.relax.kappa != 0.0:
            q = surface_tension_q(psi, self.eos.G, self.relax.kappa, self.bc, self.psi_ghost_bottom,
                                  self.psi_ghost_top)
            mstar = mstar + surface_tension_source(*q, lam)
        return np.einsum("ik,kyx->iyx", MINV, mstar)

    def stream(self, fstar):
        """f_i(x + c_i, t + 1) = f*_i(x, t); half-way bounce-back at walls."""
        fn = np.empty_like(fstar)
        for i in range(9):
            fn[i] = np.roll(fstar[i], shift=(C[i, 1], C[i, 0]), axis=(0, 1))
        if not (self.bc & BC_PERIODIC_Y):
            ny = self.ny
            for i in range(9):
                if C[i, 1] == 1:     # arrives at y = 0 from the bottom wall: reflected c_{opp(i)}
                    fn[i, 0, :] = fstar[OPP[i], 0, :]
                elif C[i, 1] == -1:  # arrives at y = ny-1 from the top wall
                    fn[i, ny - 1, :] = fstar[OPP[i], ny - 1, :]
        return fn

    def step(self, f, n=1):
        for _ in range(n):
            f = self.stream(self.collide(f))
        return f

    def init_equilibrium(self, rho0, ux0=None, uy0=None):
        """f(t = 0) = f_eq(rho0, u0) (Sec. III.A)."""
        ux0 = np.zeros_like(rho0) if ux0 is None else ux0
        uy0 = np.zeros_like(rho0) if uy0 is None else uy0
        return equilibrium(np.asarray(rho0, dtype=np.float64), ux0, uy0)


def convergence_residual(rho_now, rho_before):
    """sum |rho(t) - rho(t - 100)| / sum |rho(t)| (Sec. III.A)."""
    return float(np.abs(rho_now - rho_before).sum() / np.abs(rho_now).sum())


def vapor_density_error(rho_v_sim, rho_v_maxwell):
    """Eq. DensityError: 100 (rho_v - rho_v^M) / rho_v^M."""
    return 100.0 * (rho_v_sim - rho_v_maxwell) / rho_v_maxwell


def interface_width(profile, rho_v, rho_l):
    """Number of nodes with 0.01 < (rho - rho_v)/(rho_l - rho_v) < 0.99 along one interface
    of a 1-D profile (Sec. III.A definition); the first interface from index 0 is used."""
    phi = (np.asarray(profile) - rho_v) / (rho_l - rho_v)
    half = len(phi) // 2
    seg = phi[:half]
    return int(np.count_nonzero((seg > 0.01) & (seg < 0.99)))


def surface_tension_planar(psi_profile, G=-1.0):
    """Eq. SurfaceTension: gamma = -(G c^4/6) int (dpsi/dx)^2 dx, with a fourth-order
    central difference for dpsi/dx and Simpson's rule (Sec. IV.A).

    The profile is periodic and crosses two interfaces (a liquid slab in vapour),
    so gamma is half of the integral over the whole period."""
    p = np.asarray(psi_profile, dtype=np.float64)
    d = (-np.roll(p, -2) + 8 * np.roll(p, -1) - 8 * np.roll(p, 1) + np.roll(p, 2)) / 12.0
    g = d * d
    n = len(g)
    # composite Simpson over the periodic profile (closed on itself): append the first point
    y = np.concatenate([g, g[:1]])
    if n % 2:
        raise ValueError("Simpson's rule needs an even number of intervals")
    w = np.ones(n + 1)
    w[1:-1:2] = 4.0
    w[2:-1:2] = 2.0
    integral = float(np.sum(w * y) / 3.0)
    return -G / 6.0 * integral / 2.0
