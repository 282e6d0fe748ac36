"""Oracle: the finite-difference (MacCormack) solver of App. A, periodic domains.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). It integrates the
macroscopic equations the lattice Boltzmann method recovers, written as in
App. A:

  d_t rho   = -(rho d_g u_g + u_g d_g rho)
  d_t u_a   = -u_g d_g u_a - (1/rho) d_a p_EOS - (1/rho) d_b p'_ab + (1/rho) d_b sigma'_ab

with the viscous stress of Eq. StressTensor expanded as Eq. FDstressTensor
(mu = rho c_s^2 (tau_nu - 1/2), mu_B = rho c_s^2 (tau_e - tau_nu), Eq.
DynamicViscosity; their gradients through d mu/d rho, Eq. FDviscosityDerivative)
and d_b p'_ab of Eq. FDforce,

  d_b p'_ab = -eps (G c^4/4) (d_g psi)(d_a d_g psi) + (G c^4/12)(d_a psi)(d_g d_g psi)
              + (G c^4/6)(d_g psi)(d_a d_g psi) + (G c^4/4) psi d_a d_g d_g psi.

With the surface-tension control of the paper's Sec. V (``kappa``; Li & Luo
2013) the lattice Boltzmann method's momentum flux gains
-Q + (3/4) tr(Q) I with Q_ab = kappa (G c^4/12) psi (delta_ab lap psi + 2 d_a d_b psi)
to second order, i.e. p'_ab gains (kappa G c^4/6) psi (delta_ab lap psi - d_a d_b psi):
the coefficient of psi d_a d_b psi in Eq. GeneralPressureTensor falls by 2 kappa and
that of psi lap psi delta_ab rises by 2 kappa, so the normal component of a planar
interface is unchanged and the surface tension of Eq. IntegralSurfaceTension
becomes (1 - kappa) times its value. Its divergence adds
(kappa G c^4/6) [(d_a psi)(d_g d_g psi) - (d_g psi)(d_a d_g psi)] to d_b p'_ab.

MacCormack predictor/corrector: first derivatives of rho, u, p_EOS and mu in the
advective, pressure and viscous terms are forward differences in the predictor
and backward differences in the corrector; second derivatives are central in
both; every derivative in d_b p'_ab is a second-order central difference.
Periodic in x; in y periodic, or walls as in the grid-dependency appendix
(Eqs. B1, B2): at the bottom a layer b1 on the wall with no slip, its density and
psi extrapolated linearly from the first two fluid rows (rho_b1 = 2 rho_0 - rho_1,
psi_b1 = 2 psi_0 - psi_1, U = V = 0), and a layer b2 inside the solid with
psi_b2 = psi_b1 + 2 dy (psi_l - psi_b1); at the top reflexive layers
(rho_t1 = rho_{N-1}, psi_t1 = psi_{N-1}, U_t1 = -U_{N-1}, V_t1 = -V_{N-1},
rho_t2 = rho_{N-2} and likewise psi_t2). p_EOS on b1 and t1 is that of their
density. Lengths are in lattice units; dx is the FD grid spacing, c = 1.
"""
from __future__ import annotations

import numpy as np


def _sh(a, dy, dx):
    """a(y + dy, x + dx) on a periodic grid (a has shape (ny, nx))."""
    return np.roll(a, shift=(-dy, -dx), axis=(0, 1))


class FDSolver:
    def __init__(self, eos, eps, tau_nu=1.0, tau_e=1.0, dx=1.0, walls=False, tau_l=None, visc_ratio=None,
                 kappa=0.0):
        """tau_l, visc_ratio: the relaxation time of Eq. RelaxationTime, linear in rho
        between tau_v = 1/2 + v_r (tau_l - 1/2) at rho_v and tau_l at rho_l, in place of
        the constant tau_nu (Eqs. DynamicViscosity, FDviscosityDerivative). kappa: the
        surface-tension control (module docstring)."""
        self.eos = eos
        self.eps = eps
        self.G = eos.G
        self.dx = dx
        self.tau_nu = tau_nu
        self.tau_e = tau_e
        self.walls = walls
        self.tau_l = tau_l
        self.visc_ratio = visc_ratio
        self.kappa = kappa

    def _tau_nu(self, rho):
        """(tau_nu(rho), d tau_nu / d rho)."""
        if self.tau_l is None:
            return self.tau_nu, 0.0
        e = self.eos
        tau_v = 0.5 + self.visc_ratio * (self.tau_l - 0.5)
        tau = self.tau_l * (rho - e.rho_v) / (e.rho_l - e.rho_v) + tau_v * (rho - e.rho_l) / (e.rho_v - e.rho_l)
        return tau, (self.tau_l - tau_v) / (e.rho_l - e.rho_v)

    def _padded(self, rho, u):
        """rho, u, psi, p with two ghost rows below and above (Eqs. B1, B2 and the
        reflexive top layers); rows 2 .. ny+1 are the fluid rows."""
        psi = self.eos.psi(rho)
        pad = lambda a: np.concatenate([np.zeros((2,) + a.shape[1:]), a, np.zeros((2,) + a.shape[1:])])  # noqa: E731
        R, X, Y, S = pad(rho), pad(u[0]), pad(u[1]), pad(psi)
        psi_l = float(self.eos.psi(self.eos.rho_l))
        # bottom: b1 (row 1) on the wall, b2 (row 0) inside the solid
        R[1] = 2.0 * rho[0] - rho[1]
        S[1] = 2.0 * psi[0] - psi[1]
        X[1] = 0.0
        Y[1] = 0.0
        S[0] = S[1] + 2.0 * self.dx * (psi_l - S[1])
        R[0] = R[1]        # not used by any stencil
        # top: reflexive layers t1 (row ny+2) and t2 (row ny+3)
        R[-2], S[-2], X[-2], Y[-2] = rho[-1], psi[-1], -u[0][-1], -u[1][-1]
        R[-1], S[-1] = rho[-2], psi[-2]
        P = self.eos.pressure(R)
        return R, [X, Y], S, P

    # difference operators (axis 0 = y, axis 1 = x)
    def d1(self, a, axis, kind):
        h = self.dx
        dy, dx = (1, 0) if axis == 0 else (0, 1)
        if kind == "f":
            return (_sh(a, dy, dx) - a) / h
        if kind == "b":
            return (a - _sh(a, -dy, -dx)) / h
        return (_sh(a, dy, dx) - _sh(a, -dy, -dx)) / (2 * h)

    def d2(self, a, ax1, ax2):
        h = self.dx
        if ax1 == ax2:
            dy, dx = (1, 0) if ax1 == 0 else (0, 1)
            return (_sh(a, dy, dx) - 2 * a + _sh(a, -dy, -dx)) / h**2
        return (_sh(a, 1, 1) - _sh(a, 1, -1) - _sh(a, -1, 1) + _sh(a, -1, -1)) / (4 * h**2)

    def rhs(self, rho, u, kind):
        """Time derivatives (d_t rho, d_t u_x, d_t u_y); kind 'f' (predictor) or 'b' (corrector)."""
        if self.walls:
            # derivatives on the padded arrays (np.roll's wrap in y only touches the
            # ghost rows, whose results are dropped); the fluid rows are kept
            R, U, S, P = self._padded(rho, u)
            dr, du = self._rhs(R, U, kind, S, P)
            return dr[2:-2], [d[2:-2] for d in du]
        return self._rhs(rho, u, kind, self.eos.psi(rho), self.eos.pressure(rho))

    def _rhs(self, rho, u, kind, psi, p):
        G, eps = self.G, self.eps
        cs2 = 1.0 / 3.0
        axes = (1, 0)  # alpha = x -> axis 1, alpha = y -> axis 0
        # mass
        div = sum(self.d1(u[a], axes[a], kind) for a in range(2))
        drho = -(rho * div + sum(u[a] * self.d1(rho, axes[a], kind) for a in range(2)))
        # psi derivatives (central)
        dpsi = [self.d1(psi, axes[a], "c") for a in range(2)]
        ddpsi = [[self.d2(psi, axes[a], axes[b]) for b in range(2)] for a in range(2)]
        lap = ddpsi[0][0] + ddpsi[1][1]
        dlap = [self.d1(lap, axes[a], "c") for a in range(2)]
        # dynamic viscosities (Eq. DynamicViscosity) and their density derivatives
        # (Eq. FDviscosityDerivative), with tau_nu constant or tau_nu(rho)
        tau, dtau = self._tau_nu(rho)
        mu = rho * cs2 * (tau - 0.5)
        muB = rho * cs2 * (self.tau_e - tau)
        dmu_drho = cs2 * (tau - 0.5) + rho * cs2 * dtau
        dmuB_drho = cs2 * (self.tau_e - tau) - rho * cs2 * dtau
        drho_1 = [self.d1(rho, axes[a], kind) for a in range(2)]
        du = [[self.d1(u[b], axes[a], kind) for b in range(2)] for a in range(2)]  # du[a][b] = d_a u_b
        ddu = [[[self.d2(u[c], axes[a], axes[b]) for c in range(2)] for b in range(2)] for a in range(2)]
        dpdx = [self.d1(p, axes[a], kind) for a in range(2)]
        dgu = du[0][0] + du[1][1]
        out = []
        for a in range(2):
            adv = sum(u[g] * du[g][a] for g in range(2))
            s = sum(dpsi[g] * ddpsi[a][g] for g in range(2))
            dpprime = (-eps * G / 4.0 * s + G / 12.0 * dpsi[a] * lap + G / 6.0 * s + G / 4.0 * psi * dlap[a])
            if self.kappa != 0.0:
                dpprime = dpprime + self.kappa * G / 6.0 * (dpsi[a] * lap - s)
            visc = (sum(dmu_drho * drho_1[b] * (du[a][b] + du[b][a]) for b in range(2))
                    + mu * sum(ddu[a][b][b] + ddu[b][b][a] for b in range(2))
                    + dmuB_drho * drho_1[a] * dgu
                    + muB * sum(ddu[a][b][b] for b in range(2)))
            out.append(-adv - dpdx[a] / rho - dpprime / rho + visc / rho)
        return drho, out

    def step(self, rho, u, dt):
        """One MacCormack step; u = [u_x, u_y]."""
        r1, du1 = self.rhs(rho, u, "f")
        rho_p = rho + dt * r1
        u_p = [u[a] + dt * du1[a] for a in range(2)]
        r2, du2 = self.rhs(rho_p, u_p, "b")
        rho_n = 0.5 * (rho + rho_p + dt * r2)
        u_n = [0.5 * (u[a] + u_p[a] + dt * du2[a]) for a in range(2)]
        return rho_n, u_n

    def run(self, rho, u, t_end, dt):
        n = int(round(t_end / dt))
        for _ in range(n):
            rho, u = self.step(rho, u, dt)
        return rho, u
