"""Oracle: equations of state and their set-up, written from the paper.

TEST INFRASTRUCTURE ONLY. This module is the plain, slow CPU reference that the
CUDA path is checked against. Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It shares no code with the CUDA library and never imports it.

Contents (each function cites the passage it follows):

* Carnahan-Starling pressure and its density derivative (Sec. III, Eq. CS).
* Critical point of Eq. CS (Sec. III.B, where T_c ~ 0.3773 a/(R b) is quoted).
* Maxwell equal-area coexistence (Sec. II.B, Eq. MaxwellRule), solved from its
  definition: pressure-equality roots plus an adaptive quadrature of the area.
* The "Smooth C-S" equation of state (Sec. III.D): elliptic region 1, cubic
  region 2, elliptic region 3; p_min from alpha; p_max solved so that the
  shaped EOS obeys the Maxwell rule. Includes the higher-vapour-sound-speed
  variant (vapour branch from C-S with a_v, liquid branch C-S(a_l) + Delta P).
* The pseudopotential psi(rho) (Sec. II.B, Eq. InteractionPotential).
* The mechanical-stability epsilon (Sec. II.C, Eq. VaporLiqEq) by Newton's
  method from epsilon = 2 with Simpson's rule, and sigma = -epsilon/(16 G)
  (Sec. II.C, below Eq. NewPressureTensor; Sec. III.A).

Readings of passages that are silent or garbled:

* T_c is the exact critical point of Eq. CS, not the rounded 0.3773 a/(R b).
* Region 2's cubic is evaluated in the normalised variable
  t = (rho - rho_max)/(rho_min - rho_max); with the printed coefficients this is
  the only form that reaches p_min at rho_min with zero slope at both ends.
* Region 3's undefined p_2, rho_2 are p_min and rho_min.
* With the vapour branch from a_v: Delta P = p_sat(a_v) - p_sat(a_l), the shaped
  EOS's saturation pressure is p_sat(a_v), slopes at rho_v / rho_l are those of
  the vapour / liquid branch, and p_min = p_sat - alpha (p_sat^CS - p_min^CS)
  with the C-S quantities of the liquid branch (a_l).
* Simpson's rule is applied per region (splitting at rho_max, rho_min) in the
  variable s = ln(rho), because the integrand varies on the scale of rho_v near
  the vapour density.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy import integrate, optimize

# Coexistence EOS modes.
MODE_CS = 0           # plain Carnahan-Starling (the "standard procedure", Sec. III.B)
MODE_SMOOTH = 1       # Smooth C-S (Sec. III.D)
MODE_PENG = 2         # Peng et al. cubic loop (Sec. II.D, Eqs. PengEOS, PengTheta), Guo forcing
MODE_SMOOTH_MOD = 3   # "Modified Smooth" (Sec. IV.C): p_max from Eq. VaporLiqEq with eps = 0


# ---------------------------------------------------------------------------
# Carnahan-Starling, Eq. CS (Sec. III)
# ---------------------------------------------------------------------------
def cs_pressure(rho, a, b, R, T):
    """p = rho R T (1 + eta + eta^2 - eta^3)/(1 - eta)^3 - a rho^2, eta = b rho/4."""
    eta = b * rho / 4.0
    return rho * R * T * (1.0 + eta + eta**2 - eta**3) / (1.0 - eta) ** 3 - a * rho**2


def _cs_Z(eta):
    return (1.0 + eta + eta**2 - eta**3) / (1.0 - eta) ** 3


def _cs_dZ(eta):
    # dZ/deta of Z = 1 + (4 eta - 2 eta^2)/(1 - eta)^3
    return (4.0 + 4.0 * eta - 2.0 * eta**2) / (1.0 - eta) ** 4


def _cs_d2Z(eta):
    return (20.0 + 8.0 * eta - 4.0 * eta**2) / (1.0 - eta) ** 5


def cs_dpdrho(rho, a, b, R, T):
    """d p / d rho of Eq. CS: R T (Z + eta Z'(eta)) - 2 a rho."""
    eta = b * rho / 4.0
    return R * T * (_cs_Z(eta) + eta * _cs_dZ(eta)) - 2.0 * a * rho


def cs_d2pdrho2(rho, a, b, R, T):
    eta = b * rho / 4.0
    return R * T * (b / 4.0) * (2.0 * _cs_dZ(eta) + eta * _cs_d2Z(eta)) - 2.0 * a


def critical_point(a, b, R):
    """(rho_c, T_c, p_c): the point where dp/drho = d2p/drho2 = 0 (Sec. III, Eq. CS).

    For each eta the second condition fixes T; the first is then solved for eta.
    """
    def T_of_eta(eta):
        return 2.0 * a / (R * (b / 4.0) * (2.0 * _cs_dZ(eta) + eta * _cs_d2Z(eta)))

    def g(eta):
        rho = 4.0 * eta / b
        return cs_dpdrho(rho, a, b, R, T_of_eta(eta))

    eta_c = optimize.brentq(g, 0.05, 0.3, xtol=1e-300, rtol=4 * np.finfo(float).eps, maxiter=500)
    rho_c = 4.0 * eta_c / b
    T_c = T_of_eta(eta_c)
    return rho_c, T_c, cs_pressure(rho_c, a, b, R, T_c)


def cs_extrema(a, b, R, T):
    """(rho_max, rho_min): the local maximum and minimum of Eq. CS below T_c (Sec. III.D)."""
    rho_c, _, _ = critical_point(a, b, R)
    hi = 4.0 / b * (1.0 - 1e-9)
    kw = dict(xtol=1e-300, rtol=4 * np.finfo(float).eps, maxiter=500)
    rho_max = optimize.brentq(lambda r: cs_dpdrho(r, a, b, R, T), 1e-14, rho_c, **kw)
    rho_min = optimize.brentq(lambda r: cs_dpdrho(r, a, b, R, T), rho_c, hi, **kw)
    return rho_max, rho_min


def maxwell(a, b, R, T):
    """Maxwell equal-area coexistence of Eq. CS (Sec. II.B, Eq. MaxwellRule).

    For a trial pressure p0 the vapour and liquid densities are the outer roots
    of p(rho) = p0; the residual is int_{rho_v}^{rho_l} (p0 - p)/rho^2 d rho.
    Returns (rho_v, rho_l, p_sat).
    """
    rho_max, rho_min = cs_extrema(a, b, R, T)
    p_hi = cs_pressure(rho_max, a, b, R, T)
    p_lo = max(cs_pressure(rho_min, a, b, R, T), 0.0)
    kw = dict(xtol=1e-300, rtol=4 * np.finfo(float).eps, maxiter=500)
    top = 4.0 / b * (1.0 - 1e-12)

    def roots(p0):
        rv = optimize.brentq(lambda r: cs_pressure(r, a, b, R, T) - p0, 1e-300, rho_max, **kw)
        rl = optimize.brentq(lambda r: cs_pressure(r, a, b, R, T) - p0, rho_min, top, **kw)
        return rv, rl

    def residual(p0):
        rv, rl = roots(p0)
        f = lambda r: (p0 - cs_pressure(r, a, b, R, T)) / r**2
        total = 0.0
        for lo, hi in ((rv, rho_max), (rho_max, rho_min), (rho_min, rl)):
            val, _ = integrate.quad(f, lo, hi, epsabs=0.0, epsrel=1.2e-14, limit=500)
            total += val
        return total

    # residual -> -inf as p0 -> 0+ (rho_v -> 0) and > 0 at p0 = p(rho_max)
    lo = p_lo if p_lo > 0 else p_hi * 1e-30
    while residual(lo) > 0:
        lo *= 1e-3
    p_sat = optimize.brentq(residual, lo, p_hi * (1 - 1e-12), **kw)
    rv, rl = roots(p_sat)
    return rv, rl, p_sat


# ---------------------------------------------------------------------------
# Shaped EOS (Sec. III.D) and plain C-S as one piecewise object
# ---------------------------------------------------------------------------
def _radicand(d, asq):
    """1 - d^2 / a^2 of the ellipse constants (Sec. III.D). With r = h / (p' d) the
    ratio of the ellipse's rise h to the tangent's, a^2 = d^2 (1 - r)^2 / (1 - 2 r), so
    the radicand is r^2 / (1 - r)^2 >= 0; near r = 0 (the lower end of the p_max
    bracket) the subtraction can round to -1 ulp, which is clamped to 0."""
    return max(0.0, 1.0 - d**2 / asq)


@dataclass
class EOS:
    """A coexistence EOS at one reduced temperature.

    mode == MODE_CS: p = C-S(a_l) everywhere (a_v ignored).
    mode == MODE_SMOOTH: rho <= rho_v: C-S(a_v); (rho_v, rho_max]: ellipse 1;
    (rho_max, rho_min): cubic; [rho_min, rho_l): ellipse 2 (the paper's region 3);
    rho >= rho_l: C-S(a_l) + dP.
    """

    mode: int
    Tr: float
    a_l: float
    a_v: float
    alpha: float
    b: float = 4.0
    R: float = 1.0
    G: float = -1.0
    r_theta: float = 0.0   # MODE_PENG: theta from Eq. PengTheta

    def __post_init__(self):
        b, R = self.b, self.R
        _, self.Tc_l, _ = critical_point(self.a_l, b, R)
        _, self.Tc_v, _ = critical_point(self.a_v, b, R)
        self.T_l = self.Tr * self.Tc_l
        self.T_v = self.Tr * self.Tc_v
        self.rho_v, self.rho_l, self.p_sat_cs = maxwell(self.a_l, b, R, self.T_l)
        self.rho_max, self.rho_min = cs_extrema(self.a_l, b, R, self.T_l)
        self.p_min_cs = cs_pressure(self.rho_min, self.a_l, b, R, self.T_l)
        if self.mode == MODE_CS:
            self.p_sat = self.p_sat_cs
            self.dP = 0.0
        elif self.mode == MODE_PENG:
            self.p_sat = self.p_sat_cs
            self.dP = 0.0
            self.dpdrho_v = cs_dpdrho(self.rho_v, self.a_l, b, R, self.T_l)
            self.dpdrho_l = cs_dpdrho(self.rho_l, self.a_l, b, R, self.T_l)
            self.rho_m = self._solve_rho_m()
            self._peng_theta(self.rho_m)
        elif self.mode in (MODE_SMOOTH, MODE_SMOOTH_MOD):
            # saturation pressure of the vapour-branch EOS at the same reduced temperature
            _, _, p_sat_v = maxwell(self.a_v, b, R, self.T_v)
            self.p_sat = p_sat_v
            self.dP = p_sat_v - self.p_sat_cs
            self.dpdrho_v = cs_dpdrho(self.rho_v, self.a_v, b, R, self.T_v)
            self.dpdrho_l = cs_dpdrho(self.rho_l, self.a_l, b, R, self.T_l)
            self.p_min = self.p_sat - self.alpha * (self.p_sat_cs - self.p_min_cs)
            self._region3()
            self.p_max = self._solve_p_max()
            self._region1(self.p_max)
            if self.mode == MODE_SMOOTH_MOD:
                self.eps = 0.0
        else:
            raise ValueError("unknown EOS mode")
        self.eps = None

    # -- region constants, Sec. III.D ------------------------------------------
    def _region3(self):
        d = self.rho_l - self.rho_min
        k = (self.p_sat - self.p_min) * d / self.dpdrho_l - d**2
        self.a3sq = -(k**2) / (2.0 * k + d**2)
        self.b3 = (self.p_sat - self.p_min) / (1.0 - math.sqrt(_radicand(d, self.a3sq)))

    def _region1(self, p_max):
        d = self.rho_max - self.rho_v
        k = (p_max - self.p_sat) * d / self.dpdrho_v - d**2
        self.p_max = p_max
        self.a1sq = -(k**2) / (2.0 * k + d**2)
        self.b1 = (p_max - self.p_sat) / (1.0 - math.sqrt(_radicand(d, self.a1sq)))

    def _solve_p_max(self):
        """p_max such that the shaped EOS satisfies Eq. MaxwellRule at rho_v, rho_l."""
        d = self.rho_max - self.rho_v
        # a_1 is real only for p_max - p_sat < dp/drho(rho_v) d / 2 (condition below region 1)
        hi = self.p_sat + 0.5 * self.dpdrho_v * d * (1.0 - 1e-12)
        lo = self.p_sat * (1.0 + 1e-15) if self.p_sat > 0 else self.p_sat + 1e-300
        lo = max(lo, self.p_sat + 1e-16 * (hi - self.p_sat))
        kw = dict(xtol=1e-300, rtol=4 * np.finfo(float).eps, maxiter=500)

        def residual(pm):
            self._region1(pm)
            if self.mode == MODE_SMOOTH_MOD:
                return self.mech_stability_quad(0.0)
            return self.maxwell_residual()

        return optimize.brentq(residual, lo, hi, **kw)

    def mech_stability_quad(self, eps):
        """Eq. VaporLiqEq by adaptive quadrature over the three regions (set-up root finding)."""
        f = lambda r: (self.p_sat - float(self.pressure(r))) * float(self.dpsidrho(r)) / float(self.psi(r)) ** (1.0 + eps)
        total = 0.0
        for lo, hi in self._regions():
            val, _ = integrate.quad(f, lo, hi, epsabs=0.0, epsrel=1e-13, limit=500)
            total += val
        return total

    def _regions(self):
        if self.mode == MODE_PENG:
            return ((self.rho_v, self.rho_l),)
        return ((self.rho_v, self.rho_max), (self.rho_max, self.rho_min), (self.rho_min, self.rho_l))

    # -- Peng et al. loop, Eqs. PengEOS and PengTheta ---------------------------------
    def _peng_theta(self, rho_m):
        rv, rl = self.rho_v, self.rho_l
        self.theta = ((1.0 - self.r_theta) / ((rv - rho_m) * (rv - rl)) * self.dpdrho_v
                      + self.r_theta / ((rl - rho_m) * (rl - rv)) * self.dpdrho_l)

    def _solve_rho_m(self):
        """rho_m such that Eq. ShanVaporLiqEq (eps = 0) holds at the Maxwell densities."""
        kw = dict(xtol=1e-300, rtol=4 * np.finfo(float).eps, maxiter=500)

        def residual(rm):
            self.rho_m = rm
            self._peng_theta(rm)
            return self.mech_stability_quad(0.0)

        d = self.rho_l - self.rho_v
        grid = np.linspace(self.rho_v + 1e-3 * d, self.rho_l - 1e-3 * d, 60)
        vals = []
        for rm in grid:
            try:
                vals.append(residual(rm))
            except (ValueError, ZeroDivisionError, FloatingPointError):
                vals.append(np.nan)
        for (a, fa), (b_, fb) in zip(zip(grid[:-1], vals[:-1]), zip(grid[1:], vals[1:])):
            if np.isfinite(fa) and np.isfinite(fb) and fa * fb < 0:
                return optimize.brentq(residual, a, b_, **kw)
        raise RuntimeError("no rho_m solves the mechanical stability condition")

    def maxwell_residual(self):
        f = lambda r: (self.p_sat - self.pressure(r)) / r**2
        total = 0.0
        for lo, hi in ((self.rho_v, self.rho_max), (self.rho_max, self.rho_min), (self.rho_min, self.rho_l)):
            val, _ = integrate.quad(f, lo, hi, epsabs=0.0, epsrel=1.2e-14, limit=500)
            total += val
        return total

    # -- evaluation ---------------------------------------------------------------
    def pressure(self, rho):
        """p(rho) of the EOS in use (scalar or ndarray)."""
        rho = np.asarray(rho, dtype=np.float64)
        b, R = self.b, self.R
        if self.mode == MODE_CS:
            return cs_pressure(rho, self.a_l, b, R, self.T_l)
        if self.mode == MODE_PENG:
            p = cs_pressure(rho, self.a_l, b, R, self.T_l)
            m = (rho > self.rho_v) & (rho < self.rho_l)
            x = rho[m] if p.ndim else rho
            loop = self.p_sat + self.theta * (x - self.rho_v) * (x - self.rho_l) * (x - self.rho_m)
            if p.ndim:
                p[m] = loop
                return p
            return float(loop) if m else float(p)
        p = np.empty_like(rho)
        r1 = rho <= self.rho_v
        r2 = (rho > self.rho_v) & (rho <= self.rho_max)
        r3 = (rho > self.rho_max) & (rho < self.rho_min)
        r4 = (rho >= self.rho_min) & (rho < self.rho_l)
        r5 = rho >= self.rho_l
        p[r1] = cs_pressure(rho[r1], self.a_v, b, R, self.T_v)
        x = rho[r2]
        p[r2] = self.p_max - self.b1 + self.b1 * np.sqrt(1.0 - (x - self.rho_max) ** 2 / self.a1sq)
        t = (rho[r3] - self.rho_max) / (self.rho_min - self.rho_max)
        a2 = 2.0 * (self.p_max - self.p_min)
        b2 = 3.0 * (self.p_min - self.p_max)
        p[r3] = a2 * t**3 + b2 * t**2 + self.p_max
        x = rho[r4]
        p[r4] = self.p_min + self.b3 - self.b3 * np.sqrt(1.0 - (x - self.rho_min) ** 2 / self.a3sq)
        p[r5] = cs_pressure(rho[r5], self.a_l, b, R, self.T_l) + self.dP
        return p if p.ndim else float(p)

    def dpdrho(self, rho):
        rho = np.asarray(rho, dtype=np.float64)
        b, R = self.b, self.R
        if self.mode == MODE_CS:
            return cs_dpdrho(rho, self.a_l, b, R, self.T_l)
        if self.mode == MODE_PENG:
            d = cs_dpdrho(rho, self.a_l, b, R, self.T_l)
            m = (rho > self.rho_v) & (rho < self.rho_l)
            x = rho[m] if d.ndim else rho
            rv, rl, rm = self.rho_v, self.rho_l, self.rho_m
            loop = self.theta * ((x - rl) * (x - rm) + (x - rv) * (x - rm) + (x - rv) * (x - rl))
            if d.ndim:
                d[m] = loop
                return d
            return float(loop) if m else float(d)
        d = np.empty_like(rho)
        r1 = rho <= self.rho_v
        r2 = (rho > self.rho_v) & (rho <= self.rho_max)
        r3 = (rho > self.rho_max) & (rho < self.rho_min)
        r4 = (rho >= self.rho_min) & (rho < self.rho_l)
        r5 = rho >= self.rho_l
        d[r1] = cs_dpdrho(rho[r1], self.a_v, b, R, self.T_v)
        x = rho[r2] - self.rho_max
        d[r2] = -self.b1 * x / (self.a1sq * np.sqrt(1.0 - x**2 / self.a1sq))
        span = self.rho_min - self.rho_max
        t = (rho[r3] - self.rho_max) / span
        d[r3] = (6.0 * (self.p_max - self.p_min) * t**2 + 6.0 * (self.p_min - self.p_max) * t) / span
        x = rho[r4] - self.rho_min
        d[r4] = self.b3 * x / (self.a3sq * np.sqrt(1.0 - x**2 / self.a3sq))
        d[r5] = cs_dpdrho(rho[r5], self.a_l, b, R, self.T_l)
        return d if d.ndim else float(d)

    def psi(self, rho):
        """Eq. InteractionPotential with c = 1: psi = sqrt(2 (p - rho c_s^2) / G)."""
        rho = np.asarray(rho, dtype=np.float64)
        return np.sqrt(2.0 * (self.pressure(rho) - rho / 3.0) / self.G)

    def dpsidrho(self, rho):
        rho = np.asarray(rho, dtype=np.float64)
        return (self.dpdrho(rho) - 1.0 / 3.0) / (self.G * self.psi(rho))

    # -- mechanical stability, Eq. VaporLiqEq --------------------------------------
    def _simpson_nodes(self, n):
        """Composite-Simpson nodes and weights over [rho_v, rho_l] in s = ln rho, per region."""
        edges = [self.rho_v, self.rho_l] if self.mode == MODE_PENG else [self.rho_v, self.rho_max, self.rho_min, self.rho_l]
        rs, ws = [], []
        for lo, hi in zip(edges[:-1], edges[1:]):
            s = np.linspace(math.log(lo), math.log(hi), 2 * n + 1)
            h = s[1] - s[0]
            w = np.ones_like(s)
            w[1:-1:2] = 4.0
            w[2:-1:2] = 2.0
            rho = np.exp(s)
            rs.append(rho)
            ws.append(w * h / 3.0 * rho)   # d rho = rho ds
        return np.concatenate(rs), np.concatenate(ws)

    def mech_stability_integral(self, eps, n=20000):
        """int_{rho_v}^{rho_l} (p0 - p) psi'/psi^(1+eps) d rho with p0 = p_sat (Eq. VaporLiqEq)."""
        rho, w = self._simpson_nodes(n)
        psi = self.psi(rho)
        integrand = (self.p_sat - self.pressure(rho)) * self.dpsidrho(rho) / psi ** (1.0 + eps)
        return float(np.sum(w * integrand))

    def solve_eps(self, n=20000, tol=1e-15, maxit=100):
        """Newton's method from eps = 2 (Sec. III.A) with Simpson's rule."""
        rho, w = self._simpson_nodes(n)
        psi = self.psi(rho)
        base = (self.p_sat - self.pressure(rho)) * self.dpsidrho(rho)
        lnpsi = np.log(psi)
        eps = 2.0
        for _ in range(maxit):
            wk = base / psi ** (1.0 + eps)
            g = float(np.sum(w * wk))
            dg = float(np.sum(w * (-lnpsi) * wk))
            step = g / dg
            eps -= step
            if abs(step) <= tol * max(1.0, abs(eps)):
                break
        else:
            raise RuntimeError("Newton for epsilon did not converge")
        self.eps = eps
        return eps

    def sigma(self):
        """sigma of the Li forcing scheme from eps = -16 G sigma (Sec. II.C); the Peng and
        Modified Smooth EOS are used with the Guo scheme (sigma = 0, Sec. II.D, IV.C)."""
        if self.mode in (MODE_PENG, MODE_SMOOTH_MOD):
            return 0.0
        if self.eps is None:
            self.solve_eps()
        return -self.eps / (16.0 * self.G)


def make_eos(mode, Tr, a_l, a_v=None, alpha=0.0, b=4.0, R=1.0, G=-1.0, r_theta=0.0):
    """Convenience constructor; a_v defaults to a_l."""
    return EOS(mode=mode, Tr=Tr, a_l=a_l, a_v=a_l if a_v is None else a_v, alpha=alpha, b=b, R=R, G=G,
               r_theta=r_theta)
