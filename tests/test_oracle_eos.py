"""Pins for the oracle's equation-of-state set-up (CPU only).

Every check here compares the oracle against something other than itself: a
number printed in the paper, a closed form (the Carnahan-Starling chemical
potential), an independent quadrature, or a special case that reduces to a
known identity.
"""
import json
import math
import os

import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

from oracle import eos as E

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def gauss_legendre(fn, lo, hi, n=400, pieces=64, log=False):
    """Independent composite Gauss-Legendre quadrature (optionally in ln x)."""
    x, w = leggauss(n)
    total = 0.0
    if log:
        edges = np.linspace(math.log(lo), math.log(hi), pieces + 1)
    else:
        edges = np.linspace(lo, hi, pieces + 1)
    for a, b in zip(edges[:-1], edges[1:]):
        s = 0.5 * (b - a) * x + 0.5 * (b + a)
        if log:
            r = np.exp(s)
            total += 0.5 * (b - a) * np.sum(w * fn(r) * r)
        else:
            total += 0.5 * (b - a) * np.sum(w * fn(s))
    return total


# ---------------------------------------------------------------------------
def test_critical_point_matches_printed_constants():
    g = GOLD["critical_point"]
    for a in (0.5, 0.363, 2.0):
        rho_c, Tc, pc = E.critical_point(a, 4.0, 1.0)
        assert abs(4.0 * rho_c - g["b_rho_c"]) < 1e-4
        assert abs(a * rho_c**2 / pc - g["a_rho_c2_over_p_c"]) < 1e-3
        assert abs(Tc * rho_c / pc - g["R_Tc_rho_c_over_p_c"]) < 1e-3
        assert abs(Tc * 4.0 / a - g["Tc_Rb_over_a"]) < 5e-5


def test_critical_point_is_an_inflection_with_zero_slope():
    a, b, R = 0.5, 4.0, 1.0
    rho_c, Tc, _ = E.critical_point(a, b, R)
    h = 1e-5
    p = lambda r: E.cs_pressure(r, a, b, R, Tc)
    d1 = (p(rho_c + h) - p(rho_c - h)) / (2 * h)
    d2 = (p(rho_c + h) - 2 * p(rho_c) + p(rho_c - h)) / h**2
    assert abs(d1) < 1e-8 and abs(d2) < 1e-5
    # below T_c the isotherm has a loop, above it does not
    r = np.linspace(0.01, 0.9, 20001)
    assert np.any(np.diff(E.cs_pressure(r, a, b, R, 0.99 * Tc)) < 0)
    assert np.all(np.diff(E.cs_pressure(r, a, b, R, 1.01 * Tc)) > 0)


def test_cs_derivative_against_central_differences():
    a, b, R, T = 0.5, 4.0, 1.0, 0.03
    r = np.linspace(0.001, 0.6, 50)
    h = 1e-6
    fd = (E.cs_pressure(r + h, a, b, R, T) - E.cs_pressure(r - h, a, b, R, T)) / (2 * h)
    assert np.allclose(E.cs_dpdrho(r, a, b, R, T), fd, rtol=1e-7, atol=1e-10)


def cs_chemical_potential(rho, a, b, R, T):
    """mu = d(free energy density)/d rho for Carnahan-Starling:
    f = rho R T [ln rho - 1 + (4 eta - 3 eta^2)/(1 - eta)^2] - a rho^2, eta = b rho/4.
    (p = rho mu - f reproduces Eq. CS.)"""
    eta = b * rho / 4.0
    return R * T * (math.log(rho) + (4 * eta - 3 * eta**2) / (1 - eta) ** 2 + (4 * eta - 2 * eta**2) / (1 - eta) ** 3) - 2 * a * rho


@pytest.mark.parametrize("Tr", [0.95, 0.8, 0.6, 0.5, 0.35])
def test_maxwell_equals_equal_chemical_potential(Tr):
    a, b, R = 0.5, 4.0, 1.0
    _, Tc, _ = E.critical_point(a, b, R)
    T = Tr * Tc
    rv, rl, ps = E.maxwell(a, b, R, T)
    # equal pressure
    assert abs(E.cs_pressure(rv, a, b, R, T) - ps) <= 1e-12 * ps
    # at rho_l, p is a small difference of two O(a rho_l^2) terms: rounding is relative to those
    assert abs(E.cs_pressure(rl, a, b, R, T) - ps) <= 1e-12 * ps + 1e-14 * a * rl**2
    # equal chemical potential (closed form, independent of the quadrature)
    mv = cs_chemical_potential(rv, a, b, R, T)
    ml = cs_chemical_potential(rl, a, b, R, T)
    assert abs(mv - ml) <= 1e-11 * R * T


def test_maxwell_density_ratios_and_psat_match_paper():
    g = GOLD["maxwell"]
    _, Tc, _ = E.critical_point(0.5, 4.0, 1.0)
    for Tr_s, ratio in g["ratio"].items():
        rv, rl, _ = E.maxwell(0.5, 4.0, 1.0, float(Tr_s) * Tc)
        assert abs(rl / rv - ratio) / ratio < 0.005, (Tr_s, rl / rv)
    _, _, ps = E.maxwell(0.5, 4.0, 1.0, 0.5 * Tc)
    assert abs(ps - g["p_sat_Tr05_a05"]) / g["p_sat_Tr05_a05"] < 0.05


def test_coexistence_independent_of_a_at_fixed_Tr():
    # Sec. III.B: lowering a leaves the Maxwell densities at fixed T_r unchanged
    res = []
    for a in (0.5, 0.363, 0.141, 2.0):
        _, Tc, _ = E.critical_point(a, 4.0, 1.0)
        res.append(E.maxwell(a, 4.0, 1.0, 0.5 * Tc))
    for rv, rl, ps in res[1:]:
        assert abs(rv - res[0][0]) < 1e-12 * res[0][0]
        assert abs(rl - res[0][1]) < 1e-12 * res[0][1]


# ---------------------------------------------------------------------------
SMOOTH_CASES = [(0.6, 0.387, 2.0, 0.834), (0.5, 0.363, 2.0, 0.775), (0.5, 0.5, 0.5, 0.342),
                (0.8, 0.5, 0.5, 0.342), (0.35, 0.363, 2.0, 0.775), (0.95, 0.363, 2.0, 0.775)]


@pytest.fixture(scope="module", params=SMOOTH_CASES, ids=lambda c: "Tr%.2f_al%.3f_av%.1f_alpha%.3f" % c)
def smooth(request):
    Tr, al, av, alpha = request.param
    return E.make_eos(E.MODE_SMOOTH, Tr, al, av, alpha)


def test_smooth_keeps_coexistence_and_slopes(smooth):
    e = smooth
    assert abs(e.pressure(e.rho_v) - e.p_sat) <= 1e-13 * e.p_sat + 1e-18
    assert abs(e.pressure(e.rho_l) - e.p_sat) <= 1e-10 * e.p_sat + 1e-15
    # sound speed continuous at rho_v and rho_l: slopes equal the bulk branches
    h = 1e-7 * e.rho_v
    left = (e.pressure(e.rho_v) - e.pressure(e.rho_v - h)) / h
    right = (e.pressure(e.rho_v + h) - e.pressure(e.rho_v)) / h
    assert abs(left - right) < 1e-4 * abs(left)
    h = 1e-7
    left = (e.pressure(e.rho_l) - e.pressure(e.rho_l - h)) / h
    right = (e.pressure(e.rho_l + h) - e.pressure(e.rho_l)) / h
    assert abs(left - right) < 1e-4 * abs(left)


def test_smooth_junctions_are_C1(smooth):
    e = smooth
    for r0 in (e.rho_v, e.rho_max, e.rho_min, e.rho_l):
        h = 1e-8 * max(r0, 1e-3)
        pl, pc, pr = e.pressure(r0 - h), e.pressure(r0), e.pressure(r0 + h)
        scale = max(abs(e.p_max), abs(e.p_min), e.p_sat)
        assert abs(pr - pl) < 1e-6 * scale          # continuity
        dl = (pc - e.pressure(r0 - 2 * h)) / (2 * h)
        dr = (e.pressure(r0 + 2 * h) - pc) / (2 * h)
        # a real kink would be of the order of the loop's slope scale
        slope_scale = (e.p_max - e.p_min) / (e.rho_min - e.rho_max)
        assert abs(dl - dr) < 1e-5 * slope_scale + 1e-4 * max(abs(dl), abs(dr))
    # extrema of the loop keep the C-S densities: zero slope at rho_max and rho_min
    assert abs(e.dpdrho(e.rho_max)) < 1e-12 and abs(e.dpdrho(e.rho_min)) < 1e-12


def test_smooth_obeys_maxwell_rule_independent_quadrature(smooth):
    e = smooth
    f = lambda r: (e.p_sat - e.pressure(r)) / r**2
    total = sum(gauss_legendre(f, lo, hi, log=True) for lo, hi in
                ((e.rho_v, e.rho_max), (e.rho_max, e.rho_min), (e.rho_min, e.rho_l)))
    scale = gauss_legendre(lambda r: np.abs(e.p_sat - e.pressure(r)) / r**2, e.rho_v, e.rho_l, log=True)
    assert abs(total) < 1e-11 * scale


def test_smooth_pmin_from_alpha_and_real_a1(smooth):
    e = smooth
    assert e.p_min == pytest.approx(e.p_sat - e.alpha * (e.p_sat_cs - e.p_min_cs), rel=1e-14, abs=1e-20)
    # a_1 real: dp/drho(rho_v) > 2 (p_max - p_sat)/(rho_max - rho_v) (Sec. III.D)
    assert e.dpdrho_v > 2 * (e.p_max - e.p_sat) / (e.rho_max - e.rho_v)
    assert e.a1sq > 0 and e.a3sq > 0 and e.p_max > e.p_sat > e.p_min


def test_dpdrho_of_shaped_eos_matches_differences(smooth):
    e = smooth
    r = np.concatenate([np.linspace(e.rho_v * 1.001, e.rho_max * 0.999, 30),
                        np.linspace(e.rho_max * 1.001, e.rho_min * 0.999, 30),
                        np.linspace(e.rho_min * 1.001, e.rho_l * 0.999, 30)])
    h = 1e-7 * r
    fd = (e.pressure(r + h) - e.pressure(r - h)) / (2 * h)
    scale = max(abs(e.dpdrho(r)).max(), 1e-12)
    assert np.allclose(e.dpdrho(r), fd, rtol=1e-5, atol=1e-7 * scale)


def test_vapour_branch_variant_shifts_liquid_by_dP():
    e = E.make_eos(E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834)
    # Delta P = p_sat(a_v) - p_sat(a_l); p_sat scales linearly with a at fixed T_r
    assert e.dP == pytest.approx(e.p_sat_cs * (2.0 / 0.387 - 1.0), rel=1e-10)
    r = 1.05 * e.rho_l
    assert e.pressure(r) == pytest.approx(E.cs_pressure(r, 0.387, 4, 1, e.T_l) + e.dP, rel=1e-15)
    r = 0.5 * e.rho_v
    assert e.pressure(r) == pytest.approx(E.cs_pressure(r, 2.0, 4, 1, e.T_v), rel=1e-15)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mode,Tr,al,av,alpha", [(E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834),
                                                 (E.MODE_CS, 0.6, 0.387, 0.387, 0.0),
                                                 (E.MODE_SMOOTH, 0.35, 0.363, 2.0, 0.775),
                                                 (E.MODE_CS, 0.8, 0.5, 0.5, 0.0)])
def test_epsilon_zeroes_mechanical_stability_integral(mode, Tr, al, av, alpha):
    e = E.make_eos(mode, Tr, al, av, alpha)
    eps = e.solve_eps()
    # the ln rho / Simpson mesh has converged
    assert abs(E.make_eos(mode, Tr, al, av, alpha).solve_eps(n=40000) - eps) < 1e-10
    # independent check: Gauss-Legendre in ln rho over the three regions
    f = lambda r: (e.p_sat - e.pressure(r)) * e.dpsidrho(r) / e.psi(r) ** (1 + eps)
    edges = (e.rho_v, e.rho_max, e.rho_min, e.rho_l)
    total = sum(gauss_legendre(f, lo, hi, log=True) for lo, hi in zip(edges[:-1], edges[1:]))
    scale = sum(gauss_legendre(lambda r: np.abs(f(r)), lo, hi, log=True) for lo, hi in zip(edges[:-1], edges[1:]))
    assert abs(total) < 1e-10 * scale
    # sigma = -eps/(16 G) (Sec. II.C); Newton started at 2 lands nearby (Fig. e_CS range)
    assert e.sigma() == pytest.approx(eps / 16.0, rel=1e-15)
    assert 1.0 < eps < 2.5


def test_epsilon_integral_reduces_to_maxwell_for_exponential_psi():
    """Sec. III.A: with psi = psi0 exp(-rho0/rho) and eps = 0 the mechanical
    stability condition is the Maxwell rule (psi'/psi = rho0/rho^2)."""
    e = E.make_eos(E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834)
    rho0, psi0 = 0.7, 1.3

    class ExpPsi(E.EOS):
        def psi(self, rho):
            return psi0 * np.exp(-rho0 / np.asarray(rho))

        def dpsidrho(self, rho):
            rho = np.asarray(rho)
            return psi0 * np.exp(-rho0 / rho) * rho0 / rho**2

    x = ExpPsi.__new__(ExpPsi)
    x.__dict__.update(e.__dict__)
    lhs = x.mech_stability_integral(0.0)
    f = lambda r: (e.p_sat - e.pressure(r)) / r**2
    rhs = rho0 * sum(gauss_legendre(f, lo, hi, log=True) for lo, hi in
                     ((e.rho_v, e.rho_max), (e.rho_max, e.rho_min), (e.rho_min, e.rho_l)))
    scale = rho0 * gauss_legendre(lambda r: np.abs(f(r)), e.rho_v, e.rho_l, log=True)
    assert abs(lhs - rhs) < 1e-10 * scale
    # and since the shaped EOS obeys Maxwell, both vanish
    assert abs(lhs) < 1e-10 * scale


def test_psi_definition_and_positivity():
    e = E.make_eos(E.MODE_SMOOTH, 0.35, 0.363, 2.0, 0.775)
    r = np.geomspace(e.rho_v * 0.1, e.rho_l * 1.2, 2000)
    arg = 2.0 * (r / 3.0 - e.pressure(r))
    assert np.all(arg > 0)
    assert np.allclose(e.psi(r) ** 2, arg, rtol=1e-14, atol=0)
