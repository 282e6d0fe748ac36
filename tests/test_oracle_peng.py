"""Pins for the oracle's Peng loop (Sec. II.D, Eqs. PengEOS, PengTheta) and the
Modified Smooth EOS (Sec. IV.C), in process (CPU only): the definitions' own
conditions, checked with an independent quadrature and finite differences.

* Peng: p = p_sat + theta (rho - rho_v)(rho - rho_l)(rho - rho_m) inside
  (rho_v, rho_l), C-S outside, so p is continuous at the Maxwell densities and
  crosses p_sat at rho_m; theta weights the two bulk slopes (Eq. PengTheta), so
  r_theta = 0 gives the loop the vapour branch's slope at rho_v and r_theta = 1 the
  liquid branch's at rho_l; rho_m makes Eq. ShanVaporLiqEq (eps = 0) hold.
* Modified Smooth: the Smooth C-S regions with p_max set by Eq. VaporLiqEq at
  eps = 0 instead of the Maxwell rule: that integral vanishes, the coexistence
  densities and the loop's extrema stay.
"""
import numpy as np
import pytest

from oracle import eos as E

from test_oracle_eos import gauss_legendre

TR, A = 0.6, 0.387


def _peng(r_theta):
    return E.make_eos(E.MODE_PENG, TR, A, A, 0.0, r_theta=r_theta)


def _one_sided_slope(e, r0, h):
    """Second-order one-sided difference from r0 towards r0 + h (h may be negative)."""
    return (-3.0 * e.pressure(r0) + 4.0 * e.pressure(r0 + h) - e.pressure(r0 + 2.0 * h)) / (2.0 * h)


@pytest.mark.parametrize("r_theta", [0.0, 0.45, 1.0])
def test_peng_loop_is_continuous_and_crosses_p_sat_at_rho_m(r_theta):
    e = _peng(r_theta)
    assert e.rho_v < e.rho_m < e.rho_l
    for r0 in (e.rho_v, e.rho_l):
        h = 1e-9 * r0
        # no jump: the step across r0 is of the order of h times the slopes (a jump
        # from a wrong p_sat or rho_v, rho_l would be of the order of p_sat)
        slope = abs(E.cs_dpdrho(r0, A, 4.0, 1.0, e.T_l))
        assert abs(e.pressure(r0 + h) - e.pressure(r0 - h)) < 100.0 * h * slope
        assert e.pressure(r0) == pytest.approx(e.p_sat, rel=1e-10)
    assert e.pressure(e.rho_m) == pytest.approx(e.p_sat, rel=1e-12)
    # outside the loop the EOS is C-S
    for r in (0.5 * e.rho_v, 1.1 * e.rho_l):
        assert e.pressure(r) == pytest.approx(E.cs_pressure(r, A, 4.0, 1.0, e.T_l), rel=1e-15)


def test_peng_theta_gives_the_weighted_branch_its_slope():
    """Eq. PengTheta at its end points: r_theta = 0 matches the loop's slope at rho_v
    to the vapour branch's, r_theta = 1 at rho_l to the liquid branch's."""
    e0, e1 = _peng(0.0), _peng(1.0)
    h = 1e-6 * (e0.rho_l - e0.rho_v)
    s_v = _one_sided_slope(e0, e0.rho_v, h)               # inside the loop, above rho_v
    s_l = _one_sided_slope(e1, e1.rho_l, -h)              # inside the loop, below rho_l
    assert s_v == pytest.approx(E.cs_dpdrho(e0.rho_v, A, 4.0, 1.0, e0.T_l), rel=1e-6)
    assert s_l == pytest.approx(E.cs_dpdrho(e1.rho_l, A, 4.0, 1.0, e1.T_l), rel=1e-6)
    # and the other end is not matched (the pin discriminates)
    s_l0 = _one_sided_slope(e0, e0.rho_l, -h)
    assert abs(s_l0 / E.cs_dpdrho(e0.rho_l, A, 4.0, 1.0, e0.T_l) - 1.0) > 1e-2


def _eps0_integral(e, edges):
    f = lambda r: (e.p_sat - e.pressure(r)) * e.dpsidrho(r) / e.psi(r)
    total = sum(gauss_legendre(f, lo, hi, log=True) for lo, hi in zip(edges[:-1], edges[1:]))
    scale = sum(gauss_legendre(lambda r: np.abs(f(r)), lo, hi, log=True) for lo, hi in zip(edges[:-1], edges[1:]))
    return total, scale


@pytest.mark.parametrize("r_theta", [0.0, 0.45, 1.0])
def test_peng_rho_m_zeroes_the_eps0_mechanical_stability_condition(r_theta):
    e = _peng(r_theta)
    total, scale = _eps0_integral(e, (e.rho_v, e.rho_m, e.rho_l))
    assert abs(total) < 1e-10 * scale


def test_modified_smooth_zeroes_the_eps0_condition_and_keeps_the_loop():
    e = E.make_eos(E.MODE_SMOOTH_MOD, TR, A, 2.0, 0.446)
    total, scale = _eps0_integral(e, (e.rho_v, e.rho_max, e.rho_min, e.rho_l))
    assert abs(total) < 1e-10 * scale
    assert e.pressure(e.rho_v) == pytest.approx(e.p_sat, rel=1e-12)
    assert e.pressure(e.rho_l) == pytest.approx(e.p_sat, rel=1e-10)
    assert abs(e.dpdrho(e.rho_max)) < 1e-12 and abs(e.dpdrho(e.rho_min)) < 1e-12
    # p_max differs from the Maxwell-ruled Smooth C-S of the same alpha
    assert abs(e.p_max / E.make_eos(E.MODE_SMOOTH, TR, A, 2.0, 0.446).p_max - 1.0) > 1e-6
