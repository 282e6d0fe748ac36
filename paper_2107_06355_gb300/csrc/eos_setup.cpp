// Host set-up of the equation of state (Sec. III and Sec. III.D of the paper).
//
// Methods (chosen for accuracy at low reduced temperature, where rho_v ~ 1e-5):
//  * critical point of Eq. CS: eta_c is the root in (0, 1) of
//      1 - 5 eta - 20 eta^2 - 4 eta^3 + 5 eta^4 - eta^5 = 0,
//    which is (1 - eta)^5 (Z - eta Z' - eta^2 Z'') = 0 with Z the C-S
//    compressibility; this is dp/drho = d2p/drho2 = 0 with T eliminated;
//  * Maxwell rule (Eq. MaxwellRule) as equal pressure and equal chemical
//    potential, mu = R T [ln rho + (4 eta - 3 eta^2)/(1 - eta)^2
//    + (4 eta - 2 eta^2)/(1 - eta)^3] - 2 a rho (the C-S free energy), solved
//    by Ridders' method on the saturation pressure;
//  * integrals over [rho_v, rho_l] (the Maxwell residual of the shaped EOS and
//    Eq. VaporLiqEq) by composite Gauss-Legendre quadrature in s = ln(rho),
//    split at rho_max and rho_min where the shaped EOS is only C^1;
//  * p_max: Ridders' method on the Maxwell residual of the shaped EOS, bracketed
//    by p_sat and the real-a_1 limit of Sec. III.D;
//  * eps: Newton's method from eps = 2 (Sec. III.A).
#include <cmath>
#include <cstring>
#include <functional>

#include "../../include/pplbm.h"
#include "eos.cuh"
#include "internal.h"

namespace pplbm {
namespace {

// Gauss-Legendre nodes/weights on [-1, 1] by Newton's method on P_n (textbook construction).
struct GaussLegendre {
  static constexpr int n = 32;
  double x[n], w[n];
  GaussLegendre() {
    for (int i = 0; i < n; ++i) {
      double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
          const double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = pk;
        }
        const double dp = n * (z * p1 - p0) / (z * z - 1.0);
        const double dz = p1 / dp;
        z -= dz;
        if (std::fabs(dz) < 1e-16) {
          // weight with the converged node
          double q0 = 1.0, q1 = z;
          for (int k = 2; k <= n; ++k) {
            const double qk = ((2.0 * k - 1.0) * z * q1 - (k - 1.0) * q0) / k;
            q0 = q1;
            q1 = qk;
          }
          const double dq = n * (z * q1 - q0) / (z * z - 1.0);
          x[i] = z;
          w[i] = 2.0 / ((1.0 - z * z) * dq * dq);
          break;
        }
      }
    }
  }
};

const GaussLegendre& gl() {
  static const GaussLegendre g;
  return g;
}

// integral of fn(rho) d rho over [lo, hi], in s = ln rho with `panels` equal panels
double integrate_log(const std::function<double(double)>& fn, double lo, double hi, int panels) {
  const GaussLegendre& g = gl();
  const double s0 = std::log(lo), s1 = std::log(hi);
  const double h = (s1 - s0) / panels;
  double total = 0.0;
  for (int p = 0; p < panels; ++p) {
    const double a = s0 + p * h;
    double acc = 0.0;
    for (int k = 0; k < GaussLegendre::n; ++k) {
      const double s = a + 0.5 * h * (g.x[k] + 1.0);
      const double rho = std::exp(s);
      acc += g.w[k] * fn(rho) * rho;
    }
    total += 0.5 * h * acc;
  }
  return total;
}

// Ridders' method on [a, b] with fa, fb of opposite sign.
bool ridders(const std::function<double(double)>& fn, double a, double b, double& root, int maxit = 200) {
  double fa = fn(a), fb = fn(b);
  if (fa == 0.0) { root = a; return true; }
  if (fb == 0.0) { root = b; return true; }
  if ((fa > 0) == (fb > 0)) return false;
  double x = 0.5 * (a + b);
  for (int it = 0; it < maxit; ++it) {
    const double m = 0.5 * (a + b);
    const double fm = fn(m);
    const double s = std::sqrt(fm * fm - fa * fb);
    if (s == 0.0) { root = m; return true; }
    const double xn = m + (m - a) * ((fa >= fb ? 1.0 : -1.0) * fm / s);
    const double fx = fn(xn);
    x = xn;
    if (fx == 0.0) { root = x; return true; }
    if ((fm > 0) != (fx > 0)) { a = m; fa = fm; b = x; fb = fx; }
    else if ((fa > 0) != (fx > 0)) { b = x; fb = fx; }
    else { a = x; fa = fx; }
    if (std::fabs(b - a) <= 2e-16 * std::fabs(x)) { root = x; return true; }
  }
  root = x;
  return true;
}

double cs_Z(double eta) { return (1.0 + eta + eta * eta - eta * eta * eta) / std::pow(1.0 - eta, 3); }
double cs_dZ(double eta) { return (4.0 + 4.0 * eta - 2.0 * eta * eta) / std::pow(1.0 - eta, 4); }
double cs_d2Z(double eta) { return (20.0 + 8.0 * eta - 4.0 * eta * eta) / std::pow(1.0 - eta, 5); }

double cs_p(double rho, double a, double b, double R, double T) {
  const double eta = b * rho / 4.0;
  return rho * R * T * cs_Z(eta) - a * rho * rho;
}
double cs_dp(double rho, double a, double b, double R, double T) {
  const double eta = b * rho / 4.0;
  return R * T * (cs_Z(eta) + eta * cs_dZ(eta)) - 2.0 * a * rho;
}
double cs_mu(double rho, double a, double b, double R, double T) {
  const double eta = b * rho / 4.0;
  const double om = 1.0 - eta;
  return R * T * (std::log(rho) + (4.0 * eta - 3.0 * eta * eta) / (om * om) +
                  (4.0 * eta - 2.0 * eta * eta) / (om * om * om)) -
         2.0 * a * rho;
}

bool critical_temperature(double a, double b, double R, double& Tc, double& rho_c) {
  auto poly = [](double e) { return 1.0 + e * (-5.0 + e * (-20.0 + e * (-4.0 + e * (5.0 - e)))); };
  double eta;
  if (!ridders(poly, 0.01, 0.5, eta)) return false;
  // polish with Newton on the polynomial
  for (int it = 0; it < 5; ++it) {
    const double d = -5.0 + eta * (-40.0 + eta * (-12.0 + eta * (20.0 - 5.0 * eta)));
    eta -= poly(eta) / d;
  }
  Tc = 2.0 * a / (R * (b / 4.0) * (2.0 * cs_dZ(eta) + eta * cs_d2Z(eta)));
  rho_c = 4.0 * eta / b;
  return true;
}

struct Branch {
  double a, b, R, T;
  double p(double r) const { return cs_p(r, a, b, R, T); }
  double dp(double r) const { return cs_dp(r, a, b, R, T); }
  double mu(double r) const { return cs_mu(r, a, b, R, T); }
};

bool spinodals(const Branch& c, double rho_c, double& rho_max, double& rho_min) {
  auto d = [&](double r) { return c.dp(r); };
  if (!ridders(d, 1e-300, rho_c, rho_max)) return false;
  if (!ridders(d, rho_c, 4.0 / c.b * (1.0 - 1e-12), rho_min)) return false;
  return true;
}

// Maxwell coexistence: p(rho_v) = p(rho_l) = p_sat and mu(rho_v) = mu(rho_l).
bool maxwell(const Branch& c, double rho_max, double rho_min, double& rho_v, double& rho_l, double& p_sat) {
  const double top = 4.0 / c.b * (1.0 - 1e-13);
  auto roots = [&](double p0, double& rv, double& rl) {
    bool ok = ridders([&](double r) { return c.p(r) - p0; }, 1e-300, rho_max, rv);
    ok = ok && ridders([&](double r) { return c.p(r) - p0; }, rho_min, top, rl);
    return ok;
  };
  auto h = [&](double p0) {
    double rv, rl;
    if (!roots(p0, rv, rl)) return (double)NAN;
    return c.mu(rl) - c.mu(rv);
  };
  const double p_hi = c.p(rho_max) * (1.0 - 1e-13);
  double p_lo = c.p(rho_min);
  if (p_lo <= 0.0) p_lo = p_hi * 1e-30;
  for (int k = 0; k < 40 && h(p_lo) < 0.0; ++k) p_lo *= 1e-3;
  double ps;
  if (!ridders(h, p_lo, p_hi, ps)) return false;
  if (!roots(ps, rho_v, rho_l)) return false;
  // Newton polish on (rho_v, rho_l): p(v) - p(l) = 0, mu(v) - mu(l) = 0; d mu/d rho = p'/rho
  for (int it = 0; it < 4; ++it) {
    const double F1 = c.p(rho_v) - c.p(rho_l), F2 = c.mu(rho_v) - c.mu(rho_l);
    const double dv = c.dp(rho_v), dl = c.dp(rho_l);
    const double J11 = dv, J12 = -dl, J21 = dv / rho_v, J22 = -dl / rho_l;
    const double det = J11 * J22 - J12 * J21;
    if (!(std::fabs(det) > 0)) break;
    const double sv = (F1 * J22 - F2 * J12) / det, sl = (J11 * F2 - J21 * F1) / det;
    rho_v -= sv;
    rho_l -= sl;
  }
  p_sat = c.p(rho_v);
  return std::isfinite(rho_v) && std::isfinite(rho_l) && rho_v > 0 && rho_l > rho_v;
}

constexpr int kPanels = 48;

double maxwell_residual(const EosConst& e, double p_sat) {
  auto f = [&](double r) { return (p_sat - eos_pressure(e, r)) / (r * r); };
  return integrate_log(f, e.rho_v, e.rho_max, kPanels) + integrate_log(f, e.rho_max, e.rho_min, kPanels) +
         integrate_log(f, e.rho_min, e.rho_l, kPanels);
}

bool ellipse(double dp_dr, double delta, double dpress, double& asq, double& bb) {
  // Sec. III.D: k = dpress*delta/p'(end) - delta^2, a^2 = -k^2/(2k + delta^2),
  // b = dpress / (1 - sqrt(1 - delta^2/a^2)). With r = dpress/(p' delta) these are
  // a^2 = delta^2 (1 - r)^2/(1 - 2r), sqrt(1 - delta^2/a^2) = r/(1 - r) and
  // b = dpress (1 - r)/(1 - 2r); a is real for 0 < r < 1/2.
  const double r = dpress / (dp_dr * delta);
  if (!(r > 0.0 && r < 0.5)) return false;
  asq = delta * delta * (1.0 - r) * (1.0 - r) / (1.0 - 2.0 * r);
  bb = dpress * (1.0 - r) / (1.0 - 2.0 * r);
  return std::isfinite(asq) && std::isfinite(bb);
}

}  // namespace

EosConst make_eos_const(const pplbm_eos_derived& d) {
  EosConst e{};
  // shape of p(rho): the Modified Smooth EOS has the Smooth C-S shape
  e.mode = d.mode == PPLBM_EOS_SMOOTH_MOD ? PPLBM_EOS_SMOOTH : d.mode;
  e.b4 = d.b / 4.0;
  e.RT_l = d.R * d.T_l;
  e.a_l = d.a_l;
  if (d.mode == PPLBM_EOS_SMOOTH || d.mode == PPLBM_EOS_SMOOTH_MOD) {
    e.RT_v = d.R * d.T_v;
    e.a_v = d.a_v;
  } else {
    e.RT_v = e.RT_l;
    e.a_v = e.a_l;
  }
  e.dP = d.dP;
  e.rho_v = d.rho_v;
  e.rho_max = d.rho_max;
  e.rho_min = d.rho_min;
  e.rho_l = d.rho_l;
  e.p_max = d.p_max;
  e.b1 = d.b1;
  e.inv_a1sq = d.a1sq > 0 ? 1.0 / d.a1sq : 0.0;
  e.p_min = d.p_min;
  e.b3 = d.b3;
  e.inv_a3sq = d.a3sq > 0 ? 1.0 / d.a3sq : 0.0;
  e.inv_span = 1.0 / (d.rho_min - d.rho_max);
  e.a2 = 2.0 * (d.p_max - d.p_min);
  e.b2 = 3.0 * (d.p_min - d.p_max);
  e.psi2_scale = 2.0 / d.G;
  const double sc = e.psi2_scale;
  e.k1_v = sc * e.RT_v;
  e.k2_v = -sc * e.a_v;
  e.k4_v = 0.0;
  e.k1_l = sc * e.RT_l;
  e.k2_l = -sc * e.a_l;
  e.k4_l = sc * e.dP;
  e.k3 = -sc / 3.0;
  e.c1_v = 2.0 * e.k1_v;
  e.c1_l = 2.0 * e.k1_l;
  std::memcpy(&e.bits_rho_v, &e.rho_v, 8);
  std::memcpy(&e.bits_rho_max, &e.rho_max, 8);
  std::memcpy(&e.bits_rho_min, &e.rho_min, 8);
  std::memcpy(&e.bits_rho_l, &e.rho_l, 8);
  e.p_sat = d.p_sat;
  e.theta = d.theta;
  e.rho_m = d.rho_m;
  return e;
}

// dp/drho of the piece containing rho, from its closed form
static double eos_dpdrho(const EosConst& e, const pplbm_eos_derived& d, double r) {
  if (e.mode == PPLBM_EOS_CS) return cs_dp(r, d.a_l, d.b, d.R, d.T_l);
  if (e.mode == PPLBM_EOS_PENG) {
    if (r > e.rho_v && r < e.rho_l)
      return e.theta * ((r - e.rho_l) * (r - e.rho_m) + (r - e.rho_v) * (r - e.rho_m) + (r - e.rho_v) * (r - e.rho_l));
    return cs_dp(r, d.a_l, d.b, d.R, d.T_l);
  }
  if (r <= e.rho_v) return cs_dp(r, d.a_v, d.b, d.R, d.T_v);
  if (r <= e.rho_max) {
    const double x = r - e.rho_max;
    return -e.b1 * x * e.inv_a1sq / std::sqrt(1.0 - x * x * e.inv_a1sq);
  }
  if (r < e.rho_min) {
    const double t = (r - e.rho_max) * e.inv_span;
    return (3.0 * e.a2 * t + 2.0 * e.b2) * t * e.inv_span;
  }
  if (r < e.rho_l) {
    const double x = r - e.rho_min;
    return e.b3 * x * e.inv_a3sq / std::sqrt(1.0 - x * x * e.inv_a3sq);
  }
  return cs_dp(r, d.a_l, d.b, d.R, d.T_l);
}

// g(eps) = int_{rho_v}^{rho_l} (p_sat - p) psi'/psi^(1+eps) d rho (Eq. VaporLiqEq) and dg/deps,
// with psi^2 = (2/G)(p - rho/3): psi'/psi = (p' - 1/3)/(G psi^2); split where p is only C^1.
static void mech_integral(const pplbm_eos_derived& d, double eps, double* g_out, double* dg_out) {
  const EosConst e = make_eos_const(d);
  double edges[4] = {e.rho_v, e.rho_max, e.rho_min, e.rho_l};
  int nreg = 3;
  if (e.mode == PPLBM_EOS_PENG) {
    edges[1] = e.rho_l;
    nreg = 1;
  }
  double g = 0.0, dg = 0.0;
  for (int r = 0; r < nreg; ++r) {
    auto base = [&](double rho) {
      const double psi2 = eos_psi2(e, rho);
      const double dpsi_over_psi = (eos_dpdrho(e, d, rho) - 1.0 / 3.0) / (d.G * psi2);
      return (d.p_sat - eos_pressure(e, rho)) * dpsi_over_psi * std::pow(psi2, -0.5 * eps);
    };
    g += integrate_log(base, edges[r], edges[r + 1], kPanels);
    if (dg_out)
      dg += integrate_log([&](double rho) { return -0.5 * std::log(eos_psi2(e, rho)) * base(rho); }, edges[r],
                          edges[r + 1], kPanels);
  }
  *g_out = g;
  if (dg_out) *dg_out = dg;
}

// Newton from eps = 2 on g(eps) = 0 (Sec. III.A)
bool solve_eps(const pplbm_eos_derived& d, double& eps_out) {
  double eps = 2.0;
  for (int it = 0; it < 100; ++it) {
    double g, dg;
    mech_integral(d, eps, &g, &dg);
    if (!std::isfinite(g) || !std::isfinite(dg) || dg == 0.0) return false;
    const double step = g / dg;
    eps -= step;
    if (std::fabs(step) <= 1e-15 * std::fabs(eps)) {
      eps_out = eps;
      return true;
    }
  }
  return false;
}

}  // namespace pplbm

using namespace pplbm;

extern "C" pplbm_status pplbm_eos_setup(const pplbm_eos_params* p, double G, pplbm_eos_derived* out) {
  if (!p || !out) return PPLBM_ERR_ARG;
  if (p->mode < PPLBM_EOS_CS || p->mode > PPLBM_EOS_SMOOTH_MOD) return PPLBM_ERR_ARG;
  if (!(p->Tr > 0.0 && p->Tr < 1.0) || !(p->a_liq > 0) || !(p->b > 0) || !(p->R > 0) || !(G < 0.0))
    return PPLBM_ERR_ARG;
  const bool smooth = p->mode == PPLBM_EOS_SMOOTH || p->mode == PPLBM_EOS_SMOOTH_MOD;
  if (smooth && (!(p->a_vap > 0) || !(p->alpha > 0.0))) return PPLBM_ERR_ARG;
  if (p->mode == PPLBM_EOS_PENG && !(p->r_theta >= 0.0 && p->r_theta <= 1.0)) return PPLBM_ERR_ARG;
  pplbm_eos_derived d;
  std::memset(&d, 0, sizeof(d));
  d.mode = p->mode;
  d.G = G;
  d.b = p->b;
  d.R = p->R;
  d.a_l = p->a_liq;
  d.a_v = smooth ? p->a_vap : p->a_liq;
  double rho_c_l, rho_c_v;
  if (!critical_temperature(d.a_l, d.b, d.R, d.Tc_l, rho_c_l)) return PPLBM_ERR_EOS_SETUP;
  if (!critical_temperature(d.a_v, d.b, d.R, d.Tc_v, rho_c_v)) return PPLBM_ERR_EOS_SETUP;
  d.T_l = p->Tr * d.Tc_l;
  d.T_v = p->Tr * d.Tc_v;
  const Branch liq{d.a_l, d.b, d.R, d.T_l};
  const Branch vap{d.a_v, d.b, d.R, d.T_v};
  if (!spinodals(liq, rho_c_l, d.rho_max, d.rho_min)) return PPLBM_ERR_EOS_SETUP;
  if (!maxwell(liq, d.rho_max, d.rho_min, d.rho_v, d.rho_l, d.p_sat_cs)) return PPLBM_ERR_EOS_SETUP;
  d.p_min_cs = liq.p(d.rho_min);
  if (p->mode == PPLBM_EOS_CS) {
    d.p_sat = d.p_sat_cs;
    d.p_max = liq.p(d.rho_max);
    d.p_min = d.p_min_cs;
  } else if (p->mode == PPLBM_EOS_PENG) {
    // Eq. PengEOS: cubic through (rho_v, p_sat), (rho_l, p_sat); rho_m from Eq. VaporLiqEq with
    // eps = 0 at the Maxwell densities; theta from r_theta (Eq. PengTheta), a function of rho_m
    d.p_sat = d.p_sat_cs;
    d.p_max = liq.p(d.rho_max);
    d.p_min = d.p_min_cs;
    d.dpdrho_v = liq.dp(d.rho_v);
    d.dpdrho_l = liq.dp(d.rho_l);
    const double rt = p->r_theta;
    auto with_rho_m = [&](double rm) {
      pplbm_eos_derived t = d;
      t.rho_m = rm;
      t.theta = (1.0 - rt) / ((t.rho_v - rm) * (t.rho_v - t.rho_l)) * t.dpdrho_v +
                rt / ((t.rho_l - rm) * (t.rho_l - t.rho_v)) * t.dpdrho_l;
      return t;
    };
    auto resid = [&](double rm) {
      const pplbm_eos_derived t = with_rho_m(rm);
      const EosConst e = make_eos_const(t);
      for (int k = 0; k <= 64; ++k)  // psi^2 must stay positive on the loop
        if (!(eos_psi2(e, t.rho_v + (t.rho_l - t.rho_v) * k / 64.0) > 0.0)) return (double)NAN;
      double g;
      mech_integral(t, 0.0, &g, nullptr);
      return g;
    };
    const double span = d.rho_l - d.rho_v;
    double prev_x = d.rho_v + 1e-3 * span, prev_f = resid(prev_x), rm = NAN;
    for (int k = 1; k <= 120 && std::isnan(rm); ++k) {
      const double x = d.rho_v + span * (1e-3 + (1.0 - 2e-3) * k / 120.0);
      const double fx = resid(x);
      if (std::isfinite(prev_f) && std::isfinite(fx) && (prev_f > 0) != (fx > 0)) {
        double root;
        if (ridders(resid, prev_x, x, root)) rm = root;
      }
      prev_x = x;
      prev_f = fx;
    }
    if (std::isnan(rm)) return PPLBM_ERR_EOS_SETUP;
    const pplbm_eos_derived t = with_rho_m(rm);
    d.rho_m = t.rho_m;
    d.theta = t.theta;
  } else {
    // vapour branch: its own Maxwell construction (Eq. CS scales with a at fixed Tr, so its
    // coexistence densities coincide with the liquid branch's); p_sat is its Maxwell pressure
    double rv2, rl2, ps_v, rmax_v, rmin_v;
    if (!spinodals(vap, rho_c_v, rmax_v, rmin_v)) return PPLBM_ERR_EOS_SETUP;
    if (!maxwell(vap, rmax_v, rmin_v, rv2, rl2, ps_v)) return PPLBM_ERR_EOS_SETUP;
    d.p_sat = ps_v;
    d.dP = ps_v - d.p_sat_cs;
    d.dpdrho_v = vap.dp(d.rho_v);
    d.dpdrho_l = liq.dp(d.rho_l);
    d.p_min = d.p_sat - p->alpha * (d.p_sat_cs - d.p_min_cs);
    if (!ellipse(d.dpdrho_l, d.rho_l - d.rho_min, d.p_sat - d.p_min, d.a3sq, d.b3)) return PPLBM_ERR_EOS_SETUP;
    const double delta1 = d.rho_max - d.rho_v;
    const double hi = d.p_sat + 0.5 * d.dpdrho_v * delta1 * (1.0 - 1e-12);
    const double lo = d.p_sat + 1e-9 * (hi - d.p_sat);
    const bool modified = p->mode == PPLBM_EOS_SMOOTH_MOD;
    auto resid = [&](double pm) {
      pplbm_eos_derived t = d;
      t.p_max = pm;
      if (!ellipse(t.dpdrho_v, delta1, pm - t.p_sat, t.a1sq, t.b1)) return (double)NAN;
      if (modified) {  // Sec. IV.C: Eq. VaporLiqEq with eps = 0 instead of the Maxwell rule
        const EosConst e = make_eos_const(t);
        for (int k = 0; k <= 64; ++k)
          if (!(eos_psi2(e, t.rho_v * std::pow(t.rho_l / t.rho_v, k / 64.0)) > 0.0)) return (double)NAN;
        double g;
        mech_integral(t, 0.0, &g, nullptr);
        return g;
      }
      return maxwell_residual(make_eos_const(t), t.p_sat);
    };
    double pm;
    if (!ridders(resid, lo, hi, pm)) return PPLBM_ERR_EOS_SETUP;
    d.p_max = pm;
    if (!ellipse(d.dpdrho_v, delta1, pm - d.p_sat, d.a1sq, d.b1)) return PPLBM_ERR_EOS_SETUP;
  }
  if (p->mode == PPLBM_EOS_CS) {
    d.dpdrho_v = liq.dp(d.rho_v);
    d.dpdrho_l = liq.dp(d.rho_l);
  }
  const EosConst e = make_eos_const(d);
  const double pv2 = eos_psi2(e, d.rho_v), pl2 = eos_psi2(e, d.rho_l);
  if (!(pv2 > 0.0) || !(pl2 > 0.0)) return PPLBM_ERR_EOS_SETUP;
  d.psi_v = std::sqrt(pv2);
  d.psi_l = std::sqrt(pl2);
  // psi^2 must stay positive over the whole coexistence range
  for (int k = 0; k <= 2000; ++k) {
    const double r = d.rho_v * std::pow(1.2 * d.rho_l / d.rho_v, k / 2000.0);
    if (!(eos_psi2(e, r) > 0.0)) return PPLBM_ERR_EOS_SETUP;
  }
  if (p->mode == PPLBM_EOS_PENG || p->mode == PPLBM_EOS_SMOOTH_MOD) {
    d.eps = 0.0;  // built for the Guo scheme
  } else if (!solve_eps(d, d.eps)) {
    return PPLBM_ERR_EOS_SETUP;
  }
  *out = d;
  return PPLBM_OK;
}
