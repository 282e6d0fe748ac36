// Equation-of-state evaluation shared by the host set-up and the kernels.
//
// Carnahan-Starling (Sec. III, Eq. CS):
//   p = rho R T (1 + eta + eta^2 - eta^3) / (1 - eta)^3 - a rho^2,  eta = b rho / 4.
// Smooth C-S (Sec. III.D), piecewise in rho:
//   rho <= rho_v            : C-S with the vapour-branch a_v (and T_v = Tr Tc(a_v))
//   rho_v < rho <= rho_max  : ellipse 1: p_max - b1 + b1 sqrt(1 - (rho - rho_max)^2 / a1^2)
//   rho_max < rho < rho_min : cubic a2 t^3 + b2 t^2 + p_max, t = (rho - rho_max)/(rho_min - rho_max),
//                             a2 = 2 (p_max - p_min), b2 = 3 (p_min - p_max)
//   rho_min <= rho < rho_l  : ellipse 3: p_min + b3 - b3 sqrt(1 - (rho - rho_min)^2 / a3^2)
//   rho >= rho_l            : C-S with the liquid-branch a_l, plus Delta P
// Pseudopotential (Eq. InteractionPotential, c = 1): psi^2 = 2 (p - rho/3) / G.
#pragma once

#include <cmath>

#ifndef __CUDACC__
#define PPLBM_HD
#else
#define PPLBM_HD __host__ __device__
#endif

namespace pplbm {

// Constants for fast evaluation, built once from pplbm_eos_derived.
struct EosConst {
  int mode;            // shape of p(rho): 0 C-S everywhere, 1 Smooth C-S regions, 2 Peng cubic loop
  int pad;
  double b4;           // b / 4
  double RT_v, a_v;    // vapour branch (mode SMOOTH); equals the liquid branch for mode CS
  double RT_l, a_l, dP;
  double rho_v, rho_max, rho_min, rho_l;
  double p_max, b1, inv_a1sq;
  double p_min, b3, inv_a3sq;
  double inv_span, a2, b2;
  double psi2_scale;   // 2 / G: psi^2 = psi2_scale * (p - rho/3)
  // C-S branches folded into psi^2 (kernels): with s = 2/G,
  // psi^2 = rho (k1 num/(1 - eta)^3 + k2 rho + k3) + k4, k1 = s R T, k2 = -s a, k3 = -s/3, k4 = s dP
  double k1_v, k2_v, k4_v;
  double k1_l, k2_l, k4_l;
  double k3;
  // 2 k1 of each branch, for the kernels' form of Eq. CS: with v = 1/(1 - eta),
  // (1 + eta + eta^2 - eta^3)/(1 - eta)^3 = 2 v^3 - 2 v + 1, so that
  // k1 num/(1 - eta)^3 = c1 (v (v^2 - 1) + 1/2), c1 = 2 k1
  double c1_v, c1_l;
  // bit patterns of the branch densities (positive doubles order like their bits)
  long long bits_rho_v, bits_rho_max, bits_rho_min, bits_rho_l;
  double p_sat, theta, rho_m;  // Peng loop: p_sat + theta (rho - rho_v)(rho - rho_l)(rho - rho_m)
};

PPLBM_HD inline double cs_pressure(double rho, double b4, double RT, double a) {
  const double eta = b4 * rho;
  const double om = 1.0 - eta;
  const double num = 1.0 + eta * (1.0 + eta * (1.0 - eta));
  return rho * RT * num / (om * om * om) - a * rho * rho;
}

PPLBM_HD inline double eos_pressure(const EosConst& e, double rho) {
  if (e.mode == 0) return cs_pressure(rho, e.b4, e.RT_l, e.a_l);
  if (e.mode == 2) {
    if (rho > e.rho_v && rho < e.rho_l) return e.p_sat + e.theta * (rho - e.rho_v) * (rho - e.rho_l) * (rho - e.rho_m);
    return cs_pressure(rho, e.b4, e.RT_l, e.a_l);
  }
  if (rho <= e.rho_v) return cs_pressure(rho, e.b4, e.RT_v, e.a_v);
  if (rho <= e.rho_max) {
    const double d = rho - e.rho_max;
    return e.p_max - e.b1 + e.b1 * sqrt(1.0 - d * d * e.inv_a1sq);
  }
  if (rho < e.rho_min) {
    const double t = (rho - e.rho_max) * e.inv_span;
    return (e.a2 * t + e.b2) * t * t + e.p_max;
  }
  if (rho < e.rho_l) {
    const double d = rho - e.rho_min;
    return e.p_min + e.b3 - e.b3 * sqrt(1.0 - d * d * e.inv_a3sq);
  }
  return cs_pressure(rho, e.b4, e.RT_l, e.a_l) + e.dP;
}

PPLBM_HD inline double eos_psi2(const EosConst& e, double rho) {
  return e.psi2_scale * (eos_pressure(e, rho) - rho * (1.0 / 3.0));
}

}  // namespace pplbm
