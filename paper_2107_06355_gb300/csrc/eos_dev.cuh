// Device evaluation of psi^2(rho) for the step kernels (Sec. III.D shaped EOS,
// Eq. CS, Eq. InteractionPotential), arranged for few FP64 instructions:
//  * bulk vapour and liquid nodes (rho <= rho_v or rho >= rho_l, and every node
//    of the plain C-S EOS) take one branch-free path whose constants are
//    selected on the integer pipe; Eq. CS and psi^2 = (2/G)(p - rho/3) are folded
//    into psi^2 = rho (k1 num / (1 - eta)^3 + k2 rho + k3) + k4, with the C-S factor
//    num / (1 - eta)^3 = 2 v^3 - 2 v + 1, v = 1/(1 - eta) (9 FP64 instructions);
//  * interface nodes (rho_v < rho < rho_l, Smooth C-S) evaluate ellipse 1, the
//    cubic or ellipse 3;
//  * branch tests compare bit patterns (integer pipe).
#pragma once

#include "eos.cuh"
#include "fp64.cuh"

namespace pplbm {

__device__ __forceinline__ double eos_psi2_dev(const EosConst& e, double rho) {
  const long long rb = dbits(rho);
  const bool vap = rb <= e.bits_rho_v;
  const bool liq = rb >= e.bits_rho_l;
  if (e.mode == 2 && !vap && !liq) {  // Peng cubic loop (Eq. PengEOS)
    const double p = fma(e.theta * (rho - e.rho_v), (rho - e.rho_l) * (rho - e.rho_m), e.p_sat);
    return e.psi2_scale * fma(-rho, 1.0 / 3.0, p);
  }
  if (e.mode != 1 || vap || liq) {
    const bool use_v = (e.mode == 1) && vap;
    const double c1 = use_v ? e.c1_v : e.c1_l;
    const double k2 = use_v ? e.k2_v : e.k2_l;
    const double k4 = use_v ? e.k4_v : e.k4_l;
    // Eq. CS with v = 1/(1 - eta): (1 + eta + eta^2 - eta^3)/(1 - eta)^3 = 2 v^3 - 2 v + 1
    // (substitute eta = 1 - 1/v), i.e. k1 num/(1 - eta)^3 = c1 (v (v^2 - 1) + 1/2)
    const double v = fast_rcp(fma(-e.b4, rho, 1.0));
    const double x = fma(c1, fma(v, fma(v, v, -1.0), 0.5), fma(k2, rho, e.k3));
    return fma(rho, x, k4);
  }
  double p;
  if (rb <= e.bits_rho_max) {
    const double d = rho - e.rho_max;
    p = fma(e.b1, fast_sqrt(fma(-d * d, e.inv_a1sq, 1.0)), e.p_max - e.b1);
  } else if (rb < e.bits_rho_min) {
    const double t = (rho - e.rho_max) * e.inv_span;
    p = fma(fma(e.a2, t, e.b2), t * t, e.p_max);
  } else {
    const double d = rho - e.rho_min;
    p = fma(-e.b3, fast_sqrt(fma(-d * d, e.inv_a3sq, 1.0)), e.p_min + e.b3);
  }
  return e.psi2_scale * fma(-rho, 1.0 / 3.0, p);
}

}  // namespace pplbm
