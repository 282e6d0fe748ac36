// Host derivation of the collision arguments from a relaxation set, shared by the
// single-lattice context, the batched engine and the no-allocation entry point.
#include <cmath>

#include "internal.h"

namespace pplbm {

int collision_kind(const pplbm_relax* r) {
  if (!r || r->reserved != 0) return -1;
  if (!std::isfinite(r->kappa) || !(r->kappa < 1.0)) return -1;
  if (r->forcing != PPLBM_FORCING_GUO && r->forcing != PPLBM_FORCING_LI) return -1;
  if (r->kind == PPLBM_RELAX_TWO_PHASE) {
    if (!(r->tau_l > 0.5) || !(r->visc_ratio > 0.0) || !std::isfinite(r->tau_l) || !std::isfinite(r->visc_ratio))
      return -1;
    return kShearTau;
  }
  if (r->kind != PPLBM_RELAX_MRT) return -1;
  const double t[6] = {r->tau_rho, r->tau_e, r->tau_zeta, r->tau_j, r->tau_q, r->tau_nu};
  for (double v : t)
    if (!(v > 0.5) || !std::isfinite(v)) return -1;
  if (r->tau_rho == 1.0 && r->tau_e == 1.0 && r->tau_zeta == 1.0 && r->tau_j == 1.0 && r->tau_q == 1.0)
    return r->tau_nu == 1.0 ? kUnitTau : kShearTau;
  return kFullMrt;
}

void set_collision_args(StepArgs& a, int kind, const pplbm_relax& r, const pplbm_eos_derived& d, double G) {
  // Li forcing parameter (Eq. LiFS): 0 for the Guo scheme (Eq. GFS), or from eps of
  // Eq. VaporLiqEq for the EOS in use (Sec. III.A)
  const double sigma = r.forcing == PPLBM_FORCING_GUO ? 0.0 : r.sigma_auto ? -d.eps / (16.0 * G) : r.sigma;
  a.tau_a = a.tau_b = 0.0;
  if (kind == kShearTau) {
    if (r.kind == PPLBM_RELAX_TWO_PHASE) {
      // tau = tau_l (rho - rho_v)/(rho_l - rho_v) + tau_v (rho - rho_l)/(rho_v - rho_l),
      // tau_v = 1/2 + v_r (tau_l - 1/2) (Eq. RelaxationTime)
      const double tv = 0.5 + r.visc_ratio * (r.tau_l - 0.5);
      a.tau_b = (r.tau_l - tv) / (d.rho_l - d.rho_v);
      a.tau_a = r.tau_l - a.tau_b * d.rho_l;
    } else {
      a.tau_a = r.tau_nu;
    }
  }
  a.zz_scale = sigma * G * G / 432.0;
  a.kappa_q = r.kappa * G / 24.0;
  if (kind == kFullMrt) {
    const double t[9] = {r.tau_rho, r.tau_e, r.tau_zeta, r.tau_j, r.tau_q, r.tau_j, r.tau_q, r.tau_nu, r.tau_nu};
    for (int k = 0; k < 9; ++k) a.omega[k] = 1.0 / t[k];
    a.li_e = 12.0 * sigma / (r.tau_e - 0.5);
    a.li_z = 12.0 * sigma / (r.tau_zeta - 0.5);
  }
}

}  // namespace pplbm
