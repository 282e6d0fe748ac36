// Hand-written adjoint of the step (unit relaxation times, or the two-phase set of
// Sec. IV whose rows 7, 8 relax with 1/tau(rho), Eq. RelaxationTime), sqrt(N) checkpointed
// rollouts, and the EOS-constant sensitivities that chain the gradient to the
// shaping parameter alpha (Sec. III.D).
//
// Forward step at time t (step_device.cuh): rho, j, psi per node; g = 12 sum_i
// w_i psi(x + c_i) c_i; f*(x) = Phi(rho, j, psi(x), g; constants); push
// f^{t+1}_i(x + c_i) = f*_i(x) (bounce-back at walls). Given lambda^{t+1} =
// dL/df^{t+1}, one adjoint step is:
//   A1 (per node): mu_i(x) = lambda^{t+1}_i(x + c_i), or lambda^{t+1}_opp(i)(x)
//      beyond a wall (the transpose of the push, a gather); reverse mode through
//      Phi gives rho_bar, j_bar, psi_bar (own node), g_bar and the Li-term scale's
//      adjoint;
//   A2 (per node): psi_bar(y) += sum_c W_c (c_x gx_bar(y - c) + c_y gy_bar(y - c)),
//      the transpose of the psi stencil written as a gather (W = 4 axis, 1
//      diagonal; neighbours beyond a wall are ghosts with no adjoint), and with the
//      surface-tension source the transposes of its stencil sums t, sd, xd
//      (step_device.cuh; symmetric stencils, so the same sums of their adjoints); then
//      through psi = sqrt(psi^2(rho; constants)) to rho_bar and the constants'
//      adjoints; lambda^t_i = rho_bar + c_i . j_bar (+ the rows 7, 8 of Eq. MatrixMRT
//      times the stress moments' adjoints with the two-phase set).
// Constant adjoints are reduced per block and summed in a fixed order
// (deterministic); over a checkpointed rollout each block's sums accumulate
// across the steps and are reduced once at the end. Blocks with no node on a
// branch whose constants depend on alpha skip those reductions. The host maps
// the adjoints to d/d alpha with dconstants/dalpha.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "../../include/pplbm.h"
#include "ctx.h"
#include "step_device.cuh"

namespace pplbm {
namespace {

constexpr int kTX = 32, kTY = 8, kNT = kTX * kTY;
// adjoint workspace: kBarPlanes adjoint planes, two 9-plane lambda buffers, per-block partials
constexpr int kBarPlanes = 11;
constexpr int kLamOffset = kBarPlanes;            // in planes of n values
constexpr int kPartialOffset = kBarPlanes + 18;
// gradient slots: the constants of the shaped branches (which alpha moves), the
// Li-term scale, the bulk C-S constants the parameters a_vap and a_liq move, and the
// surface-tension control's kappa
enum {
  G_PMAX = 0, G_B1, G_IA1, G_A2, G_B2, G_PMIN, G_B3, G_IA3, G_ZZ, G_K1V, G_K2V, G_K1L, G_K2L, G_K4L, G_KAPPA, kNGrad
};
static_assert(kNGrad == PPLBM_NGRAD, "gradient slot count");
// A1 reduces G_ZZ and G_KAPPA (two values per block), A2 every other slot; A2's
// local index of slot k (k != G_ZZ, k < G_KAPPA)
constexpr int kA2 = kNGrad - 2;
__host__ __device__ constexpr int a2_index(int k) { return k < G_ZZ ? k : k - 1; }

struct AdjArgs {
  StepArgs a;            // forward arguments of step t (psi, mom filled by K1 on f^t)
  const double* lam1;    // lambda^{t+1}, 9 planes
  double* lam0;          // lambda^t, 9 planes
  double* bar;           // kBarPlanes planes: rho_bar, jx_bar, jy_bar, psi_bar (own), gx_bar, gy_bar,
                         // the surface-tension sums' t_bar, sd_bar, xd_bar, and (two-phase set)
                         // the stress moments' m7_bar, m8_bar
  double* partial1;      // per A1 block: the zz-scale and kappa adjoints
  double* partial2;      // per A2 block: kA2 constant adjoints (slot order without G_ZZ, G_KAPPA)
  int accumulate;        // add this step's block sums to the partials (a rollout) instead of storing them
  unsigned slots;        // bit k set: gradient slot k is accumulated (others stay 0)
};

// bits of the slots [k0, k1] of a group
__host__ __device__ constexpr unsigned slot_bits(int k0, int k1) { return ((2u << k1) - 1u) & ~((1u << k0) - 1u); }

// reverse mode of collide_reduced<kUnitTau> (see its comments for the forward). The
// surface-tension source only adds to zz, axp, ayp and Pxy, so the adjoints of those
// four (zq_b) are all it needs; they are returned when zq_b is not null.
__device__ __forceinline__ void collide_unit_reverse(const StepArgs& a, double rho, double jx, double jy, double psi0,
                                                     double gx, double gy, const double* mu, double* rho_b,
                                                     double* jx_b, double* jy_b, double* psi_b, double* gx_b,
                                                     double* gy_b, double* zs_b, double* zq_b = nullptr) {
  // forward recompute
  const double cH = a.half_force * psi0;
  const double hx = cH * gx, hy = cH * gy;
  const double inv = fast_rcp(rho);
  const double Jx = add_int(jx, hx), Jy = add_int(jy, hy);
  const double ux = Jx * inv, uy = Jy * inv;
  const double Px = fma(2.0, hx, jx), Py = fma(2.0, hy, jy);
  const double g2 = fma(gx, gx, gy * gy);
  // reverse
  const double dp_b = add_int(mu[5], mu[7]), ps_b = sub_int(mu[5], mu[7]) * (1.0 / 12.0);
  const double dm_b = add_int(mu[6], mu[8]), pd_b = sub_int(mu[6], mu[8]) * (1.0 / 12.0);
  const double Dq_b = add_int(dp_b, dm_b);
  const double Pxy_b = 0.25 * sub_int(dp_b, dm_b);
  const double D_b = Dq_b * (1.0 / 36.0);
  double zz_b = Dq_b;
  double r_b = D_b;
  double tr_b = 3.0 * D_b;
  const double axp_b = add_int(mu[1], mu[3]), ayp_b = add_int(mu[2], mu[4]);
  double Px_b = fma(sub_int(mu[1], mu[3]), 1.0 / 3.0, sub_int(ps_b, pd_b));
  double Py_b = fma(sub_int(mu[2], mu[4]), 1.0 / 3.0, add_int(ps_b, pd_b));
  const double Q_b = add_int(axp_b, ayp_b);
  double Pxx_b = 0.5 * axp_b, Pyy_b = 0.5 * ayp_b;
  const double B0_b = (4.0 / 9.0) * mu[0] + Q_b * (1.0 / 9.0);
  zz_b = add_int(zz_b, fma(-8.0, mu[0], Q_b));
  r_b = add_int(r_b, B0_b);
  tr_b += -1.5 * B0_b;
  Pxx_b = add_int(Pxx_b, tr_b);
  Pyy_b = add_int(Pyy_b, tr_b);
  // Pxy = ux Py + uy hx
  double ux_b = Pxy_b * Py, uy_b = Pxy_b * hx, hx_b = Pxy_b * uy;
  Py_b += Pxy_b * ux;
  // Pxx = ux (Px + hx), Pyy = uy (Py + hy)
  ux_b = fma(Pxx_b, add_int(Px, hx), ux_b);
  Px_b += Pxx_b * ux;
  hx_b += Pxx_b * ux;
  uy_b = fma(Pyy_b, add_int(Py, hy), uy_b);
  Py_b += Pyy_b * uy;
  double hy_b = Pyy_b * uy;
  // Px = jx + 2 hx, Py = jy + 2 hy
  double jx_bb = Px_b, jy_bb = Py_b;
  hx_b += 2.0 * Px_b;
  hy_b += 2.0 * Py_b;
  // ux = Jx inv, uy = Jy inv
  const double Jx_b = ux_b * inv, Jy_b = uy_b * inv;
  const double inv_b = ux_b * Jx + uy_b * Jy;
  jx_bb = add_int(jx_bb, Jx_b);
  hx_b = add_int(hx_b, Jx_b);
  jy_bb = add_int(jy_bb, Jy_b);
  hy_b = add_int(hy_b, Jy_b);
  r_b += -inv_b * inv * inv;
  // zz = zs g2
  const double zs = a.zz_scale;
  double gx_bb = 2.0 * zs * gx * zz_b, gy_bb = 2.0 * zs * gy * zz_b;
  *zs_b = zz_b * g2;
  // hx = cH gx, hy = cH gy, cH = hf psi0
  const double cH_b = hx_b * gx + hy_b * gy;
  gx_bb += hx_b * cH;
  gy_bb += hy_b * cH;
  *psi_b = cH_b * a.half_force;
  if (zq_b) {
    zq_b[0] = zz_b;
    zq_b[1] = axp_b;
    zq_b[2] = ayp_b;
    zq_b[3] = Pxy_b;
  }
  *rho_b = r_b;
  *jx_b = jx_bb;
  *jy_b = jy_bb;
  *gx_b = gx_bb;
  *gy_b = gy_bb;
}

// reverse mode of collide_reduced<kShearTau> (see its comments for the forward): rows
// 7, 8 relax with omega = 1/tau(rho), tau = tau_a + tau_b rho, as
//   m7* = (Pi_xx - Pi_yy) + (1 - omega) A7,  A7 = m7 - ux (jx - hx) + uy (jy - hy),
//   m8* = Pi_xy + (1 - omega) A8,           A8 = m8 - ux jy + uy hx,
// so the adjoint reaches rho also through omega, and m7, m8 (the density pass's stress
// moments) directly. With the surface-tension source (sq not null: zz += k t,
// m7* -= 4 omega k sd, m8* -= omega k xd) it returns st_b = {k_b, t_b, sd_b, xd_b}.
__device__ __forceinline__ void collide_shear_reverse(const StepArgs& a, double rho, double jx, double jy, double m7,
                                                      double m8, double psi0, double gx, double gy, const double* mu,
                                                      const SurfQ* sq, double* rho_b, double* jx_b, double* jy_b,
                                                      double* m7_b, double* m8_b, double* psi_b, double* gx_b,
                                                      double* gy_b, double* zs_b, double* st_b) {
  // forward recompute
  const double cH = a.half_force * psi0;
  const double hx = cH * gx, hy = cH * gy;
  const double inv = fast_rcp(rho);
  const double Jx = add_int(jx, hx), Jy = add_int(jy, hy);
  const double ux = Jx * inv, uy = Jy * inv;
  const double Px = fma(2.0, hx, jx), Py = fma(2.0, hy, jy);
  const double g2 = fma(gx, gx, gy * gy);
  const double om = fast_rcp(fma(a.tau_b, rho, a.tau_a));
  const double omc = sub_int(1.0, om);
  const double Kx = sub_int(jx, hx), Ky = sub_int(jy, hy);
  const double A7 = fma(-ux, Kx, fma(uy, Ky, m7));
  const double A8 = fma(-ux, jy, fma(uy, hx, m8));
  // reverse: population-space reconstruction
  const double dp_b = add_int(mu[5], mu[7]), ps_b = sub_int(mu[5], mu[7]) * (1.0 / 12.0);
  const double dm_b = add_int(mu[6], mu[8]), pd_b = sub_int(mu[6], mu[8]) * (1.0 / 12.0);
  const double Dq_b = add_int(dp_b, dm_b);
  const double Pxy_b = 0.25 * sub_int(dp_b, dm_b);
  double zz_b = Dq_b;
  double r_b = Dq_b * (1.0 / 36.0);
  double tr_b = Dq_b * (1.0 / 12.0);
  const double axp_b = add_int(mu[1], mu[3]), ayp_b = add_int(mu[2], mu[4]);
  double Px_b = fma(sub_int(mu[1], mu[3]), 1.0 / 3.0, sub_int(ps_b, pd_b));
  double Py_b = fma(sub_int(mu[2], mu[4]), 1.0 / 3.0, add_int(ps_b, pd_b));
  // axp, ayp = T4 +- m7*/4, T4 = Q + tr/4
  const double T4_b = add_int(axp_b, ayp_b);
  const double m7s_b = 0.25 * sub_int(axp_b, ayp_b);
  tr_b += 0.25 * T4_b;
  const double B0_b = (4.0 / 9.0) * mu[0] + T4_b * (1.0 / 9.0);
  zz_b = add_int(zz_b, fma(-8.0, mu[0], T4_b));
  r_b = add_int(r_b, B0_b);
  tr_b += -1.5 * B0_b;
  // rows 7, 8 (and the source's terms)
  const double A8_b = Pxy_b * omc, A7_b = m7s_b * omc;
  double om_b = -(Pxy_b * A8 + m7s_b * A7);  // through omc = 1 - omega
  if (sq) {
    const double w = fma(4.0 * sq->sd, m7s_b, sq->xd * Pxy_b);
    st_b[0] = fma(zz_b, sq->t, -om * w);  // k_b
    st_b[1] = zz_b * sq->k;               // t_b
    st_b[2] = -4.0 * om * sq->k * m7s_b;  // sd_b
    st_b[3] = -om * sq->k * Pxy_b;        // xd_b
    om_b -= sq->k * w;
  }
  r_b += -om_b * om * om * a.tau_b;  // d omega / d rho = -tau_b omega^2
  const double Pxx_b = add_int(m7s_b, tr_b), Pyy_b = sub_int(tr_b, m7s_b);
  // A8 = m8 - ux jy + uy hx
  double ux_b = -A8_b * jy, uy_b = A8_b * hx, hx_b = A8_b * uy;
  double jx_bb = 0.0, jy_bb = -A8_b * ux;
  // A7 = m7 - ux (jx - hx) + uy (jy - hy)
  ux_b -= A7_b * Kx;
  uy_b += A7_b * Ky;
  jx_bb -= A7_b * ux;
  hx_b += A7_b * ux;
  jy_bb += A7_b * uy;
  double hy_b = -A7_b * uy;
  // Pi_xy = ux Py + uy hx
  ux_b += Pxy_b * Py;
  Py_b += Pxy_b * ux;
  uy_b += Pxy_b * hx;
  hx_b += Pxy_b * uy;
  // Pi_xx = ux (Px + hx), Pi_yy = uy (Py + hy)
  ux_b = fma(Pxx_b, add_int(Px, hx), ux_b);
  Px_b += Pxx_b * ux;
  hx_b += Pxx_b * ux;
  uy_b = fma(Pyy_b, add_int(Py, hy), uy_b);
  Py_b += Pyy_b * uy;
  hy_b += Pyy_b * uy;
  // Px = jx + 2 hx, Py = jy + 2 hy
  jx_bb = add_int(jx_bb, Px_b);
  hx_b += 2.0 * Px_b;
  jy_bb = add_int(jy_bb, Py_b);
  hy_b += 2.0 * Py_b;
  // ux = Jx inv, uy = Jy inv
  const double Jx_b = ux_b * inv, Jy_b = uy_b * inv;
  const double inv_b = ux_b * Jx + uy_b * Jy;
  jx_bb = add_int(jx_bb, Jx_b);
  hx_b = add_int(hx_b, Jx_b);
  jy_bb = add_int(jy_bb, Jy_b);
  hy_b = add_int(hy_b, Jy_b);
  r_b += -inv_b * inv * inv;
  // zz = zs g2
  const double zs = a.zz_scale;
  double gx_bb = 2.0 * zs * gx * zz_b, gy_bb = 2.0 * zs * gy * zz_b;
  *zs_b = zz_b * g2;
  // hx = cH gx, hy = cH gy, cH = hf psi0
  const double cH_b = hx_b * gx + hy_b * gy;
  gx_bb += hx_b * cH;
  gy_bb += hy_b * cH;
  *psi_b = cH_b * a.half_force;
  *rho_b = r_b;
  *jx_b = jx_bb;
  *jy_b = jy_bb;
  *m7_b = A7_b;
  *m8_b = A8_b;
  *gx_b = gx_bb;
  *gy_b = gy_bb;
}

// Reverse mode of collide_reduced_fx (step_device.cuh), the collision the forward pass
// runs without the surface-tension source: unit relaxation times, or with SHEAR the
// rows 7, 8 relaxing at omega = 1/tau(rho). Forward, with s = 1/36:
//   h = cH g (cH = hf psi0); J, P, P + h (and K = j - h) from j_h_combos;
//   u' = J / (36 rho); xx = u'_x (P_x + h_x), yy likewise, xy = u'_x P_y + u'_y h_x;
//   zz = zs |g|^2; SHEAR: p7 = (1 - omega) A7, A7 = s m7 - u'_x K_x + u'_y K_y,
//   p8 = (1 - omega) A8, A8 = s m8 - u'_x j_y + u'_y h_x;
//   f* = reduced_populations(s rho, xx, yy, xy, s P_x, s P_y, zz, p7, p8).
// The adjoints of the populations' inputs come from the transposed integer stage
// (fx::reduced_populations_transpose), those of j and h from the transposed sums
// (fx::j_h_combos_transpose); the products between them are FP64.
// With SRC (a kernel built with the surface-tension source, run at kappa = 0, when the
// kappa gradient is asked for) it also returns src = {zz adjoint, row-7 adjoint, mixed
// moment adjoint, omega}: the source adds nothing at kappa = 0, and these give its
// adjoints.
template <bool SHEAR, bool SRC = false>
__device__ __forceinline__ void collide_reduced_reverse(const StepArgs& a, double rho, double jx, double jy,
                                                        double m7, double m8, double psi0, double gx, double gy,
                                                        const double* mu, double* rho_b, double* jx_b, double* jy_b,
                                                        double* m7_b, double* m8_b, double* psi_b, double* gx_b,
                                                        double* gy_b, double* zs_b, double* src = nullptr) {
  constexpr double s36 = 1.0 / 36.0;
  // forward recompute
  const double cH = a.half_force * psi0;
  const double hx = cH * gx, hy = cH * gy;
  double Jx, Px, Qx, Kx = 0.0, Jy, Py, Qy, Ky = 0.0;
  fx::j_h_combos<SHEAR>(jx, hx, &Jx, &Px, &Qx, &Kx);
  fx::j_h_combos<SHEAR>(jy, hy, &Jy, &Py, &Qy, &Ky);
  const double inv36 = fast_rcp(36.0 * rho);
  const double ux = Jx * inv36, uy = Jy * inv36;
  const double g2 = fma(gx, gx, gy * gy);
  // reverse: the populations' inputs
  const double m[9] = {mu[0], mu[1], mu[2], mu[3], mu[4], mu[5], mu[6], mu[7], mu[8]};
  double U[9];
  fx::reduced_populations_transpose<SHEAR, SHEAR || SRC>(m, U);
  if (SRC) {
    // the adjoints of zz, of the row-7 moment m7* (the axis populations carry +-m7*/4:
    // (mu1 + mu3 - mu2 - mu4)/4 = U7/36) and of the mixed moment Pi_xy*
    // ((mu5 + mu7 - mu6 - mu8)/4 = U8/36)
    src[0] = U[6];
    src[1] = U[7] * s36;
    src[2] = U[8] * s36;
    src[3] = 0.0;
  }
  double r_b = U[0] * s36;
  double Px_b = U[4] * s36, Py_b = U[5] * s36;
  // xx = ux Qx, yy = uy Qy, xy = ux Py + uy hx
  double ux_b = fma(U[3], Py, U[1] * Qx);
  double uy_b = fma(U[3], hx, U[2] * Qy);
  const double Qx_b = U[1] * ux, Qy_b = U[2] * uy;
  Py_b = fma(U[3], ux, Py_b);
  double hx_b = U[3] * uy, hy_b = 0.0;
  double Kx_b = 0.0, Ky_b = 0.0, jy_0 = 0.0;
  if (SHEAR) {
    const double om = fast_rcp(fma(a.tau_b, rho, a.tau_a));
    if (SRC) src[3] = om;
    const double omc = 1.0 - om;
    const double A7 = fma(-ux, Kx, fma(uy, Ky, m7 * s36));
    const double A8 = fma(-ux, jy, fma(uy, hx, m8 * s36));
    const double A7_b = U[7] * omc, A8_b = U[8] * omc;
    const double om_b = -fma(U[7], A7, U[8] * A8);  // through omc = 1 - omega
    r_b = fma(-om_b * om, om * a.tau_b, r_b);       // d omega / d rho = -tau_b omega^2
    *m7_b = A7_b * s36;
    *m8_b = A8_b * s36;
    // A7 = s m7 - ux Kx + uy Ky, A8 = s m8 - ux jy + uy hx
    ux_b = fma(-A7_b, Kx, fma(-A8_b, jy, ux_b));
    uy_b = fma(A7_b, Ky, fma(A8_b, hx, uy_b));
    Kx_b = -A7_b * ux;
    Ky_b = A7_b * uy;
    jy_0 = -A8_b * ux;
    hx_b = fma(A8_b, uy, hx_b);
  }
  // u' = J inv36, inv36 = 1/(36 rho): d inv36 / d rho = -36 inv36^2
  const double Jx_b = ux_b * inv36, Jy_b = uy_b * inv36;
  const double inv_b = fma(ux_b, Jx, uy_b * Jy);
  r_b = fma(-36.0 * inv_b * inv36, inv36, r_b);
  // J = j + h, P = j + 2h, P + h = j + 3h, K = j - h
  double jxb, hxb, jyb, hyb;
  fx::j_h_combos_transpose<SHEAR>(Jx_b, Px_b, Qx_b, Kx_b, 0.0, hx_b, &jxb, &hxb);
  fx::j_h_combos_transpose<SHEAR>(Jy_b, Py_b, Qy_b, Ky_b, jy_0, hy_b, &jyb, &hyb);
  // zz = zs g2
  const double zs = a.zz_scale;
  const double zg = 2.0 * zs * U[6];
  *zs_b = U[6] * g2;
  // h = cH g, cH = hf psi0
  const double cH_b = fma(hxb, gx, hyb * gy);
  *gx_b = fma(hxb, cH, zg * gx);
  *gy_b = fma(hyb, cH, zg * gy);
  *psi_b = cH_b * a.half_force;
  *rho_b = r_b;
  *jx_b = jxb;
  *jy_b = jyb;
}

// psi^2(rho) and its derivatives w.r.t. rho and the alpha-dependent constants (eos_dev.cuh);
// the C-S branch constants' derivatives only when bulk_slots (a uniform flag)
__device__ __forceinline__ double psi2_grad(const EosConst& e, double rho, bool bulk_slots, double* dc) {
  for (int k = 0; k < kA2; ++k) dc[k] = 0.0;
  const long long rb = dbits(rho);
  const bool vap = rb <= e.bits_rho_v, liq = rb >= e.bits_rho_l;
  if (e.mode == 2 && !vap && !liq) {  // Peng cubic loop: no alpha-dependent constants
    const double dv = rho - e.rho_v, dl = rho - e.rho_l, dm = rho - e.rho_m;
    const double dp = e.theta * (dl * dm + dv * dm + dv * dl);
    return e.psi2_scale * (dp - 1.0 / 3.0);
  }
  if (e.mode != 1 || vap || liq) {
    const bool use_v = (e.mode == 1) && vap;
    const double k1 = use_v ? e.k1_v : e.k1_l, k2 = use_v ? e.k2_v : e.k2_l;
    const double eta = e.b4 * rho, om = 1.0 - eta;
    const double r = fast_rcp(om), r2 = r * r;
    // psi^2 = rho (k1 Z + k2 rho + k3) + k4 (k4 of the vapour branch is 0), Z of Eq. CS;
    // d(rho Z)/drho = Z + eta Z'(eta) = (1 + 4 eta + 4 eta^2 - 4 eta^3 + eta^4) / (1 - eta)^4
    const double P = fma(eta, fma(eta, fma(eta, eta - 4.0, 4.0), 4.0), 1.0);
    if (bulk_slots) {  // constant indices only, so dc stays in registers
      const double Z = fma(eta, fma(eta, om, 1.0), 1.0) * (r2 * r);
      const double rz = rho * Z, rr = rho * rho;
      dc[a2_index(G_K1V)] = use_v ? rz : 0.0;
      dc[a2_index(G_K2V)] = use_v ? rr : 0.0;
      dc[a2_index(G_K1L)] = use_v ? 0.0 : rz;
      dc[a2_index(G_K2L)] = use_v ? 0.0 : rr;
      dc[a2_index(G_K4L)] = use_v ? 0.0 : 1.0;
    }
    return fma(k1 * (r2 * r2), P, fma(2.0 * k2, rho, e.k3));
  }
  const double s = e.psi2_scale;
  double dp;
  if (rb <= e.bits_rho_max) {
    const double d = rho - e.rho_max;
    const double s1 = fast_sqrt(fma(-d * d, e.inv_a1sq, 1.0));
    const double q = e.b1 * d * fast_rcp(s1);
    dp = -q * e.inv_a1sq;
    dc[a2_index(G_PMAX)] = s;
    dc[a2_index(G_B1)] = s * (s1 - 1.0);
    dc[a2_index(G_IA1)] = -0.5 * s * q * d;
  } else if (rb < e.bits_rho_min) {
    const double t = (rho - e.rho_max) * e.inv_span;
    dp = (3.0 * e.a2 * t + 2.0 * e.b2) * t * e.inv_span;
    dc[a2_index(G_PMAX)] = s;
    dc[a2_index(G_A2)] = s * t * t * t;
    dc[a2_index(G_B2)] = s * t * t;
  } else {
    const double d = rho - e.rho_min;
    const double s3 = fast_sqrt(fma(-d * d, e.inv_a3sq, 1.0));
    const double q = e.b3 * d * fast_rcp(s3);
    dp = q * e.inv_a3sq;
    dc[a2_index(G_PMIN)] = s;
    dc[a2_index(G_B3)] = s * (1.0 - s3);
    dc[a2_index(G_IA3)] = 0.5 * s * q * d;
  }
  return s * (dp - 1.0 / 3.0);
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  red[threadIdx.y * kTX + threadIdx.x] = v;
  __syncthreads();
  for (int w = kNT / 2; w > 0; w >>= 1) {
    const int t = threadIdx.y * kTX + threadIdx.x;
    if (t < w) red[t] += red[t + w];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

template <int KIND, bool ST>
__global__ void __launch_bounds__(kNT) k_adj_collide(const AdjArgs g) {
  __shared__ double sp[(kTY + 2) * (kTX + 2)];
  __shared__ double red[kNT];
  const StepArgs& a = g.a;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  load_psi_tile(a, sp, x0, y0, kTX, kTY, threadIdx.x, threadIdx.y, threadIdx.y * kTX + threadIdx.x, kNT);
  __syncthreads();
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
  double zs_b = 0.0, kap_b = 0.0;
  if (x < a.nx && y < a.ny) {
    const int c = (threadIdx.y + 1) * (kTX + 2) + threadIdx.x + 1, sw = kTX + 2;
    const double p0 = sp[c];
    // the forward collision pass's stencil sums (same arithmetic, same force)
    double gx, gy;
    fx::shan_chen_stencil(sp[c + 1], sp[c - 1], sp[c + sw], sp[c - sw], sp[c + sw + 1], sp[c + sw - 1],
                          sp[c - sw - 1], sp[c - sw + 1], &gx, &gy);
    const int64_t N = a.n, node = (int64_t)y * a.nx + x;
    const int nx = a.nx, ny = a.ny;
    const int xe = (x + 1 == nx) ? 0 : x + 1, xw = (x == 0) ? nx - 1 : x - 1;
    int yn = y + 1, ys = y - 1;
    bool up = false, down = false;
    if (a.walls) {
      up = (yn == ny);
      down = (ys < 0);
    } else {
      if (yn == ny) yn = 0;
      if (ys < 0) ys = ny - 1;
    }
    const int64_t row = (int64_t)y * nx, rn = (int64_t)yn * nx, rs = (int64_t)ys * nx;
    const double* L1 = g.lam1;
    // mu_i(x) = lambda^{t+1} at the node the push sent f*_i to
    double mu[9];
    mu[0] = L1[node];
    mu[1] = L1[N + row + xe];
    mu[3] = L1[3 * N + row + xw];
    mu[2] = up ? L1[4 * N + node] : L1[2 * N + rn + x];
    mu[5] = up ? L1[7 * N + node] : L1[5 * N + rn + xe];
    mu[6] = up ? L1[8 * N + node] : L1[6 * N + rn + xw];
    mu[4] = down ? L1[2 * N + node] : L1[4 * N + rs + x];
    mu[7] = down ? L1[5 * N + node] : L1[7 * N + rs + xw];
    mu[8] = down ? L1[6 * N + node] : L1[8 * N + rs + xe];
    double rb, jxb, jyb, pb, gxb, gyb;
    double st_b[4] = {0.0, 0.0, 0.0, 0.0};  // the source's k_b, t_b, sd_b, xd_b
    SurfQ sq = {0.0, 0.0, 0.0, 0.0};
    if (ST)
      sq = surface_q(a, p0, sp[c + 1], sp[c - 1], sp[c + sw], sp[c - sw], sp[c + sw + 1], sp[c + sw - 1],
                     sp[c - sw - 1], sp[c - sw + 1]);
    double* B = g.bar;
    if (!ST || a.kappa_q == 0.0) {
      // the forward ran collide_reduced_fx (no source, or kappa = 0 in a kernel with it)
      double m7b = 0.0, m8b = 0.0, src[4] = {0.0, 0.0, 0.0, 0.0};
      const bool shear = KIND == kShearTau;
      collide_reduced_reverse<KIND == kShearTau, ST>(a, a.mom[node], a.mom[N + node], a.mom[2 * N + node],
                                                     shear ? a.mom[3 * N + node] : 0.0,
                                                     shear ? a.mom[4 * N + node] : 0.0, p0, gx, gy, mu, &rb, &jxb,
                                                     &jyb, &m7b, &m8b, &pb, &gxb, &gyb, &zs_b, src);
      if (shear) {
        B[9 * N + node] = m7b;
        B[10 * N + node] = m8b;
      }
      if (ST) {
        // the source's adjoints at k = kappa_q psi = 0 (forward: zz += k t; unit: the
        // axis populations' m7*/4 parts -= +-k sd, Pxy -= k xd; two-phase: m7* -= 4 omega
        // k sd, m8* -= omega k xd): only the k adjoint is non-zero
        if (shear)
          st_b[0] = fma(src[0], sq.t, -src[3] * fma(4.0 * sq.sd, src[1], sq.xd * src[2]));
        else
          st_b[0] = fma(src[0], sq.t, -fma(4.0 * src[1], sq.sd, src[2] * sq.xd));
      }
    } else if (KIND == kShearTau) {
      double m7b, m8b;
      collide_shear_reverse(a, a.mom[node], a.mom[N + node], a.mom[2 * N + node], a.mom[3 * N + node],
                            a.mom[4 * N + node], p0, gx, gy, mu, ST ? &sq : nullptr, &rb, &jxb, &jyb, &m7b, &m8b, &pb,
                            &gxb, &gyb, &zs_b, st_b);
      B[9 * N + node] = m7b;
      B[10 * N + node] = m8b;
    } else {
      double zq_b[4];
      collide_unit_reverse(a, a.mom[node], a.mom[N + node], a.mom[2 * N + node], p0, gx, gy, mu, &rb, &jxb, &jyb,
                           &pb, &gxb, &gyb, &zs_b, ST ? zq_b : nullptr);
      if (ST) {
        // forward: zz += k t, axp -= k sd, ayp += k sd, Pxy -= k xd, k = kappa_q psi(x)
        const double dsd = zq_b[2] - zq_b[1];
        st_b[0] = fma(zq_b[0], sq.t, fma(dsd, sq.sd, -zq_b[3] * sq.xd));
        st_b[1] = zq_b[0] * sq.k;
        st_b[2] = dsd * sq.k;
        st_b[3] = -zq_b[3] * sq.k;
      }
    }
    if (ST) {
      // own node: k = kappa_q psi(x), and t carries -psi(x); kappa_q = kappa G / 24
      pb += fma(st_b[0], a.kappa_q, -st_b[1]);
      kap_b = st_b[0] * p0 * (a.G / 24.0);
      B[6 * N + node] = st_b[1];
      B[7 * N + node] = st_b[2];
      B[8 * N + node] = st_b[3];
    }
    B[node] = rb;
    B[N + node] = jxb;
    B[2 * N + node] = jyb;
    B[3 * N + node] = pb;
    B[4 * N + node] = gxb;
    B[5 * N + node] = gyb;
  }
  // grid-uniform tests
  const double s = (g.slots >> G_ZZ) & 1u ? block_sum(zs_b, red) : 0.0;
  const double sk = ST && ((g.slots >> G_KAPPA) & 1u) ? block_sum(kap_b, red) : 0.0;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    double* dst = g.partial1 + 2 * (blockIdx.y * gridDim.x + blockIdx.x);
    dst[0] = g.accumulate ? dst[0] + s : s;
    dst[1] = g.accumulate ? dst[1] + sk : sk;
  }
}

// tiles of adjoint planes p0 .. p0 + NP - 1 with a one-node halo (zero beyond a wall:
// ghosts carry no adjoint); tile j at s + j * (kTY + 2) * (kTX + 2)
template <int NP>
__device__ __forceinline__ void load_bar_tiles(const AdjArgs& g, int p0, double* s, int x0, int y0) {
  const StepArgs& a = g.a;
  const int sw = kTX + 2, ts = (kTY + 2) * sw;
  for (int k = threadIdx.y * kTX + threadIdx.x; k < ts; k += kNT) {
    const int ty = k / sw, tx = k - ty * sw;
    const int gx = wrap_index(x0 + tx - 1, a.nx);
    int gy = y0 + ty - 1;
    const bool in = !a.walls || (gy >= 0 && gy < a.ny);
    if (!a.walls) gy = wrap_index(gy, a.ny);
#pragma unroll
    for (int j = 0; j < NP; ++j) s[j * ts + k] = in ? g.bar[(p0 + j) * a.n + (int64_t)gy * a.nx + gx] : 0.0;
  }
}

// 4 resident blocks per SM (64 registers, 8-16 bytes spilled): at 71 registers and 3
// blocks the pass's FP64 pipe waits on latency (125 against 109 us on 1024^2)
template <int KIND, bool ST>
__global__ void __launch_bounds__(kNT, 4) k_adj_rho_psi(const AdjArgs g) {
  constexpr int ts = (kTY + 2) * (kTX + 2);
  __shared__ double tiles[(ST ? 5 : 2) * ts];  // gx_bar, gy_bar (and t_bar, sd_bar, xd_bar)
  __shared__ double red[kNT];
  double* sx = tiles;
  double* sy = tiles + ts;
  const StepArgs& a = g.a;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  load_bar_tiles<ST ? 5 : 2>(g, 4, tiles, x0, y0);
  __syncthreads();
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
  double dcsum[kA2];
  for (int k = 0; k < kA2; ++k) dcsum[k] = 0.0;
  // which constants this node's branch uses: the shaped loop's, the vapour C-S's
  // or the liquid C-S's
  bool shaped = false, vap_side = false, liq_side = false;
  if (x < a.nx && y < a.ny) {
    const int c = (threadIdx.y + 1) * (kTX + 2) + threadIdx.x + 1, sw = kTX + 2;
    // transpose of g = 12 sum_c w_c psi(x + c) c, gathered at this node y, plus the
    // node's own psi adjoint (one fixed-point frame, fixsum.cuh)
    const int64_t N = a.n, node = (int64_t)y * a.nx + x;
    const double gv[13] = {g.bar[3 * N + node], sx[c - 1], sx[c + 1], sy[c - sw], sy[c + sw],
                           sx[c - sw - 1], sy[c - sw - 1], sx[c + sw + 1], sy[c + sw + 1],
                           sx[c + sw - 1], sy[c + sw - 1], sx[c - sw + 1], sy[c - sw + 1]};
    double psi_b = fx::psi_adjoint_gather(gv);
    if constexpr (ST) {
      // transposes of t = (axis sum)/6 + (diagonal sum)/12 - psi(x), sd = (pE + pW) - (pN + pS),
      // xd = (pNE + pSW) - (pNW + pSE) at the neighbours (the -psi(x) term is A1's)
      const double* st = tiles + 2 * ts;
      const double* sd = tiles + 3 * ts;
      const double* sq = tiles + 4 * ts;
      const double ta = (st[c + 1] + st[c - 1]) + (st[c + sw] + st[c - sw]);
      const double tg = (st[c + sw + 1] + st[c - sw - 1]) + (st[c + sw - 1] + st[c - sw + 1]);
      psi_b += fma(1.0 / 6.0, ta, fma(1.0 / 12.0, tg, ((sd[c + 1] + sd[c - 1]) - (sd[c + sw] + sd[c - sw])) +
                                                      ((sq[c + sw + 1] + sq[c - sw - 1]) - (sq[c + sw - 1] + sq[c - sw + 1]))));
    }
    const double rho = a.mom[node];
    const double psi = a.psi[node];
    double dc[kA2];
    const double dpsi2 = psi2_grad(a.eos, rho, (g.slots & slot_bits(G_K1V, G_K4L)) != 0u, dc);
    const double psi2_b = 0.5 * psi_b * fast_rcp(psi);  // psi = sqrt(psi^2) > 0 (checked by the step)
    const double rho_b = g.bar[node] + psi2_b * dpsi2;
    const long long rb = dbits(rho);
    const bool vap = rb <= a.eos.bits_rho_v, liq = rb >= a.eos.bits_rho_l;
    // as in psi2_grad: C-S (shape 0) uses the liquid constants everywhere, the Peng
    // loop (2) outside (rho_v, rho_l), the shaped EOS (1) on its liquid branch
    const int m = a.eos.mode;
    shaped = m == 1 && !vap && !liq && (g.slots & slot_bits(G_PMAX, G_IA3));
    vap_side = m == 1 && vap && (g.slots & slot_bits(G_K1V, G_K2V));
    liq_side = (m == 0 || (m == 2 && (vap || liq)) || (m == 1 && liq)) && (g.slots & slot_bits(G_K1L, G_K4L));
    // only the group this node's branch uses is non-zero (constant loop bounds)
    if (shaped)
      for (int k = a2_index(G_PMAX); k <= a2_index(G_IA3); ++k) dcsum[k] = psi2_b * dc[k];
    if (vap_side)
      for (int k = a2_index(G_K1V); k <= a2_index(G_K2V); ++k) dcsum[k] = psi2_b * dc[k];
    if (liq_side)
      for (int k = a2_index(G_K1L); k <= a2_index(G_K4L); ++k) dcsum[k] = psi2_b * dc[k];
    const double jxb = g.bar[N + node], jyb = g.bar[2 * N + node];
    // lambda^t_i = rho_bar + c_i . j_bar (+ rows 7, 8 of Eq. MatrixMRT times the stress
    // moments' adjoints with the two-phase set), exact in one frame (fixsum.cuh)
    constexpr bool kShear = KIND == kShearTau;
    double l[9];
    fx::lambda_assembly<kShear>(rho_b, jxb, jyb, kShear ? g.bar[9 * N + node] : 0.0,
                                kShear ? g.bar[10 * N + node] : 0.0, l);
    double* L0 = g.lam0;
#pragma unroll
    for (int k = 0; k < 9; ++k) L0[k * N + node] = l[k];
  }
  const int blk = blockIdx.y * gridDim.x + blockIdx.x;
  double* dst = g.partial2 + (int64_t)blk * kA2;
  // Block-uniform tests: a group of constants that no node of the block uses adds
  // exact zeros, so its reductions are skipped.
  const bool any_shaped = __syncthreads_or(shaped);
  const bool any_vap = __syncthreads_or(vap_side);
  const bool any_liq = __syncthreads_or(liq_side);
  auto group = [&](int k0, int k1, bool used) {
    for (int k = k0; k < k1; ++k) {
      const int slot = k < G_ZZ ? k : k + 1;
      const double s = used && ((g.slots >> slot) & 1u) ? block_sum(dcsum[k], red) : 0.0;
      if (threadIdx.x == 0 && threadIdx.y == 0) dst[k] = g.accumulate ? dst[k] + s : s;
    }
  };
  group(a2_index(G_PMAX), a2_index(G_IA3) + 1, any_shaped);
  group(a2_index(G_K1V), a2_index(G_K2V) + 1, any_vap);
  group(a2_index(G_K1L), a2_index(G_K4L) + 1, any_liq);
}

// grad[k] += sum over blocks, in a fixed order; one block per gradient slot
__global__ void __launch_bounds__(256) k_adj_reduce(const double* partial1, const double* partial2, int nblocks,
                                                    double* grad) {
  __shared__ double red[256];
  const int k = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += 256)
    acc += k == G_ZZ ? partial1[2 * b] : k == G_KAPPA ? partial1[2 * b + 1] : partial2[(int64_t)b * kA2 + a2_index(k)];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) grad[k] += red[0];
}

// f_i = w_i rho0 is f^eq at rest; its transpose: rho0_bar = sum_i w_i lambda_i
__global__ void k_adj_init(int64_t n, const double* lam, double* rho_bar) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double w[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
  double s = 0.0;
  for (int k = 0; k < 9; ++k) s += w[k] * lam[k * n + i];
  rho_bar[i] = s;
}

int nblocks(const StepArgs& a) { return ((a.nx + kTX - 1) / kTX) * ((a.ny + kTY - 1) / kTY); }

}  // namespace
}  // namespace pplbm

using namespace pplbm;

namespace {

size_t adj_bytes(const pplbm_lattice* l) {
  const size_t n = (size_t)l->nx * l->ny;
  const size_t nb = (size_t)((l->nx + kTX - 1) / kTX) * ((l->ny + kTY - 1) / kTY);
  return sizeof(double) * (kPartialOffset * n + nb * kNGrad + 64);
}

// one adjoint step given the forward arguments of step t whose psi and moment
// planes hold psi(f^t) and the moments of f^t: lambda_next -> lambda_t, grad += ...
pplbm_status adjoint_core(pplbm_ctx* c, const StepArgs& a, const double* lam1, double* lam0, double* grad,
                          double* ws, bool accumulate, bool reduce) {
  AdjArgs g;
  g.a = a;
  g.lam1 = lam1;
  g.lam0 = lam0;
  g.bar = ws;
  const int nb = nblocks(a);
  g.partial1 = ws + kPartialOffset * c->n;
  g.partial2 = g.partial1 + 2 * nb;
  g.accumulate = accumulate ? 1 : 0;
  g.slots = c->adj_slots;
  const dim3 grid((a.nx + kTX - 1) / kTX, (a.ny + kTY - 1) / kTY), block(kTX, kTY);
  const bool st = a.kappa_q != 0.0 || ((g.slots >> G_KAPPA) & 1u);  // with the source (kappa_q may be 0)
  if (a.kind == kShearTau) {
    if (st) {
      k_adj_collide<kShearTau, true><<<grid, block, 0, c->stream>>>(g);
      k_adj_rho_psi<kShearTau, true><<<grid, block, 0, c->stream>>>(g);
    } else {
      k_adj_collide<kShearTau, false><<<grid, block, 0, c->stream>>>(g);
      k_adj_rho_psi<kShearTau, false><<<grid, block, 0, c->stream>>>(g);
    }
  } else if (st) {
    k_adj_collide<kUnitTau, true><<<grid, block, 0, c->stream>>>(g);
    k_adj_rho_psi<kUnitTau, true><<<grid, block, 0, c->stream>>>(g);
  } else {
    k_adj_collide<kUnitTau, false><<<grid, block, 0, c->stream>>>(g);
    k_adj_rho_psi<kUnitTau, false><<<grid, block, 0, c->stream>>>(g);
  }
  if (reduce) k_adj_reduce<<<kNGrad, 256, 0, c->stream>>>(g.partial1, g.partial2, nb, grad);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    c->msg = cudaGetErrorString(e);
    return PPLBM_ERR_CUDA;
  }
  return PPLBM_OK;
}

// one adjoint step at state f_t (device): the density pass fills the context's
// psi and moment planes first
pplbm_status adjoint_step(pplbm_ctx* c, const double* f_t, const double* lam1, double* lam0, double* grad,
                          double* ws, bool accumulate, bool reduce) {
  StepArgs a = c->args;
  a.f_in = f_t;
  a.f_out = nullptr;
  launch_rho_psi(a, c->stream);
  return adjoint_core(c, a, lam1, lam0, grad, ws, accumulate, reduce);
}

pplbm_status forward_into(pplbm_ctx* c, const double* fin, double* fout) {
  StepArgs a = c->args;
  a.f_in = fin;
  a.f_out = fout;
  launch_rho_psi(a, c->stream);
  launch_collide(a, c->stream);
  return cudaGetLastError() == cudaSuccess ? PPLBM_OK : PPLBM_ERR_CUDA;
}

}  // namespace

extern "C" {

size_t pplbm_adjoint_workspace_bytes(const pplbm_lattice* lattice) {
  if (!lattice || lattice->nx < 1 || lattice->ny < 1) return 0;
  return adj_bytes(lattice);
}

// the adjoint differentiates collide_reduced<kUnitTau> and <kShearTau> (with or without
// the surface-tension source); the general six-time MRT set is not covered
static pplbm_status adjoint_supported(pplbm_ctx* c) {
  if (c->args.kind != kUnitTau && c->args.kind != kShearTau) {
    c->msg = "the adjoint covers unit relaxation times and the two-phase set only";
    return PPLBM_ERR_STATE;
  }
  return PPLBM_OK;
}

// planes kept per step by the stored and segment modes: psi and the moment planes
static int field_planes(const pplbm_ctx* c) { return 1 + moment_planes(c->args.kind); }

pplbm_status pplbm_adjoint_step(pplbm_ctx* c, const double* f_t, const double* lambda_next, double* lambda_t,
                                double* grad, void* adj_workspace, size_t adj_workspace_bytes) {
  if (!c || !f_t || !lambda_next || !lambda_t || !grad || !adj_workspace) return PPLBM_ERR_ARG;
  if (pplbm_status s = adjoint_supported(c)) return s;
  if (adj_workspace_bytes < adj_bytes(&c->lat)) return PPLBM_ERR_ARG;
  return adjoint_step(c, f_t, lambda_next, lambda_t, grad, (double*)adj_workspace, false, true);
}

pplbm_status pplbm_forward_checkpointed(pplbm_ctx* c, int64_t nsteps, int64_t interval, double* checkpoints) {
  if (!c || nsteps < 0 || interval < 1 || !checkpoints) return PPLBM_ERR_ARG;
  if (c->sticky) return c->sticky;
  const int64_t stride = 9 * c->n;
  for (int64_t t = 0; t < nsteps; ++t) {
    if (t % interval == 0) {
      if (cudaMemcpyAsync(checkpoints + (t / interval) * stride, c->fA, sizeof(double) * stride,
                          cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
        return PPLBM_ERR_CUDA;
    }
    if (pplbm_status s = pplbm_step(c, 1)) return s;
  }
  return PPLBM_OK;
}

pplbm_status pplbm_backward_checkpointed(pplbm_ctx* c, int64_t nsteps, int64_t interval, const double* checkpoints,
                                         double* segment, const double* lambda_N, double* lambda_0, double* grad,
                                         void* adj_workspace, size_t adj_workspace_bytes) {
  if (!c || nsteps < 0 || interval < 1 || !checkpoints || !segment || !lambda_N || !lambda_0 || !grad ||
      !adj_workspace)
    return PPLBM_ERR_ARG;
  if (pplbm_status s = adjoint_supported(c)) return s;
  if (adj_workspace_bytes < adj_bytes(&c->lat)) return PPLBM_ERR_ARG;
  if (c->sticky) return c->sticky;
  const int64_t stride = 9 * c->n;
  double* ws = (double*)adj_workspace;
  double* lamA = ws + kLamOffset * c->n;  // lambda ping-pong inside the adjoint workspace
  double* lamB = lamA + stride;
  cudaStream_t s = c->stream;
  if (cudaMemcpyAsync(lamA, lambda_N, sizeof(double) * stride, cudaMemcpyDefault, s) != cudaSuccess)
    return PPLBM_ERR_CUDA;
  double* cur = lamA;
  double* nxt = lamB;
  // per-block constant adjoints are summed over the whole rollout, then reduced once
  const size_t nb = (size_t)nblocks(c->args);
  double* partials = ws + kPartialOffset * c->n;
  if (cudaMemsetAsync(partials, 0, sizeof(double) * nb * kNGrad, s) != cudaSuccess) return PPLBM_ERR_CUDA;
  if (nsteps > 0) {
    const int64_t nseg = (nsteps + interval - 1) / interval;
    // With interval >= 4 the segment buffer (interval x 9 planes) holds two f
    // buffers plus psi and the three moments of every state of the segment: the
    // recomputation keeps what its density passes produce and the adjoint steps
    // reuse it. Shorter intervals store the states themselves.
    const int fp = field_planes(c);
    const bool keep_fields = 9 * interval >= 18 + fp * interval;
    const int64_t n = c->n;
    for (int64_t j = nseg - 1; j >= 0; --j) {
      const int64_t t0 = j * interval, t1 = std::min(nsteps, t0 + interval);
      if (cudaMemcpyAsync(segment, checkpoints + j * stride, sizeof(double) * stride, cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess)
        return PPLBM_ERR_CUDA;
      if (keep_fields) {
        double* fb[2] = {segment, segment + stride};
        double* fields = segment + 2 * stride;  // per state: psi and the moment planes
        for (int64_t t = t0; t < t1; ++t) {
          StepArgs a = c->args;
          a.f_in = fb[(t - t0) & 1];
          a.f_out = fb[(t - t0 + 1) & 1];
          a.psi = fields + (t - t0) * fp * n;
          a.mom = a.psi + n;
          launch_rho_psi(a, s);
          if (t + 1 < t1) launch_collide(a, s);
        }
        if (cudaGetLastError() != cudaSuccess) return PPLBM_ERR_CUDA;
        for (int64_t t = t1 - 1; t >= t0; --t) {
          StepArgs a = c->args;
          a.psi = fields + (t - t0) * fp * n;
          a.mom = a.psi + n;
          if (pplbm_status st = adjoint_core(c, a, cur, nxt, grad, ws, true, false)) return st;
          std::swap(cur, nxt);
        }
      } else {
        for (int64_t t = t0; t + 1 < t1; ++t)
          if (pplbm_status st = forward_into(c, segment + (t - t0) * stride, segment + (t - t0 + 1) * stride))
            return st;
        for (int64_t t = t1 - 1; t >= t0; --t) {
          if (pplbm_status st = adjoint_step(c, segment + (t - t0) * stride, cur, nxt, grad, ws, true, false))
            return st;
          std::swap(cur, nxt);
        }
      }
    }
  }
  k_adj_reduce<<<kNGrad, 256, 0, s>>>(partials, partials + 2 * nb, (int)nb, grad);
  if (cudaGetLastError() != cudaSuccess) return PPLBM_ERR_CUDA;
  if (cudaMemcpyAsync(lambda_0, cur, sizeof(double) * stride, cudaMemcpyDefault, s) != cudaSuccess)
    return PPLBM_ERR_CUDA;
  return PPLBM_OK;
}

pplbm_status pplbm_forward_stored(pplbm_ctx* c, int64_t nsteps, double* fields) {
  if (!c || nsteps < 0 || !fields) return PPLBM_ERR_ARG;
  if (pplbm_status s = adjoint_supported(c)) return s;
  if (c->sticky) return c->sticky;
  const int64_t n = c->n;
  for (int64_t t = 0; t < nsteps; ++t) {
    // the density pass of step t writes psi, rho, j of f^t into slot t, which the
    // collision pass reads: the same arithmetic as pplbm_step, kept per step
    StepArgs a = c->args;
    a.f_in = c->fA;
    a.f_out = c->fB;
    a.psi = fields + t * field_planes(c) * n;
    a.mom = a.psi + n;
    launch_rho_psi(a, c->stream);
    launch_collide(a, c->stream);
    std::swap(c->fA, c->fB);
  }
  if (cudaGetLastError() != cudaSuccess) return PPLBM_ERR_CUDA;
  c->steps += nsteps;
  return PPLBM_OK;
}

pplbm_status pplbm_backward_stored(pplbm_ctx* c, int64_t nsteps, const double* fields, const double* lambda_N,
                                   double* lambda_0, double* grad, void* adj_workspace, size_t adj_workspace_bytes) {
  if (!c || nsteps < 0 || !fields || !lambda_N || !lambda_0 || !grad || !adj_workspace) return PPLBM_ERR_ARG;
  if (pplbm_status s = adjoint_supported(c)) return s;
  if (adj_workspace_bytes < adj_bytes(&c->lat)) return PPLBM_ERR_ARG;
  if (c->sticky) return c->sticky;
  const int64_t n = c->n, stride = 9 * n;
  double* ws = (double*)adj_workspace;
  double* cur = ws + kLamOffset * n;
  double* nxt = cur + stride;
  cudaStream_t s = c->stream;
  if (cudaMemcpyAsync(cur, lambda_N, sizeof(double) * stride, cudaMemcpyDefault, s) != cudaSuccess)
    return PPLBM_ERR_CUDA;
  const size_t nb = (size_t)nblocks(c->args);
  double* partials = ws + kPartialOffset * n;
  if (cudaMemsetAsync(partials, 0, sizeof(double) * nb * kNGrad, s) != cudaSuccess) return PPLBM_ERR_CUDA;
  for (int64_t t = nsteps - 1; t >= 0; --t) {
    StepArgs a = c->args;
    a.psi = const_cast<double*>(fields) + t * field_planes(c) * n;
    a.mom = a.psi + n;
    if (pplbm_status st = adjoint_core(c, a, cur, nxt, grad, ws, true, false)) return st;
    std::swap(cur, nxt);
  }
  k_adj_reduce<<<kNGrad, 256, 0, s>>>(partials, partials + 2 * nb, (int)nb, grad);
  if (cudaGetLastError() != cudaSuccess) return PPLBM_ERR_CUDA;
  if (cudaMemcpyAsync(lambda_0, cur, sizeof(double) * stride, cudaMemcpyDefault, s) != cudaSuccess)
    return PPLBM_ERR_CUDA;
  return PPLBM_OK;
}

pplbm_status pplbm_adjoint_set_slots(pplbm_ctx* c, uint32_t mask) {
  if (!c || (mask >> kNGrad) != 0u) return PPLBM_ERR_ARG;
  c->adj_slots = mask;
  return PPLBM_OK;
}

pplbm_status pplbm_adjoint_set_param(pplbm_ctx* c, int32_t which, double h) {
  if (!c || which < 0 || which > 3 || !(h > 0.0)) return PPLBM_ERR_ARG;
  double dc[PPLBM_NGRAD];
  if (pplbm_status s = pplbm_eos_constant_sensitivity(&c->eos_params, c->G, &c->relax, which, h, dc)) return s;
  uint32_t mask = 0u;
  for (int k = 0; k < PPLBM_NGRAD; ++k) {
    c->adj_dc[k] = dc[k];
    if (dc[k] != 0.0) mask |= 1u << k;
  }
  c->adj_param = which;
  c->adj_slots = mask;
  return PPLBM_OK;
}

pplbm_status pplbm_adjoint_param_gradient(pplbm_ctx* c, const double* grad, double* out) {
  if (!c || !grad || !out) return PPLBM_ERR_ARG;
  if (c->adj_param < 0) return PPLBM_ERR_STATE;
  double g[PPLBM_NGRAD];
  if (cudaMemcpyAsync(g, grad, sizeof(g), cudaMemcpyDefault, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return PPLBM_ERR_CUDA;
  double acc = 0.0;  // fixed slot order: deterministic
  for (int k = 0; k < PPLBM_NGRAD; ++k)
    if (c->adj_slots & (1u << k)) acc += g[k] * c->adj_dc[k];
  out[0] = acc;
  return PPLBM_OK;
}

pplbm_status pplbm_adjoint_initial_density(pplbm_ctx* c, const double* lambda_0, double* rho0_bar) {
  if (!c || !lambda_0 || !rho0_bar) return PPLBM_ERR_ARG;
  k_adj_init<<<(unsigned)((c->n + 255) / 256), 256, 0, c->stream>>>(c->n, lambda_0, rho0_bar);
  return cudaGetLastError() == cudaSuccess ? PPLBM_OK : PPLBM_ERR_CUDA;
}

pplbm_status pplbm_eos_grad_constants(const pplbm_eos_derived* d, double c[PPLBM_NGRAD]) {
  if (!d || !c) return PPLBM_ERR_ARG;
  const EosConst e = make_eos_const(*d);
  const double vals[PPLBM_NGRAD] = {e.p_max, e.b1, e.inv_a1sq, e.a2, e.b2, e.p_min, e.b3,
                                    e.inv_a3sq, 0.0, e.k1_v, e.k2_v, e.k1_l, e.k2_l, e.k4_l, 0.0};
  std::memcpy(c, vals, sizeof(vals));
  return PPLBM_OK;
}

pplbm_status pplbm_eos_constant_sensitivity(const pplbm_eos_params* p, double G, const pplbm_relax* relax,
                                            int32_t which, double h, double dc[PPLBM_NGRAD]) {
  if (!p || !relax || !dc || which < 0 || which > 3 || !(h > 0.0)) return PPLBM_ERR_ARG;
  if (which == 3) {  // kappa is its own slot
    for (int k = 0; k < PPLBM_NGRAD; ++k) dc[k] = k == G_KAPPA ? 1.0 : 0.0;
    return PPLBM_OK;
  }
  auto at = [&](double v, double* out) -> pplbm_status {
    pplbm_eos_params q = *p;
    (which == 0 ? q.alpha : which == 1 ? q.a_vap : q.a_liq) = v;
    pplbm_eos_derived d;
    if (pplbm_status s = pplbm_eos_setup(&q, G, &d)) return s;
    pplbm_eos_grad_constants(&d, out);
    const double sigma = relax->forcing == PPLBM_FORCING_GUO ? 0.0
                         : relax->sigma_auto               ? -d.eps / (16.0 * G)
                                                           : relax->sigma;
    out[G_ZZ] = sigma * G * G / 432.0;
    return PPLBM_OK;
  };
  double a1[PPLBM_NGRAD], a2[PPLBM_NGRAD], b1[PPLBM_NGRAD], b2[PPLBM_NGRAD];
  const double a0 = which == 0 ? p->alpha : which == 1 ? p->a_vap : p->a_liq;
  if (pplbm_status s = at(a0 + h, a1)) return s;
  if (pplbm_status s = at(a0 - h, a2)) return s;
  if (pplbm_status s = at(a0 + h / 2, b1)) return s;
  if (pplbm_status s = at(a0 - h / 2, b2)) return s;
  for (int k = 0; k < PPLBM_NGRAD; ++k) {
    const double d1 = (a1[k] - a2[k]) / (2 * h), d2 = (b1[k] - b2[k]) / h;
    dc[k] = (4 * d2 - d1) / 3;  // Richardson: O(h^4)
  }
  return PPLBM_OK;
}

}  // extern "C"
