// Per-node device code of the two step kernels, shared by the single-lattice
// kernels (step_kernels.cu) and the batched multi-lattice kernels (batch.cu) so
// that both perform identical arithmetic.
//
// The GB300 FP64 pipe issues about 0.6e12 instructions/s, some 60x below FP32,
// so these kernels are bound by FP64 issue rather than HBM: the arithmetic is
// arranged to minimise FP64 instructions per node.
//  * K1 hands K2 the moments instead of the populations, so K2 never re-sums f.
//  * With Lambda = I or with only the shear rates relaxing, f* is rebuilt
//    directly as w_i [rho + 3 c.P + 4.5 (c c - I/3) : Pi] plus the sigma term of
//    the Li scheme, which M^-1 maps onto (-8, 1, ..., 1) z. This equals
//    M^-1 m* for the moment vector m* of Eq. LiFS / GFS.
//  * |F|^2 / psi^2 is (G^2/144) |g|^2 with g the weighted psi differences, so the
//    Li term needs no division by psi^2.
//  * The optional surface-tension control (template flag ST) adds Li & Luo's
//    source C to m*; in population space it joins the Li term's z and the rows
//    7, 8 terms, so it costs about 15 FP64 instructions per node, and nothing when
//    the flag is off.
#pragma once

#include <cuda_runtime.h>

#include "eos_dev.cuh"
#include "fixsum.cuh"
#include "fp64.cuh"
#include "internal.h"

namespace pplbm {

// K1 body for node i: moments, EOS, psi (Eqs. Density, Momentum, CS, Sec. III.D,
// InteractionPotential); error word on a non-finite or non-positive density or psi^2.
template <int KIND>
__device__ __forceinline__ void rho_psi_node(const StepArgs& a, const double* __restrict__ f, int64_t i) {
  const int64_t N = a.n;
  const double f0 = f[i], f1 = f[N + i], f2 = f[2 * N + i], f3 = f[3 * N + i], f4 = f[4 * N + i];
  const double f5 = f[5 * N + i], f6 = f[6 * N + i], f7 = f[7 * N + i], f8 = f[8 * N + i];
  double rho, jx, jy, m7 = 0.0, m8 = 0.0;
  // When all nine populations are positive normal doubles (every bulk and interface
  // node of a physical state), the moments are exact integer sums in one fixed-point
  // frame, each rounded once (fixsum.cuh): integer-pipe work only, leaving the FP64
  // pipe, the pass's bottleneck, the EOS. Otherwise the same moments as IEEE sums.
  const double fv[9] = {f0, f1, f2, f3, f4, f5, f6, f7, f8};
  unsigned max_hi = 0;
  if (KIND != kFullMrt && fx::positive_normal_range(fv, &max_hi)) {
    fx::density_moments<KIND == kShearTau>(fv, fx::frame_top(max_hi), &rho, &jx, &jy, &m7, &m8);
  } else if (KIND == kShearTau) {
    // rows 7, 8 of Eq. MatrixMRT share their pair sums with rho
    const double a13 = f1 + f3, a24 = f2 + f4, a57 = f5 + f7, a68 = f6 + f8;
    rho = f0 + ((a13 + a24) + (a57 + a68));
    const double p = f5 - f7, q = f6 - f8;
    jx = (f1 - f3) + (p - q);
    jy = (f2 - f4) + (p + q);
    m7 = a13 - a24;
    m8 = a57 - a68;
  } else {
    const double sxp = f1 + f5 + f8;  // populations with c_x = +1
    const double sxm = f3 + f6 + f7;  // c_x = -1
    rho = (f0 + f2 + f4) + (sxp + sxm);
    jx = sxp - sxm;
    jy = (f2 + f5 + f6) - (f4 + f7 + f8);
  }
  const double psi2 = eos_psi2_dev(a.eos, rho);
  // 0 < rho < 1e300 and 0 < psi^2 < inf, tested on the bit patterns (integer pipe)
  const long long rb = dbits(rho), pb = dbits(psi2);
  if (!(rb > 0 && rb < 0x7E37E43C8800759CLL && pb > 0 && pb < 0x7FF0000000000000LL)) atomicOr(a.err, 1);
  a.psi[i] = fast_sqrt(psi2);
  double* __restrict__ m = a.mom;
  m[i] = rho;
  m[N + i] = jx;
  m[2 * N + i] = jy;
  if (KIND == kShearTau) {
    m[3 * N + i] = m7;  // row 7 of Eq. MatrixMRT
    m[4 * N + i] = m8;  // row 8
  } else if (KIND == kFullMrt) {
    const double ax = f1 + f2 + f3 + f4, dg = f5 + f6 + f7 + f8;
    m[3 * N + i] = -4.0 * f0 - ax + 2.0 * dg;                    // row 1 (e)
    m[4 * N + i] = 4.0 * f0 - 2.0 * ax + dg;                     // row 2 (varsigma)
    m[5 * N + i] = -2.0 * (f1 - f3) + ((f5 - f6) - (f7 - f8));   // row 4 (q_x)
    m[6 * N + i] = -2.0 * (f2 - f4) + ((f5 + f6) - (f7 + f8));   // row 6 (q_y)
    m[7 * N + i] = (f1 + f3) - (f2 + f4);                        // row 7
    m[8 * N + i] = (f5 + f7) - (f6 + f8);                        // row 8
  }
}

__device__ __forceinline__ int wrap_index(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// v mod n for v in [-n, 2n) by one conditional add or subtract (no division); other
// values (a lattice narrower than a tile) through the remainder
__device__ __forceinline__ int wrap_near(int v, int n) {
  v += v < 0 ? n : 0;
  v -= v >= n ? n : 0;
  return (v >= 0 && v < n) ? v : wrap_index(v, n);
}

// psi at lattice column gx (any integer: periodic wrap) and row gy in [-1, ny]
// (periodic, or the wall ghost values beyond the walls)
__device__ __forceinline__ double psi_wrapped(const StepArgs& a, int gx, int gy) {
  gx = wrap_near(gx, a.nx);
  if (a.walls) {
    if (gy < 0) return a.psi_ghost_bottom;
    if (gy >= a.ny) return a.psi_ghost_top;
  } else {
    gy = wrap_near(gy, a.ny);
  }
  return a.psi[(int64_t)gy * a.nx + gx];
}

// psi of the tile [x0 - 1, x0 + tw] x [y0 - 1, y0 + th] into sp (row stride tw + 2):
// periodic wrap in x; periodic in y, or the wall ghost values beyond the walls. The
// block has tw * th threads: thread (lx, ly) loads its own node, then the 2 (tw + 2)
// + 2 th halo values are shared out, rows first (no division by the tile width).
__device__ __forceinline__ void load_psi_tile(const StepArgs& a, double* sp, int x0, int y0, int tw, int th, int lx,
                                              int ly, int tid, int nthreads) {
  const int sw = tw + 2;
  sp[(ly + 1) * sw + lx + 1] = psi_wrapped(a, x0 + lx, y0 + ly);
  const int nh = 2 * sw + 2 * th;
  for (int k = tid; k < nh; k += nthreads) {
    int tx, ty;
    if (k < 2 * sw) {
      const bool top = k >= sw;
      ty = top ? th + 1 : 0;
      tx = top ? k - sw : k;
    } else {
      const int j = k - 2 * sw;
      ty = 1 + (j >> 1);
      tx = (j & 1) ? tw + 1 : 0;
    }
    sp[ty * sw + tx] = psi_wrapped(a, x0 + tx - 1, y0 + ty - 1);
  }
}

struct Post {
  double f[9];
};

// Surface-tension control (the technique of the paper's Sec. V; Li & Luo 2013):
// Q_ab = kappa (G/2) psi(x) sum_i w(|c_i|^2) [psi(x + c_i) - psi(x)] c_ia c_ib, kept as
// raw stencil sums with the scale k = kappa_q psi(x) (kappa_q = kappa G / 24), so that
// each use is one FMA:
//   (Q_xx + Q_yy) / 24 = k t,  t = (pE + pW + pN + pS)/6 + (four diagonals)/12 - psi,
//   Q_xx - Q_yy = 4 k sd,     sd = (pE + pW) - (pN + pS),
//   Q_xy = k xd,              xd = (pNE + pSW) - (pNW + pSE)
// (12 sum_i w_i [psi_i - psi] c_x^2 = 4 (pE + pW) + diagonals - 12 psi, likewise in y).
struct SurfQ {
  double k, t, sd, xd;
};

__device__ __forceinline__ SurfQ surface_q(const StepArgs& a, double p0, double pE, double pW, double pN, double pS,
                                           double pNE, double pNW, double pSW, double pSE) {
  const double sA = pE + pW, sB = pN + pS;
  const double dP = pNE + pSW, dM = pNW + pSE;
  SurfQ q;
  q.k = a.kappa_q * p0;
  q.t = fma(1.0 / 6.0, sA + sB, fma(1.0 / 12.0, dP + dM, -p0));
  q.sd = sA - sB;
  q.xd = dP - dM;
  return q;
}

// Collision for Lambda = I (KIND kUnitTau) or shear-only relaxation (kShearTau).
//
// With h = F/2: J = j + h = rho u (Eq. Momentum), P = j + 2h (momentum after the
// step), and the post-collision second moments (Lambda = I)
//   Pi_xx = rho ux^2 + ux Fx = ux (P_x + h_x),  Pi_yy = uy (P_y + h_y),
//   Pi_xy = rho ux uy + (ux Fy + uy Fx)/2 = ux P_y + uy h_x.
// These are rows 1, 7, 8 of m* = m_eq + S/2 (Eqs. LiFS, GFS with tau = 1);
// kShearTau relaxes rows 7, 8 with omega = 1/tau(rho) instead (Eq. RelaxationTime).
// Then
//   f*_i = w_i [rho + 3 c_i.P + 4.5 (c_i c_i - I/3) : Pi] + z_i,
// z_i = zz (-8, 1, 1, 1, 1, 1, 1, 1, 1) being M^-1 applied to the Li sigma terms
// +-12 sigma |F|^2 / psi^2 of rows 1 and 2 (tau_e = tau_zeta = 1), zz = sigma |F|^2 / (3 psi^2).
// With ST, the surface-tension source's rows 1, 2 (+-1.5 tr Q) map onto the same
// shape with zz += tr Q / 24, and rows 7, 8 (-l_nu (Q_xx - Q_yy), -l_nu Q_xy) add to
// the post-collision m_7, m_8 (l_nu = 1, or omega for kShearTau).
template <int KIND, bool ST = false>
__device__ __forceinline__ void collide_reduced(const StepArgs& a, int64_t node, double rho, double jx, double jy,
                                                double psi0, double gx, double gy, const SurfQ& sq, Post& out,
                                                double* ux_o, double* uy_o) {
  // Additions run on the integer pipe (add_int, bitwise the FP64 add): the FP64
  // pipe, this pass's bottleneck, keeps the products and fused multiply-adds.
  const double cH = a.half_force * psi0;  // h = cH g, cH = -G psi / 24
  const double hx = cH * gx, hy = cH * gy;
  const double inv_rho = fast_rcp(rho);
  const double ux = add_int(jx, hx) * inv_rho, uy = add_int(jy, hy) * inv_rho;
  *ux_o = ux;
  *uy_o = uy;
  const double Px = fma(2.0, hx, jx), Py = fma(2.0, hy, jy);
  const double Pxx = ux * add_int(Px, hx), Pyy = uy * add_int(Py, hy);
  const double tr = add_int(Pxx, Pyy);
  const double Pxy_eq = fma(ux, Py, uy * hx);
  double zz = a.zz_scale * fma(gx, gx, gy * gy);
  if (ST) zz = fma(sq.k, sq.t, zz);  // + tr Q / 24
  const double B0 = fma(-1.5, tr, rho);
  const double Q = fma(B0, 1.0 / 9.0, zz);
  double axp, ayp, Pxy;
  if (KIND == kUnitTau) {
    axp = fma(0.5, Pxx, Q);
    ayp = fma(0.5, Pyy, Q);
    Pxy = Pxy_eq;
    if (ST) {
      axp = fma(-sq.k, sq.sd, axp);  // m_7* -= Q_xx - Q_yy, n_7 = m_7 / 4
      ayp = fma(sq.k, sq.sd, ayp);
      Pxy = fma(-sq.k, sq.xd, Pxy);  // m_8* -= Q_xy
    }
  } else {
    // rows 7, 8: m* = m - omega (m - m_eq) + (1 - omega/2) S. With m_eq + S/2 the
    // unit-tau values Pi_xx - Pi_yy and Pi_xy above, this is
    //   m* = (m_eq + S/2) + (1 - omega) (m + S - m_eq - S/2),
    // and the brackets reduce to m7 - ux (jx - hx) + uy (jy - hy) and m8 - ux jy + uy hx.
    const double om = fast_rcp(fma(a.tau_b, rho, a.tau_a));
    const double omc = sub_int(1.0, om);
    const double m7 = a.mom[3 * a.n + node], m8 = a.mom[4 * a.n + node];
    const double A7 = fma(-ux, sub_int(jx, hx), fma(uy, sub_int(jy, hy), m7));
    const double A8 = fma(-ux, jy, fma(uy, hx, m8));
    double m7s = fma(omc, A7, sub_int(Pxx, Pyy));
    Pxy = fma(omc, A8, Pxy_eq);
    if (ST) {
      const double ok = om * sq.k;
      m7s = fma(-4.0 * ok, sq.sd, m7s);  // -omega (Q_xx - Q_yy)
      Pxy = fma(-ok, sq.xd, Pxy);        // -omega Q_xy
    }
    const double T4 = fma(0.25, tr, Q);
    axp = fma(0.25, m7s, T4);  // Q + Pi_xx/2 with Pi_xx = (tr + m7*)/2
    ayp = fma(-0.25, m7s, T4);
  }
  out.f[0] = fma(4.0 / 9.0, B0, -8.0 * zz);
  out.f[1] = fma(Px, 1.0 / 3.0, axp);
  out.f[3] = fma(-Px, 1.0 / 3.0, axp);
  out.f[2] = fma(Py, 1.0 / 3.0, ayp);
  out.f[4] = fma(-Py, 1.0 / 3.0, ayp);
  const double Dq = fma(fma(3.0, tr, rho), 1.0 / 36.0, zz);
  const double dp = fma(0.25, Pxy, Dq), dm = fma(-0.25, Pxy, Dq);
  const double ps = add_int(Px, Py), pd = sub_int(Py, Px);
  out.f[5] = fma(ps, 1.0 / 12.0, dp);
  out.f[7] = fma(-ps, 1.0 / 12.0, dp);
  out.f[6] = fma(pd, 1.0 / 12.0, dm);
  out.f[8] = fma(-pd, 1.0 / 12.0, dm);
}

// The same collision (Lambda = I, or rows 7, 8 at omega = 1/tau(rho) for kShearTau),
// without the surface-tension source, arranged so that the FP64 pipe does only the
// products, the reciprocals and the Li term (19 FP64 instructions per node for unit
// relaxation times, 32 for the two-phase set): the sums J = j + h, P = j + 2h,
// P + h (and j - h) come from one fixed-point frame, and the nine populations are
// exact small-integer combinations of the inputs scaled by 1/36 (fixsum.cuh), each
// rounded once, instead of chains of FP64 fused multiply-adds.
template <int KIND>
__device__ __forceinline__ void collide_reduced_fx(const StepArgs& a, int64_t node, double rho, double jx, double jy,
                                                   double psi0, double gx, double gy, Post& out) {
  constexpr bool kShear = KIND == kShearTau;
  const double cH = a.half_force * psi0;  // h = F/2 = cH g, cH = -G psi / 24
  const double hx = cH * gx, hy = cH * gy;
  double Jx, Px, Qx, Kx = 0.0, Jy, Py, Qy, Ky = 0.0;
  fx::j_h_combos<kShear>(jx, hx, &Jx, &Px, &Qx, &Kx);
  fx::j_h_combos<kShear>(jy, hy, &Jy, &Py, &Qy, &Ky);
  const double inv36 = fast_rcp(36.0 * rho);
  const double ux = Jx * inv36, uy = Jy * inv36;  // u / 36
  const double xx = ux * Qx, yy = uy * Qy;        // Pi_xx / 36 = u_x (P_x + h_x) / 36
  const double xy = fma(ux, Py, uy * hx);         // Pi_xy / 36
  const double zz = a.zz_scale * fma(gx, gx, gy * gy);
  constexpr double s36 = 1.0 / 36.0;
  double p7 = 0.0, p8 = 0.0;
  if (kShear) {
    // rows 7, 8: m* = m_eq + S/2 + (1 - omega)(m + S/2 - m_eq), the brackets
    // A7 = m7 - u_x (j_x - h_x) + u_y (j_y - h_y), A8 = m8 - u_x j_y + u_y h_x
    const double om = fast_rcp(fma(a.tau_b, rho, a.tau_a));
    const double omc = 1.0 - om;
    const double A7 = fma(-ux, Kx, fma(uy, Ky, a.mom[3 * a.n + node] * s36));
    const double A8 = fma(-ux, jy, fma(uy, hx, a.mom[4 * a.n + node] * s36));
    p7 = omc * A7;
    p8 = omc * A8;
  }
  fx::reduced_populations<kShear>(rho * s36, xx, yy, xy, Px * s36, Py * s36, zz, p7, p8, out.f);
}

// General MRT collision in moment space (six relaxation times). With ST the
// surface-tension source C_k = l_k D_k enters as the shift D of m_eq in rows 1, 2,
// 7, 8 (+1.5 tr Q, -1.5 tr Q, -(Q_xx - Q_yy), -Q_xy), since m - l (m - m_eq - D) =
// m - l (m - m_eq) + l D.
template <bool ST = false>
__device__ __forceinline__ void collide_full(const StepArgs& a, int64_t node, double psi0, double gx, double gy,
                                             const SurfQ& sq, Post& out, double* rho_o, double* ux_o,
                                             double* uy_o) {
  const int64_t N = a.n;
  double m[9];
  m[0] = a.mom[node];
  m[3] = a.mom[N + node];
  m[5] = a.mom[2 * N + node];
  m[1] = a.mom[3 * N + node];
  m[2] = a.mom[4 * N + node];
  m[4] = a.mom[5 * N + node];
  m[6] = a.mom[6 * N + node];
  m[7] = a.mom[7 * N + node];
  m[8] = a.mom[8 * N + node];
  const double rho = m[0];
  const double cF = 2.0 * a.half_force * psi0;
  const double Fx = cF * gx, Fy = cF * gy;
  const double Jx = fma(0.5, Fx, m[3]), Jy = fma(0.5, Fy, m[5]);
  const double inv_rho = fast_rcp(rho);
  const double ux = Jx * inv_rho, uy = Jy * inv_rho;
  *rho_o = rho;
  *ux_o = ux;
  *uy_o = uy;
  const double ru2 = fma(ux, Jx, uy * Jy);
  const double uF = fma(ux, Fx, uy * Fy);
  const double F2p = a.G * a.G * (1.0 / 144.0) * fma(gx, gx, gy * gy);  // |F|^2 / psi^2
  double meq[9], S[9];
  meq[0] = rho;                   S[0] = 0.0;
  meq[1] = fma(3.0, ru2, -2.0 * rho); S[1] = fma(6.0, uF, a.li_e * F2p);
  meq[2] = fma(-3.0, ru2, rho);   S[2] = -fma(6.0, uF, a.li_z * F2p);
  meq[3] = Jx;                    S[3] = Fx;
  meq[4] = -Jx;                   S[4] = -Fx;
  meq[5] = Jy;                    S[5] = Fy;
  meq[6] = -Jy;                   S[6] = -Fy;
  meq[7] = fma(ux, Jx, -uy * Jy); S[7] = 2.0 * fma(ux, Fx, -uy * Fy);
  meq[8] = ux * Jy;               S[8] = fma(ux, Fy, uy * Fx);
  if (ST) {
    const double k36 = 36.0 * sq.k;  // 1.5 tr Q = 36 k t
    meq[1] = fma(k36, sq.t, meq[1]);
    meq[2] = fma(-k36, sq.t, meq[2]);
    meq[7] = fma(-4.0 * sq.k, sq.sd, meq[7]);
    meq[8] = fma(-sq.k, sq.xd, meq[8]);
  }
  double n[9];
  const double inv_norm[9] = {1.0 / 9.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 6.0, 1.0 / 12.0,
                              1.0 / 6.0, 1.0 / 12.0, 1.0 / 4.0,  1.0 / 4.0};
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const double om = a.omega[k];
    const double ms = fma(fma(-0.5, om, 1.0), S[k], fma(-om, m[k] - meq[k], m[k]));
    n[k] = ms * inv_norm[k];
  }
  // f* = M^T n (M^-1 = M^T diag(1/|row|^2))
  out.f[0] = n[0] - 4.0 * n[1] + 4.0 * n[2];
  const double A = n[0] - n[1] - 2.0 * n[2];
  const double X = n[3] - 2.0 * n[4], Y = n[5] - 2.0 * n[6];
  out.f[1] = A + X + n[7];
  out.f[3] = A - X + n[7];
  out.f[2] = A + Y - n[7];
  out.f[4] = A - Y - n[7];
  const double B = n[0] + 2.0 * n[1] + n[2];
  const double Px = n[3] + n[4], Py = n[5] + n[6];
  const double bp = B + n[8], bm = B - n[8];
  out.f[5] = bp + (Px + Py);
  out.f[7] = bp - (Px + Py);
  out.f[6] = bm + (Py - Px);
  out.f[8] = bm - (Py - Px);
}

// K2 body for node (x, y), whose psi sits at sp[c] of a tile with row stride sw:
// force, collision (with the surface-tension source when ST), then push streaming
// (or the macroscopic fields when FIELDS, which the source does not change).
template <int KIND, bool FIELDS, bool ST = false>
__device__ __forceinline__ void collide_node(const StepArgs& a, int x, int y, const double* sp, int c, int sw,
                                             double* rho_o, double* ux_o, double* uy_o, double* psi_o) {
  const double p0 = sp[c];
  const double pE = sp[c + 1], pW = sp[c - 1], pN = sp[c + sw], pS = sp[c - sw];
  const double pNE = sp[c + sw + 1], pNW = sp[c + sw - 1], pSW = sp[c - sw - 1], pSE = sp[c - sw + 1];
  // 12 * sum_i w(|c_i|^2) psi(x + c_i) c_i  (w = 1/3 axis, 1/12 diagonal): exact
  // integer sums in one fixed-point frame, rounded once (fixsum.cuh); psi > 0 is
  // normal and finite wherever the density pass left the error word clear
  double gx, gy;
  fx::shan_chen_stencil(pE, pW, pN, pS, pNE, pNW, pSW, pSE, &gx, &gy);
  const int64_t N = a.n;
  const int64_t node = (int64_t)y * a.nx + x;
  Post o;
  double rho, ux, uy;
  SurfQ sq = {0.0, 0.0, 0.0, 0.0};
  if (ST && !FIELDS) sq = surface_q(a, p0, pE, pW, pN, pS, pNE, pNW, pSW, pSE);
  constexpr bool kST = ST && !FIELDS;
  if (KIND == kFullMrt) {
    collide_full<kST>(a, node, p0, gx, gy, sq, o, &rho, &ux, &uy);
  } else if (!FIELDS && (!kST || a.kappa_q == 0.0)) {
    // (a kernel built with the source runs lattices without it, kappa = 0, in a batch:
    // they take the same arithmetic as in the kernel without the source)
    rho = a.mom[node];
    collide_reduced_fx<KIND>(a, node, rho, a.mom[N + node], a.mom[2 * N + node], p0, gx, gy, o);
  } else {
    rho = a.mom[node];
    collide_reduced<KIND, kST>(a, node, rho, a.mom[N + node], a.mom[2 * N + node], p0, gx, gy, sq, o, &ux, &uy);
  }
  if (FIELDS) {
    if (rho_o) rho_o[node] = rho;
    if (ux_o) ux_o[node] = ux;
    if (uy_o) uy_o[node] = uy;
    if (psi_o) psi_o[node] = p0;
    return;
  }
  // push streaming: f_i(x + c_i, t + 1) = f*_i(x, t); bounce-back into the opposite
  // population of the same node when x + c_i lies in a wall
  double* __restrict__ out = a.f_out;
  const int nx = a.nx, ny = a.ny;
  const int xe = (x + 1 == nx) ? 0 : x + 1;
  const int xw = (x == 0) ? nx - 1 : x - 1;
  const int64_t row = (int64_t)y * nx;
  out[node] = o.f[0];
  out[N + row + xe] = o.f[1];
  out[3 * N + row + xw] = o.f[3];
  bool up_wall = false, down_wall = false;
  int yn = y + 1, ys = y - 1;
  if (a.walls) {
    up_wall = (yn == ny);
    down_wall = (ys < 0);
  } else {
    if (yn == ny) yn = 0;
    if (ys < 0) ys = ny - 1;
  }
  const int64_t rn = (int64_t)yn * nx, rs = (int64_t)ys * nx;
  if (up_wall) {
    out[4 * N + node] = o.f[2];
    out[7 * N + node] = o.f[5];
    out[8 * N + node] = o.f[6];
  } else {
    out[2 * N + rn + x] = o.f[2];
    out[5 * N + rn + xe] = o.f[5];
    out[6 * N + rn + xw] = o.f[6];
  }
  if (down_wall) {
    out[2 * N + node] = o.f[4];
    out[5 * N + node] = o.f[7];
    out[6 * N + node] = o.f[8];
  } else {
    out[4 * N + rs + x] = o.f[4];
    out[7 * N + rs + xw] = o.f[7];
    out[8 * N + rs + xe] = o.f[8];
  }
}

// ---- per-M-step guard (Sec. III.A convergence check, mass, stability) --------------

constexpr int kGuardQ = 4;  // mass, max |u|, bad-node count, sum |rho - rho'|

// psi at (x + dx, y + dy) for 0 <= x < nx, 0 <= y < ny, |dx|, |dy| <= 1
__device__ __forceinline__ double psi_near(const StepArgs& a, int x, int y, int dx, int dy) {
  const int gx = wrap_index(x + dx, a.nx);
  int gy = y + dy;
  if (a.walls) {
    if (gy < 0) return a.psi_ghost_bottom;
    if (gy >= a.ny) return a.psi_ghost_top;
  } else {
    gy = wrap_index(gy, a.ny);
  }
  return a.psi[(int64_t)gy * a.nx + gx];
}

// Guard terms of node i, read from the psi and moment planes a density pass has just
// written for the current state: adds rho to v[0], raises v[1] to |u| with
// u = (j + F/2)/rho the fluid velocity of Eq. Momentum (F of Eq. ShanChenForce, wall
// ghosts as in the collision pass), and, when snap_valid, adds |rho - rho'| to v[3]
// with rho' = snap[i] the density of the previous guard call (the numerator of the
// Sec. III.A criterion). A non-finite or non-positive density adds 1 to v[2] and
// nothing else. Refreshes snap[i] = rho. IEEE division and sqrt: not on the hot path.
__device__ __forceinline__ void guard_node(const StepArgs& a, int64_t i, double* snap, bool snap_valid,
                                           double v[kGuardQ]) {
  const int64_t n = a.n;
  const double rho = a.mom[i];
  if (!(rho > 0.0 && rho < 1e300)) {
    v[2] += 1.0;
  } else {
    const int y = (int)(i / a.nx), x = (int)(i - (int64_t)y * a.nx);
    // the collision pass's stencil sums (the same arithmetic, so the same force)
    double gx, gy;
    fx::shan_chen_stencil(psi_near(a, x, y, 1, 0), psi_near(a, x, y, -1, 0), psi_near(a, x, y, 0, 1),
                          psi_near(a, x, y, 0, -1), psi_near(a, x, y, 1, 1), psi_near(a, x, y, -1, 1),
                          psi_near(a, x, y, -1, -1), psi_near(a, x, y, 1, -1), &gx, &gy);
    const double cH = a.half_force * a.psi[i];
    const double ux = (a.mom[n + i] + cH * gx) / rho, uy = (a.mom[2 * n + i] + cH * gy) / rho;
    v[0] += rho;
    v[1] = fmax(v[1], sqrt(ux * ux + uy * uy));
    if (snap_valid) v[3] += fabs(rho - snap[i]);
  }
  snap[i] = rho;
}

// Fixed-order tree reduction of the guard terms over a block of `nthreads` (a power
// of two); s[q][0] holds the block's result.
template <int kNThreads>
__device__ __forceinline__ void guard_block_reduce(const double v[kGuardQ], double (*s)[kNThreads]) {
  for (int q = 0; q < kGuardQ; ++q) s[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int w = kNThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s[0][threadIdx.x] += s[0][threadIdx.x + w];
      s[1][threadIdx.x] = fmax(s[1][threadIdx.x], s[1][threadIdx.x + w]);
      s[2][threadIdx.x] += s[2][threadIdx.x + w];
      s[3][threadIdx.x] += s[3][threadIdx.x + w];
    }
    __syncthreads();
  }
}

}  // namespace pplbm
