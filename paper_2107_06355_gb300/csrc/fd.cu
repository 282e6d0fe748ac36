// Finite-difference (MacCormack) solver of the macroscopic equations the method
// recovers (App. A), periodic grids, FP64.
//
//   d_t rho = -(rho d_g u_g + u_g d_g rho)
//   d_t u_a = -u_g d_g u_a - d_a p_EOS / rho - d_b p'_ab / rho + d_b sigma'_ab / rho
// with sigma' of Eq. StressTensor expanded as Eq. FDstressTensor (mu = rho/3
// (tau_nu - 1/2), mu_B = rho/3 (tau_e - tau_nu), Eq. DynamicViscosity; gradients
// via dmu/drho, Eq. FDviscosityDerivative) and d_b p'_ab of Eq. FDforce
//   -eps (G/4)(d_g psi)(d_a d_g psi) + (G/12)(d_a psi) lap psi + (G/6)(d_g psi)(d_a d_g psi)
//   + (G/4) psi d_a lap psi          (c = 1),
// plus, with the surface-tension control of Sec. V's technique (kappa), the
// divergence of its second-order pressure tensor (kappa G/6) psi (delta lap psi -
// d_a d_b psi): (kappa G/6) [(d_a psi) lap psi - (d_g psi)(d_a d_g psi)], which only
// changes the coefficients of the first and third terms above.
// Predictor: first derivatives of rho, u, p_EOS and rho in the viscous terms are
// forward differences; corrector: backward; second derivatives central; every
// derivative of psi central (the third derivative through lap psi at +-1).
// One MacCormack step = EOS pass (psi, p of U) + predictor pass (U* = U + dt R_f(U))
// + EOS pass (of U*) + corrector pass (U <- (U + U* + dt R_b(U*)) / 2, in place:
// the corrector reads U only at its own node).
// x is periodic; y is periodic or bounded by the wall layers of the grid-dependency
// appendix (Eqs. B1, B2): every plane then carries two ghost rows below and above
// the fluid rows, which a boundary pass fills after each EOS pass.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "../../include/pplbm.h"
#include "eos_dev.cuh"
#include "fixsum.cuh"
#include "fp64.cuh"
#include "internal.h"

namespace pplbm {
namespace {

struct FDArgs {
  const double* rho;  // source state of the RHS (U for the predictor, U* for the corrector)
  const double* ux;
  const double* uy;
  const double* psi;  // psi(rho), p_EOS(rho) of the source state
  const double* p;
  const double* rho0;  // corrector: U^n
  const double* ux0;
  const double* uy0;
  double* orho;  // output state
  double* oux;
  double* ouy;
  int nx, ny;
  int walls;  // 1: planes hold ghost rows (fluid row y at row y + 2), y not periodic
  // Every derivative is formed from raw stencil differences; the powers of
  // h = 1/dx, the time step and the force and viscosity coefficients are folded
  // into these constants on the host (mu = mu_c rho, mu_B = muB_c rho):
  double cA;              // dt h: advection, mass flux, pressure gradient
  double kS, kL, kD;      // dt (h^3/2) (G/6 - eps G/4), dt (h^3/2) G/12, dt (h^3/2) G/4
  double v1, v2, v3, v4;  // dt h^2 mu_c, dt h^2 muB_c, dt h^2 (2 mu_c + muB_c), dt h^2 (mu_c + muB_c)/4
  // tau_nu(rho) = ta + tb rho (Eq. RelaxationTime) in the VV kernels: mu = dt h^2 rho (g0 + g1 rho),
  // mu_B = dt h^2 rho (e0 - g1 rho), and d/drho of both (Eq. FDviscosityDerivative)
  double g0, g1, e0;
};

__global__ void k_fd_eos(const EosConst e, const double* __restrict__ rho, double* __restrict__ psi,
                         double* __restrict__ p, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double r = rho[i];
  const double pr = eos_pressure(e, r);
  p[i] = pr;
  const double psi2 = e.psi2_scale * (pr - r * (1.0 / 3.0));
  psi[i] = psi2 > 0.0 ? fast_sqrt(psi2) : sqrt(psi2);  // IEEE result at 0, below 0 and NaN
}

// Wall layers (Eqs. B1, B2), one thread per column of a padded plane set: b1 (row
// 1) on the bottom wall, no slip, density and psi extrapolated from the first two
// fluid rows, p of that density; b2 (row 0) in the solid, psi_b2 = psi_b1 + 2 dy
// (psi_l - psi_b1); top rows mirror the last fluid rows with the velocity
// reversed (reflexive layers t1 = row ny + 2, t2 = row ny + 3).
__global__ void k_fd_walls(const EosConst e, double* rho, double* ux, double* uy, double* psi, double* p, int nx,
                           int ny, double two_dy, double psi_l) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= nx) return;
  auto at = [&](int row) { return (int64_t)row * nx + x; };
  const double rb1 = 2.0 * rho[at(2)] - rho[at(3)];
  const double sb1 = 2.0 * psi[at(2)] - psi[at(3)];
  const double pb1 = eos_pressure(e, rb1);
  rho[at(1)] = rb1;
  psi[at(1)] = sb1;
  p[at(1)] = pb1;
  ux[at(1)] = 0.0;
  uy[at(1)] = 0.0;
  rho[at(0)] = rb1;
  psi[at(0)] = fma(two_dy, psi_l - sb1, sb1);
  p[at(0)] = pb1;
  ux[at(0)] = 0.0;
  uy[at(0)] = 0.0;
  const int t1 = ny + 2, t2 = ny + 3, f1 = ny + 1, f2 = ny;
  rho[at(t1)] = rho[at(f1)];
  psi[at(t1)] = psi[at(f1)];
  p[at(t1)] = p[at(f1)];
  ux[at(t1)] = -ux[at(f1)];
  uy[at(t1)] = -uy[at(f1)];
  rho[at(t2)] = rho[at(f2)];
  psi[at(t2)] = psi[at(f2)];
  p[at(t2)] = p[at(f2)];
  ux[at(t2)] = 0.0;
  uy[at(t2)] = 0.0;
}

// Stencil differences as exact integer combinations in one fixed-point frame per
// field (fixsum.cuh), each rounded once: integer-pipe work in place of chains of
// software IEEE additions and FP64 fused multiply-adds.
using fx::u64;

// psi's raw differences at a point from the 13 values of its 5 x 5 cross and
// diagonals: central first differences Pd, second differences Pxx, Pyy, the mixed
// one q = Dxy / 4, the Laplacian Lc = Pxx + Pyy and the differences DL of the
// 5-point Laplacians at +-1 (their coefficients sum to 14 at most: headroom 5 + sign).
// A value out of the frames' range (non-finite, or at or above 2^1008) makes them all
// NaN.
struct PsiDiffs {
  double Pd0, Pd1, Pxx, Pyy, q, Lc, DL0, DL1;
};

__device__ __forceinline__ PsiDiffs psi_diffs(double c, double e, double w, double n, double s, double ne, double nw,
                                              double sw, double se, double ee, double ww, double nn, double ss) {
  const double v[13] = {c, e, w, n, s, ne, nw, sw, se, ee, ww, nn, ss};
  u64 b[13];
  unsigned mx = 0;
#pragma unroll
  for (int k = 0; k < 13; ++k) {
    b[k] = fx::bits_of(v[k]);
    mx = max(mx, fx::mag_hi(b[k]));
  }
  const int eg = (int)(mx >> 20) + 6;
  u64 t[13];
#pragma unroll
  for (int k = 0; k < 13; ++k) t[k] = (u64)fx::sterm(b[k], eg);
  const u64 tC = t[0], tE = t[1], tW = t[2], tN = t[3], tS = t[4], tNE = t[5], tNW = t[6], tSW = t[7], tSE = t[8];
  const u64 pd0 = tE - tW, pd1 = tN - tS;
  const u64 pxx = tE + tW - 2 * tC, pyy = tN + tS - 2 * tC;
  const u64 dxy = (tNE - tSE) - (tNW - tSW);
  const u64 dl0 = (t[9] - t[10]) + (tNE + tSE) - (tNW + tSW) - 4 * pd0;  // L5(1, 0) - L5(-1, 0)
  const u64 dl1 = (t[11] - t[12]) + (tNE + tNW) - (tSE + tSW) - 4 * pd1;  // L5(0, 1) - L5(0, -1)
  const bool bad = mx >= fx::kFrameMaxHi;
  auto out = [&](u64 x, int shift) {
    return fx::double_of(bad ? fx::kNaN : fx::round_frame_s((fx::i64)x, eg + shift));
  };
  PsiDiffs r;
  r.Pd0 = out(pd0, 0);
  r.Pd1 = out(pd1, 0);
  r.Pxx = out(pxx, 0);
  r.Pyy = out(pyy, 0);
  r.q = out(dxy, -2);
  r.Lc = out(pxx + pyy, 0);
  r.DL0 = out(dl0, 0);
  r.DL1 = out(dl1, 0);
  return r;
}

// a velocity component's raw differences from its 3 x 3 neighbourhood: the one-sided
// first differences along x and y (forward in the predictor, backward in the
// corrector) and the central Dxx, Dyy, Dxy (coefficients sum to 4: headroom 3 + sign)
struct VelDiffs {
  double D0, D1, xx, yy, xy;
};

template <bool PRED>
__device__ __forceinline__ VelDiffs vel_diffs(double c, double e, double w, double n, double s, double ne, double nw,
                                              double sw, double se) {
  const double v[9] = {c, e, w, n, s, ne, nw, sw, se};
  u64 b[9];
  unsigned mx = 0;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    b[k] = fx::bits_of(v[k]);
    mx = max(mx, fx::mag_hi(b[k]));
  }
  const int eg = (int)(mx >> 20) + 4;
  u64 t[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) t[k] = (u64)fx::sterm(b[k], eg);
  const u64 tC = t[0], tE = t[1], tW = t[2], tN = t[3], tS = t[4];
  const bool bad = mx >= fx::kFrameMaxHi;
  auto out = [&](u64 x) { return fx::double_of(bad ? fx::kNaN : fx::round_frame_s((fx::i64)x, eg)); };
  VelDiffs r;
  r.D0 = out(PRED ? tE - tC : tC - tW);
  r.D1 = out(PRED ? tN - tC : tC - tS);
  r.xx = out(tE + tW - 2 * tC);
  r.yy = out(tN + tS - 2 * tC);
  r.xy = out((t[5] - t[8]) - (t[6] - t[7]));
  return r;
}

// PRED: predictor (forward differences) or corrector (backward); VV: tau_nu(rho)
// viscosities, a compile-time choice so the constant-viscosity kernel carries none
// of their arithmetic
// 3 resident blocks per SM (80 registers, 16-36 bytes spilled): the two arithmetic pipes
// issue 10 % faster than at 2 blocks and 89-94 registers
template <bool PRED, bool VV>
__global__ void __launch_bounds__(256, 3) k_fd_update(const FDArgs a) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 8 + threadIdx.y;
  if (x >= a.nx || y >= a.ny) return;
  const int nx = a.nx, ny = a.ny;
  // periodic columns and row offsets of the 5 x 5 neighbourhood, wrapped once
  // (offsets reach +-2, so a grid of width 1 or 2 wraps twice)
  auto wrap = [](int v, int n) {
    if (v < 0) v += n;
    if (v < 0) v += n;
    if (v >= n) v -= n;
    if (v >= n) v -= n;
    return v;
  };
  int cx[5];
  int64_t ry[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    cx[k] = wrap(x + k - 2, nx);
    ry[k] = (int64_t)(a.walls ? y + k : wrap(y + k - 2, ny)) * nx;  // walls: padded rows, no wrap
  }
  auto at = [&](const double* f, int dx, int dy) { return f[ry[dy + 2] + cx[dx + 2]]; };
  // one-sided first difference along x (axis 0) or y (axis 1) of rho and p: forward in
  // the predictor, backward in the corrector; true derivative = h D (integer pipe,
  // add_int: bitwise the FP64 add)
  auto D1 = [&](const double* f, int axis) {
    const double c = at(f, 0, 0);
    if (PRED) return axis == 0 ? sub_int(at(f, 1, 0), c) : sub_int(at(f, 0, 1), c);
    return axis == 0 ? sub_int(c, at(f, -1, 0)) : sub_int(c, at(f, 0, -1));
  };
  auto vel = [&](const double* f) {
    return vel_diffs<PRED>(at(f, 0, 0), at(f, 1, 0), at(f, -1, 0), at(f, 0, 1), at(f, 0, -1), at(f, 1, 1),
                           at(f, -1, 1), at(f, -1, -1), at(f, 1, -1));
  };
  const double rho = at(a.rho, 0, 0), ux = at(a.ux, 0, 0), uy = at(a.uy, 0, 0);
  // velocity differences: Du_ab = d_a u_b (one-sided), second differences central
  // (d_xx = h^2 Dxx, d_xy = (h^2/4) Dxy)
  const VelDiffs vx = vel(a.ux), vy = vel(a.uy);
  const double Du00 = vx.D0, Du01 = vy.D0, Du10 = vx.D1, Du11 = vy.D1;
  // mass: d_t rho = -(rho div u + u . grad rho)
  const double Dr0 = D1(a.rho, 0), Dr1 = D1(a.rho, 1);
  const double Dv = add_int(Du00, Du11), Sh = add_int(Du01, Du10);
  const double drho = -a.cA * fma(rho, Dv, fma(ux, Dr0, uy * Dr1));
  // psi: dpsi = (h/2) Pd, d_ab psi from Pxx, Pyy, q = Dxy/4, lap = h^2 Lc, and the
  // derivative of lap psi = (h^3/2) DL from the 5-point sums at +-1
  const double* ps = a.psi;
  const double psi = at(ps, 0, 0);
  const PsiDiffs pd = psi_diffs(psi, at(ps, 1, 0), at(ps, -1, 0), at(ps, 0, 1), at(ps, 0, -1), at(ps, 1, 1),
                                at(ps, -1, 1), at(ps, -1, -1), at(ps, 1, -1), at(ps, 2, 0), at(ps, -2, 0),
                                at(ps, 0, 2), at(ps, 0, -2));
  const double Pd0 = pd.Pd0, Pd1 = pd.Pd1, Pxx = pd.Pxx, Pyy = pd.Pyy, q = pd.q, Lc = pd.Lc;
  const double DL0 = pd.DL0, DL1 = pd.DL1;
  // d_b p'_ab (Eq. FDforce) = (h^3/2) [(G/6 - eps G/4) S_a + (G/12) Pd_a Lc + (G/4) psi DL_a],
  // S_a = sum_g Pd_g (d_a d_g psi in the same units)
  const double S0 = fma(Pd0, Pxx, q * Pd1), S1 = fma(Pd1, Pyy, q * Pd0);
  const double kDpsi = a.kD * psi;
  const double F0 = fma(a.kS, S0, fma(a.kL * Pd0, Lc, kDpsi * DL0));
  const double F1 = fma(a.kS, S1, fma(a.kL * Pd1, Lc, kDpsi * DL1));
  // d_b sigma'_ab (Eqs. FDstressTensor, FDviscosityDerivative) with one-sided grad rho, grad u
  // and central second derivatives of u
  const double U0xx = vx.xx, U0yy = vx.yy, U1xx = vy.xx, U1yy = vy.yy;
  const double U0xy = vx.xy, U1xy = vy.xy;
  double V0, V1;
  if (!VV) {
    V0 = fma(a.v1, fma(2.0 * Dr0, Du00, Dr1 * Sh),
             fma(a.v2 * Dr0, Dv, rho * fma(a.v3, U0xx, fma(a.v4, U1xy, a.v1 * U0yy))));
    V1 = fma(a.v1, fma(2.0 * Dr1, Du11, Dr0 * Sh),
             fma(a.v2 * Dr1, Dv, rho * fma(a.v3, U1yy, fma(a.v4, U0xy, a.v1 * U1xx))));
  } else {
    const double mu = rho * fma(a.g1, rho, a.g0), muB = rho * fma(-a.g1, rho, a.e0);
    const double dmu = fma(2.0 * a.g1, rho, a.g0), dmuB = fma(-2.0 * a.g1, rho, a.e0);
    const double c2 = 2.0 * mu + muB, c4 = 0.25 * (mu + muB);
    V0 = fma(dmu, fma(2.0 * Dr0, Du00, Dr1 * Sh), fma(dmuB * Dr0, Dv, fma(c2, U0xx, fma(c4, U1xy, mu * U0yy))));
    V1 = fma(dmu, fma(2.0 * Dr1, Du11, Dr0 * Sh), fma(dmuB * Dr1, Dv, fma(c2, U1yy, fma(c4, U0xy, mu * U1xx))));
  }
  // dt d_t u_a = -dt u . grad u_a + (dt/rho)(d_b sigma'_ab - d_a p_EOS - d_b p'_ab)
  const double inv_rho = fast_rcp(rho);
  const double dux = fma(V0 - F0 - a.cA * D1(a.p, 0), inv_rho, -a.cA * fma(ux, Du00, uy * Du10));
  const double duy = fma(V1 - F1 - a.cA * D1(a.p, 1), inv_rho, -a.cA * fma(ux, Du01, uy * Du11));
  const int64_t i = (int64_t)(a.walls ? y + 2 : y) * nx + x;
  if (PRED) {
    a.orho[i] = rho + drho;
    a.oux[i] = ux + dux;
    a.ouy[i] = uy + duy;
  } else {
    a.orho[i] = 0.5 * (a.rho0[i] + (rho + drho));
    a.oux[i] = 0.5 * (a.ux0[i] + (ux + dux));
    a.ouy[i] = 0.5 * (a.uy0[i] + (uy + duy));
  }
}

}  // namespace
}  // namespace pplbm

using namespace pplbm;

struct pplbm_fd {
  int nx, ny;
  int64_t n;     // fluid nodes
  bool walls;
  int64_t np;    // values per plane: n, or nx (ny + 4) with walls
  int64_t off;   // first fluid value of a plane: 0, or 2 nx with walls
  EosConst eos;
  pplbm_eos_derived derived;
  double G, eps, dx, mu_c, muB_c, tau_e;
  double kappa;   // surface-tension control, 0 = off
  bool var_visc;  // tau_nu(rho) = ta + tb rho instead of a constant
  double ta, tb;
  double* U;   // rho, ux, uy
  double* S;   // predictor state
  double* psi;
  double* p;
  cudaStream_t stream;
  int64_t steps;
};

extern "C" {

namespace {
// 0: periodic y, 1: walls, -1: not accepted
int fd_walls(const pplbm_lattice* l) {
  if (l->bc == (PPLBM_BC_PERIODIC_X | PPLBM_BC_PERIODIC_Y)) return 0;
  if (l->bc == (PPLBM_BC_PERIODIC_X | PPLBM_BC_WALL_BOTTOM | PPLBM_BC_WALL_TOP) && l->ny >= 2) return 1;
  return -1;
}
}  // namespace

size_t pplbm_fd_workspace_bytes(const pplbm_lattice* lattice) {
  if (!lattice || lattice->nx < 1 || lattice->ny < 1 || lattice->ny > 65535 * 8) return 0;
  const int w = fd_walls(lattice);
  if (w < 0) return 0;
  return sizeof(double) * 8 * (size_t)lattice->nx * (size_t)(lattice->ny + 4 * w);
}

pplbm_status pplbm_fd_create(pplbm_fd** out, const pplbm_lattice* lattice, const pplbm_eos_params* eos, double G,
                             double tau_nu, double tau_e, double dx, void* workspace, size_t workspace_bytes,
                             void* stream) {
  if (!out) return PPLBM_ERR_ARG;
  *out = nullptr;
  if (!lattice || !eos || !workspace || lattice->nx < 1 || lattice->ny < 1 || lattice->reserved != 0) return PPLBM_ERR_ARG;
  if (lattice->ny > 65535 * 8) return PPLBM_ERR_ARG;  // the update pass's grid: 8-row tiles on its y axis
  if (fd_walls(lattice) < 0) return PPLBM_ERR_ARG;
  if (!(tau_nu > 0.5) || !(tau_e > 0.0) || !(dx > 0.0)) return PPLBM_ERR_ARG;
  if (workspace_bytes < pplbm_fd_workspace_bytes(lattice)) return PPLBM_ERR_ARG;
  pplbm_eos_derived d;
  const pplbm_status st = pplbm_eos_setup(eos, G, &d);
  if (st != PPLBM_OK) return st;
  pplbm_fd* f = new (std::nothrow) pplbm_fd();
  if (!f) return PPLBM_ERR_ARG;
  f->nx = lattice->nx;
  f->ny = lattice->ny;
  f->n = (int64_t)f->nx * f->ny;
  f->walls = fd_walls(lattice) == 1;
  f->np = (int64_t)f->nx * (f->ny + (f->walls ? 4 : 0));
  f->off = f->walls ? 2 * (int64_t)f->nx : 0;
  f->derived = d;
  f->eos = make_eos_const(d);
  f->G = G;
  f->eps = d.eps;
  f->dx = dx;
  f->mu_c = (tau_nu - 0.5) / 3.0;
  f->muB_c = (tau_e - tau_nu) / 3.0;
  f->tau_e = tau_e;
  f->kappa = 0.0;
  f->var_visc = false;
  double* w = (double*)workspace;
  f->U = w;
  f->S = w + 3 * f->np;
  f->psi = w + 6 * f->np;
  f->p = w + 7 * f->np;
  f->stream = (cudaStream_t)stream;
  *out = f;
  return PPLBM_OK;
}

pplbm_status pplbm_fd_set_state(pplbm_fd* f, const double* rho, const double* ux, const double* uy) {
  if (!f || !rho || !ux || !uy) return PPLBM_ERR_ARG;
  const double* src[3] = {rho, ux, uy};
  for (int k = 0; k < 3; ++k)
    if (cudaMemcpyAsync(f->U + k * f->np + f->off, src[k], sizeof(double) * f->n, cudaMemcpyDefault, f->stream) !=
        cudaSuccess)
      return PPLBM_ERR_CUDA;
  return cudaStreamSynchronize(f->stream) == cudaSuccess ? PPLBM_OK : PPLBM_ERR_CUDA;
}

pplbm_status pplbm_fd_get_state(pplbm_fd* f, double* rho, double* ux, double* uy) {
  if (!f) return PPLBM_ERR_ARG;
  double* dst[3] = {rho, ux, uy};
  for (int k = 0; k < 3; ++k)
    if (dst[k] &&
        cudaMemcpyAsync(dst[k], f->U + k * f->np + f->off, sizeof(double) * f->n, cudaMemcpyDefault, f->stream) !=
            cudaSuccess)
      return PPLBM_ERR_CUDA;
  return cudaStreamSynchronize(f->stream) == cudaSuccess ? PPLBM_OK : PPLBM_ERR_CUDA;
}

pplbm_status pplbm_fd_step(pplbm_fd* f, int64_t nsteps, double dt) {
  if (!f || nsteps < 0 || !(dt > 0.0)) return PPLBM_ERR_ARG;
  const unsigned eb = (unsigned)((f->n + 255) / 256);
  const dim3 grid((f->nx + 31) / 32, (f->ny + 7) / 8), block(32, 8);
  FDArgs a;
  std::memset(&a, 0, sizeof(a));
  a.nx = f->nx;
  a.ny = f->ny;
  a.walls = f->walls ? 1 : 0;
  const double h = 1.0 / f->dx, h2 = h * h, h3 = h2 * h;
  a.cA = dt * h;
  a.kS = dt * 0.5 * h3 * (f->G / 6.0 - f->eps * f->G / 4.0 - f->kappa * f->G / 6.0);
  a.kL = dt * 0.5 * h3 * (f->G / 12.0 + f->kappa * f->G / 6.0);
  a.kD = dt * 0.5 * h3 * (f->G / 4.0);
  a.v1 = dt * h2 * f->mu_c;
  a.v2 = dt * h2 * f->muB_c;
  a.v3 = dt * h2 * (2.0 * f->mu_c + f->muB_c);
  a.v4 = dt * h2 * (f->mu_c + f->muB_c) * 0.25;
  if (f->var_visc) {
    a.g0 = dt * h2 * (f->ta - 0.5) / 3.0;
    a.g1 = dt * h2 * f->tb / 3.0;
    a.e0 = dt * h2 * (f->tau_e - f->ta) / 3.0;
  }
  a.psi = f->psi;
  a.p = f->p;
  const int64_t n = f->n, np = f->np, off = f->off;
  const unsigned wb = (unsigned)((f->nx + 255) / 256);
  const double two_dy = 2.0 * f->dx, psi_l = f->derived.psi_l;
  // psi and p of the state in X, then its wall layers
  auto eos_pass = [&](double* X) {
    k_fd_eos<<<eb, 256, 0, f->stream>>>(f->eos, X + off, f->psi + off, f->p + off, n);
    if (f->walls)
      k_fd_walls<<<wb, 256, 0, f->stream>>>(f->eos, X, X + np, X + 2 * np, f->psi, f->p, f->nx, f->ny, two_dy,
                                           psi_l);
  };
  for (int64_t s = 0; s < nsteps; ++s) {
    // predictor: U* = U + dt R_f(U)
    eos_pass(f->U);
    a.rho = f->U;
    a.ux = f->U + np;
    a.uy = f->U + 2 * np;
    a.orho = f->S;
    a.oux = f->S + np;
    a.ouy = f->S + 2 * np;
    if (f->var_visc)
      k_fd_update<true, true><<<grid, block, 0, f->stream>>>(a);
    else
      k_fd_update<true, false><<<grid, block, 0, f->stream>>>(a);
    // corrector: U <- (U + U* + dt R_b(U*)) / 2
    eos_pass(f->S);
    a.rho = f->S;
    a.ux = f->S + np;
    a.uy = f->S + 2 * np;
    a.rho0 = f->U;
    a.ux0 = f->U + np;
    a.uy0 = f->U + 2 * np;
    a.orho = f->U;
    a.oux = f->U + np;
    a.ouy = f->U + 2 * np;
    if (f->var_visc)
      k_fd_update<false, true><<<grid, block, 0, f->stream>>>(a);
    else
      k_fd_update<false, false><<<grid, block, 0, f->stream>>>(a);
  }
  f->steps += nsteps;
  return cudaGetLastError() == cudaSuccess ? PPLBM_OK : PPLBM_ERR_CUDA;
}

pplbm_status pplbm_fd_set_two_phase_viscosity(pplbm_fd* f, double tau_l, double visc_ratio) {
  if (!f || !(tau_l > 0.5) || !(visc_ratio > 0.0)) return PPLBM_ERR_ARG;
  const double tau_v = 0.5 + visc_ratio * (tau_l - 0.5);
  const double rv = f->derived.rho_v, rl = f->derived.rho_l;
  f->tb = (tau_l - tau_v) / (rl - rv);
  f->ta = tau_l - f->tb * rl;
  f->var_visc = true;
  return PPLBM_OK;
}

pplbm_status pplbm_fd_set_surface_tension(pplbm_fd* f, double kappa) {
  if (!f || !std::isfinite(kappa) || !(kappa < 1.0)) return PPLBM_ERR_ARG;
  f->kappa = kappa;
  return PPLBM_OK;
}

pplbm_status pplbm_fd_sync(pplbm_fd* f) {
  if (!f) return PPLBM_ERR_ARG;
  return cudaStreamSynchronize(f->stream) == cudaSuccess ? PPLBM_OK : PPLBM_ERR_CUDA;
}

void pplbm_fd_destroy(pplbm_fd* f) { delete f; }

}  // extern "C"
