// Finite-difference (MacCormack) solver of the macroscopic equations the method
// recovers (App. A), periodic grids, FP64.
//
//   d_t rho = -(rho d_g u_g + u_g d_g rho)
//   d_t u_a = -u_g d_g u_a - d_a p_EOS / rho - d_b p'_ab / rho + d_b sigma'_ab / rho
// with sigma' of Eq. StressTensor expanded as Eq. FDstressTensor (mu = rho/3
// (tau_nu - 1/2), mu_B = rho/3 (tau_e - tau_nu), Eq. DynamicViscosity; gradients
// via dmu/drho, Eq. FDviscosityDerivative) and d_b p'_ab of Eq. FDforce
//   -eps (G/4)(d_g psi)(d_a d_g psi) + (G/12)(d_a psi) lap psi + (G/6)(d_g psi)(d_a d_g psi)
//   + (G/4) psi d_a lap psi          (c = 1).
// Predictor: first derivatives of rho, u, p_EOS and rho in the viscous terms are
// forward differences; corrector: backward; second derivatives central; every
// derivative of psi central (the third derivative through lap psi at +-1).
// One MacCormack step = EOS pass (psi, p of U) + predictor pass (U* = U + dt R_f(U))
// + EOS pass (of U*) + corrector pass (U <- (U + U* + dt R_b(U*)) / 2, in place:
// the corrector reads U only at its own node).
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <string>

#include "../../include/pplbm.h"
#include "eos_dev.cuh"
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
  double inv_dx, inv_dx2, dt;
  double G, eps;
  double mu_c, muB_c;  // mu = mu_c rho, mu_B = muB_c rho
};

__global__ void k_fd_eos(const EosConst e, const double* __restrict__ rho, double* __restrict__ psi,
                         double* __restrict__ p, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double r = rho[i];
  const double pr = eos_pressure(e, r);
  p[i] = pr;
  psi[i] = sqrt(e.psi2_scale * (pr - r * (1.0 / 3.0)));
}

template <bool PRED>
__global__ void __launch_bounds__(256) k_fd_update(const FDArgs a) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 8 + threadIdx.y;
  if (x >= a.nx || y >= a.ny) return;
  const int nx = a.nx, ny = a.ny;
  auto X = [&](int dx) { int v = x + dx; v %= nx; return v < 0 ? v + nx : v; };
  auto Y = [&](int dy) { int v = y + dy; v %= ny; return v < 0 ? v + ny : v; };
  auto at = [&](const double* f, int dx, int dy) { return f[(int64_t)Y(dy) * nx + X(dx)]; };
  const double h = a.inv_dx, h2 = a.inv_dx2;
  // one-sided first derivative along x (axis 0) or y (axis 1)
  auto d1 = [&](const double* f, int axis) {
    const double c = at(f, 0, 0);
    if (PRED) return (axis == 0 ? at(f, 1, 0) - c : at(f, 0, 1) - c) * h;
    return (axis == 0 ? c - at(f, -1, 0) : c - at(f, 0, -1)) * h;
  };
  auto dc = [&](const double* f, int axis, int ox, int oy) {  // central first derivative at (x+ox, y+oy)
    return (axis == 0 ? at(f, ox + 1, oy) - at(f, ox - 1, oy) : at(f, ox, oy + 1) - at(f, ox, oy - 1)) * (0.5 * h);
  };
  auto d2 = [&](const double* f, int ax1, int ax2, int ox, int oy) {  // central second derivatives
    if (ax1 == ax2) {
      if (ax1 == 0) return (at(f, ox + 1, oy) - 2.0 * at(f, ox, oy) + at(f, ox - 1, oy)) * h2;
      return (at(f, ox, oy + 1) - 2.0 * at(f, ox, oy) + at(f, ox, oy - 1)) * h2;
    }
    return (at(f, ox + 1, oy + 1) - at(f, ox + 1, oy - 1) - at(f, ox - 1, oy + 1) + at(f, ox - 1, oy - 1)) *
           (0.25 * h2);
  };
  const double rho = at(a.rho, 0, 0);
  const double u[2] = {at(a.ux, 0, 0), at(a.uy, 0, 0)};
  const double* uf[2] = {a.ux, a.uy};
  // mass
  const double drho_1[2] = {d1(a.rho, 0), d1(a.rho, 1)};
  double du[2][2];  // du[a][b] = d_a u_b (one-sided)
  for (int ax = 0; ax < 2; ++ax)
    for (int b = 0; b < 2; ++b) du[ax][b] = d1(uf[b], ax);
  const double div = du[0][0] + du[1][1];
  const double rhs_rho = -(rho * div + (u[0] * drho_1[0] + u[1] * drho_1[1]));
  // psi derivatives (central)
  const double psi = at(a.psi, 0, 0);
  const double dpsi[2] = {dc(a.psi, 0, 0, 0), dc(a.psi, 1, 0, 0)};
  double ddpsi[2][2];
  ddpsi[0][0] = d2(a.psi, 0, 0, 0, 0);
  ddpsi[1][1] = d2(a.psi, 1, 1, 0, 0);
  ddpsi[0][1] = ddpsi[1][0] = d2(a.psi, 0, 1, 0, 0);
  const double lap = ddpsi[0][0] + ddpsi[1][1];
  auto lap_at = [&](int ox, int oy) { return d2(a.psi, 0, 0, ox, oy) + d2(a.psi, 1, 1, ox, oy); };
  const double dlap[2] = {(lap_at(1, 0) - lap_at(-1, 0)) * (0.5 * h), (lap_at(0, 1) - lap_at(0, -1)) * (0.5 * h)};
  const double dp_1[2] = {d1(a.p, 0), d1(a.p, 1)};
  double out[2];
  for (int al = 0; al < 2; ++al) {
    const double adv = u[0] * du[0][al] + u[1] * du[1][al];
    const double s = dpsi[0] * ddpsi[al][0] + dpsi[1] * ddpsi[al][1];
    const double dpp = -a.eps * a.G * 0.25 * s + a.G * (1.0 / 12.0) * dpsi[al] * lap + a.G * (1.0 / 6.0) * s +
                       a.G * 0.25 * psi * dlap[al];
    double visc = 0.0;
    for (int b = 0; b < 2; ++b) visc += a.mu_c * drho_1[b] * (du[al][b] + du[b][al]);
    double lapu = 0.0;
    for (int b = 0; b < 2; ++b) lapu += d2(uf[b], al, b, 0, 0) + d2(uf[al], b, b, 0, 0);
    visc += a.mu_c * rho * lapu;
    visc += a.muB_c * drho_1[al] * div;
    double gdiv = 0.0;
    for (int b = 0; b < 2; ++b) gdiv += d2(uf[b], al, b, 0, 0);
    visc += a.muB_c * rho * gdiv;
    out[al] = -adv - dp_1[al] / rho - dpp / rho + visc / rho;
  }
  const int64_t i = (int64_t)y * nx + x;
  if (PRED) {
    a.orho[i] = rho + a.dt * rhs_rho;
    a.oux[i] = u[0] + a.dt * out[0];
    a.ouy[i] = u[1] + a.dt * out[1];
  } else {
    a.orho[i] = 0.5 * (a.rho0[i] + rho + a.dt * rhs_rho);
    a.oux[i] = 0.5 * (a.ux0[i] + u[0] + a.dt * out[0]);
    a.ouy[i] = 0.5 * (a.uy0[i] + u[1] + a.dt * out[1]);
  }
}

}  // namespace
}  // namespace pplbm

using namespace pplbm;

struct pplbm_fd {
  int nx, ny;
  int64_t n;
  EosConst eos;
  pplbm_eos_derived derived;
  double G, eps, dx, mu_c, muB_c;
  double* U;   // rho, ux, uy
  double* S;   // predictor state
  double* psi;
  double* p;
  cudaStream_t stream;
  int64_t steps;
};

extern "C" {

size_t pplbm_fd_workspace_bytes(const pplbm_lattice* lattice) {
  if (!lattice || lattice->nx < 1 || lattice->ny < 1) return 0;
  return sizeof(double) * 8 * (size_t)lattice->nx * lattice->ny;
}

pplbm_status pplbm_fd_create(pplbm_fd** out, const pplbm_lattice* lattice, const pplbm_eos_params* eos, double G,
                             double tau_nu, double tau_e, double dx, void* workspace, size_t workspace_bytes,
                             void* stream) {
  if (!out) return PPLBM_ERR_ARG;
  *out = nullptr;
  if (!lattice || !eos || !workspace || lattice->nx < 1 || lattice->ny < 1 || lattice->reserved != 0) return PPLBM_ERR_ARG;
  if (lattice->bc != (PPLBM_BC_PERIODIC_X | PPLBM_BC_PERIODIC_Y)) return PPLBM_ERR_ARG;
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
  f->derived = d;
  f->eos = make_eos_const(d);
  f->G = G;
  f->eps = d.eps;
  f->dx = dx;
  f->mu_c = (tau_nu - 0.5) / 3.0;
  f->muB_c = (tau_e - tau_nu) / 3.0;
  double* w = (double*)workspace;
  f->U = w;
  f->S = w + 3 * f->n;
  f->psi = w + 6 * f->n;
  f->p = w + 7 * f->n;
  f->stream = (cudaStream_t)stream;
  *out = f;
  return PPLBM_OK;
}

pplbm_status pplbm_fd_set_state(pplbm_fd* f, const double* rho, const double* ux, const double* uy) {
  if (!f || !rho || !ux || !uy) return PPLBM_ERR_ARG;
  const double* src[3] = {rho, ux, uy};
  for (int k = 0; k < 3; ++k)
    if (cudaMemcpyAsync(f->U + k * f->n, src[k], sizeof(double) * f->n, cudaMemcpyDefault, f->stream) != cudaSuccess)
      return PPLBM_ERR_CUDA;
  return cudaStreamSynchronize(f->stream) == cudaSuccess ? PPLBM_OK : PPLBM_ERR_CUDA;
}

pplbm_status pplbm_fd_get_state(pplbm_fd* f, double* rho, double* ux, double* uy) {
  if (!f) return PPLBM_ERR_ARG;
  double* dst[3] = {rho, ux, uy};
  for (int k = 0; k < 3; ++k)
    if (dst[k] &&
        cudaMemcpyAsync(dst[k], f->U + k * f->n, sizeof(double) * f->n, cudaMemcpyDefault, f->stream) != cudaSuccess)
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
  a.inv_dx = 1.0 / f->dx;
  a.inv_dx2 = a.inv_dx * a.inv_dx;
  a.dt = dt;
  a.G = f->G;
  a.eps = f->eps;
  a.mu_c = f->mu_c;
  a.muB_c = f->muB_c;
  a.psi = f->psi;
  a.p = f->p;
  const int64_t n = f->n;
  for (int64_t s = 0; s < nsteps; ++s) {
    // predictor: U* = U + dt R_f(U)
    k_fd_eos<<<eb, 256, 0, f->stream>>>(f->eos, f->U, f->psi, f->p, n);
    a.rho = f->U;
    a.ux = f->U + n;
    a.uy = f->U + 2 * n;
    a.orho = f->S;
    a.oux = f->S + n;
    a.ouy = f->S + 2 * n;
    k_fd_update<true><<<grid, block, 0, f->stream>>>(a);
    // corrector: U <- (U + U* + dt R_b(U*)) / 2
    k_fd_eos<<<eb, 256, 0, f->stream>>>(f->eos, f->S, f->psi, f->p, n);
    a.rho = f->S;
    a.ux = f->S + n;
    a.uy = f->S + 2 * n;
    a.rho0 = f->U;
    a.ux0 = f->U + n;
    a.uy0 = f->U + 2 * n;
    a.orho = f->U;
    a.oux = f->U + n;
    a.ouy = f->U + 2 * n;
    k_fd_update<false><<<grid, block, 0, f->stream>>>(a);
  }
  f->steps += nsteps;
  return cudaGetLastError() == cudaSuccess ? PPLBM_OK : PPLBM_ERR_CUDA;
}

pplbm_status pplbm_fd_sync(pplbm_fd* f) {
  if (!f) return PPLBM_ERR_ARG;
  return cudaStreamSynchronize(f->stream) == cudaSuccess ? PPLBM_OK : PPLBM_ERR_CUDA;
}

void pplbm_fd_destroy(pplbm_fd* f) { delete f; }

}  // extern "C"
