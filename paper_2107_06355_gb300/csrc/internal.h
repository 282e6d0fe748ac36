// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cstddef>
#include <cstdint>

#include "../../include/pplbm.h"
#include "eos.cuh"

namespace pplbm {

EosConst make_eos_const(const pplbm_eos_derived& d);

// Collision variants, chosen on the host from the relaxation set.
enum CollideKind : int {
  kUnitTau = 0,   // every relaxation time 1 (Lambda = I)
  kShearTau = 1,  // Lambda = diag(1,...,1, omega_nu, omega_nu), omega_nu constant or from tau(rho)
  kFullMrt = 2    // six independent relaxation times
};

// Number of moment planes K1 hands to K2 for each collision kind.
inline int moment_planes(int kind) { return kind == kUnitTau ? 3 : (kind == kShearTau ? 5 : 9); }

// Arguments of one lattice's step kernels (passed by value).
struct StepArgs {
  const double* f_in;   // 9 planes, pre-collision f(t)
  double* f_out;        // 9 planes, f(t+1)
  double* psi;          // 1 plane
  double* mom;          // moment planes (3, 5 or 9)
  int* err;             // sticky error word
  int nx, ny;
  int64_t n;            // nx * ny
  int walls;            // 1: bounce-back walls at y = -1/2 and y = ny - 1/2; 0: periodic y
  int kind;             // CollideKind
  EosConst eos;
  double G;
  double half_force;    // -G / 24: F/2 = half_force * psi(x) * g, g = 12 sum_i w_i psi(x + c_i) c_i
  double psi_ghost_bottom, psi_ghost_top;
  // kShearTau: omega = 1/tau with tau = tau_a + tau_b * rho (Eq. RelaxationTime); constant if tau_b == 0
  double tau_a, tau_b;
  // Li forcing, scaled: sigma * G^2 / (432 tau_e) (kUnitTau / kShearTau, tau_e = tau_zeta = 1)
  double zz_scale;
  // kFullMrt: relaxation rates for the 9 moments and the Li sigma terms 12 sigma/(tau - 1/2)
  double omega[9];
  double li_e, li_z;
  // surface-tension control: kappa G / 24, so Q = kappa_q psi(x) q with
  // q = 12 sum_i w_i [psi(x + c_i) - psi(x)] c_i c_i; 0 when off
  double kappa_q;
};

// Collision kind of a relaxation set (kUnitTau, kShearTau, kFullMrt), -1 if the set
// is invalid (reserved word, forcing, kappa finite and < 1, relaxation times > 1/2)
// (collision_args.cpp).
int collision_kind(const pplbm_relax* r);
// The collision fields of a (tau_a, tau_b, zz_scale, kappa_q, omega, li_e, li_z) for
// the relaxation set r of collision kind `kind`, the EOS d and the interaction G.
void set_collision_args(StepArgs& a, int kind, const pplbm_relax& r, const pplbm_eos_derived& d, double G);

// Launchers (step_kernels.cu); all asynchronous on `stream`.
void launch_rho_psi(const StepArgs& a, void* stream);
void launch_collide(const StepArgs& a, void* stream);
void launch_fields(const StepArgs& a, double* rho, double* ux, double* uy, double* psi_out, void* stream);
void launch_init_eq(const StepArgs& a, double* f, const double* rho0, const double* ux0, const double* uy0,
                    void* stream);
// Guard of the state a.f_in: a density pass (psi and the moment planes), then a
// deterministic reduction of the guard terms (step_device.cuh, guard_node) into
// out[kGuardQ]: mass, max |u|, bad-node count, residual against the density in snap
// (-1 unless snap_valid); snap is refreshed. partials has room for
// guard_blocks() * kGuardQ doubles.
int guard_blocks();
void launch_guard(const StepArgs& a, double* snap, int snap_valid, double* partials, double* out, void* stream);

}  // namespace pplbm
