// The two step kernels of the pseudopotential D2Q9 lattice Boltzmann method for
// one lattice, and their helpers (sm_103a, FP64). The per-node arithmetic is in
// step_device.cuh.
//
// K1 rho_psi : reads the 9 pre-collision populations of a node (coalesced SoA),
//              forms the moments the collision needs (rho = sum f, Eq. Density;
//              j = sum f c; plus the stress moments when they relax), evaluates the
//              equation of state and psi (Eq. InteractionPotential), writes psi and
//              the moments.
// K2 collide : stages a (32+2) x (8+2) psi tile in shared memory (periodic wrap in
//              x, periodic or wall ghost rows in y), computes the Shan-Chen force
//              (Eq. ShanChenForce), the velocity with the F/2 shift (Eq. Momentum),
//              the MRT collision with the Li source (Eqs. OperatorMRT, LiFS,
//              GFS), optionally the surface-tension source of Sec. V's
//              technique, and pushes f* to the neighbours (streaming, Eq. LBE),
//              with half-way bounce-back at walls (Sec. IV).
#include <cuda_runtime.h>

#include "step_device.cuh"

namespace pplbm {

namespace {

constexpr int kTX = 32;  // K2 tile width (one warp along x)
constexpr int kTY = 8;   // K2 tile height

template <int KIND>
__global__ void __launch_bounds__(256) k_rho_psi(const StepArgs a) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  rho_psi_node<KIND>(a, a.f_in, i);
}

// 5 resident blocks per SM (48 registers, 8-16 bytes spilled) except the two-phase
// kernel with the surface-tension source, which would spill 60 bytes: the
// integer-bound pass issues faster with the extra warps
constexpr int collide_blocks(int kind, bool st) { return (st && kind == kShearTau) ? 4 : 5; }

template <int KIND, bool FIELDS, bool ST = false>
__global__ void __launch_bounds__(kTX* kTY, collide_blocks(KIND, ST)) k_collide(const StepArgs a, double* rho_o, double* ux_o, double* uy_o,
                                                      double* psi_o) {
  __shared__ double sp[(kTY + 2) * (kTX + 2)];
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  load_psi_tile(a, sp, x0, y0, kTX, kTY, threadIdx.x, threadIdx.y, threadIdx.y * kTX + threadIdx.x, kTX * kTY);
  __syncthreads();
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
  if (x >= a.nx || y >= a.ny) return;
  collide_node<KIND, FIELDS, ST>(a, x, y, sp, (threadIdx.y + 1) * (kTX + 2) + threadIdx.x + 1, kTX + 2, rho_o, ux_o,
                                 uy_o, psi_o);
}

// f_i = f_i^eq(rho0, u0), Eq. EquilibriumDistribution (c_s^2 = 1/3)
__global__ void k_init_eq(int64_t n, double* f, const double* rho0, const double* ux0, const double* uy0,
                          int* err) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double rho = rho0[i];
  const double ux = ux0 ? ux0[i] : 0.0, uy = uy0 ? uy0[i] : 0.0;
  if (!(rho > 0.0 && rho < 1e300)) atomicOr(err, 1);
  const double uu = ux * ux + uy * uy;
  const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  const double w[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const double cu = cx[k] * ux + cy[k] * uy;
    f[k * n + i] = w[k] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
  }
}

// guard: a density pass over the current state, then per-block partials of the
// guard terms (guard_node) over a fixed grid-stride partition, then one block
// reduces them in a fixed order: deterministic
constexpr int kGuardBlocks = 304;
constexpr int kGuardThreads = 256;

__global__ void __launch_bounds__(kGuardThreads) k_guard_partial(const StepArgs a, double* snap, int snap_valid,
                                                                 double* partials) {
  __shared__ double s[kGuardQ][kGuardThreads];
  double v[kGuardQ] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)kGuardThreads + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * kGuardThreads)
    guard_node(a, i, snap, snap_valid != 0, v);
  guard_block_reduce<kGuardThreads>(v, s);
  if (threadIdx.x < kGuardQ) partials[kGuardQ * blockIdx.x + threadIdx.x] = s[threadIdx.x][0];
}

__global__ void __launch_bounds__(kGuardThreads) k_guard_final(const double* partials, int nblocks, int snap_valid,
                                                               double* out) {
  __shared__ double s[kGuardQ][kGuardThreads];
  double v[kGuardQ] = {0.0, 0.0, 0.0, 0.0};
  for (int k = threadIdx.x; k < nblocks; k += kGuardThreads) {
    v[0] += partials[kGuardQ * k];
    v[1] = fmax(v[1], partials[kGuardQ * k + 1]);
    v[2] += partials[kGuardQ * k + 2];
    v[3] += partials[kGuardQ * k + 3];
  }
  guard_block_reduce<kGuardThreads>(v, s);
  if (threadIdx.x == 0) {
    out[0] = s[0][0];
    out[1] = s[1][0];
    out[2] = s[2][0];
    out[3] = snap_valid ? s[3][0] / s[0][0] : -1.0;
  }
}

dim3 collide_grid(const StepArgs& a) { return dim3((a.nx + kTX - 1) / kTX, (a.ny + kTY - 1) / kTY); }

}  // namespace

void launch_rho_psi(const StepArgs& a, void* stream) {
  const unsigned blocks = (unsigned)((a.n + 255) / 256);
  cudaStream_t s = (cudaStream_t)stream;
  switch (a.kind) {
    case kUnitTau: k_rho_psi<kUnitTau><<<blocks, 256, 0, s>>>(a); break;
    case kShearTau: k_rho_psi<kShearTau><<<blocks, 256, 0, s>>>(a); break;
    default: k_rho_psi<kFullMrt><<<blocks, 256, 0, s>>>(a); break;
  }
}

void launch_collide(const StepArgs& a, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const dim3 block(kTX, kTY);
  if (a.kappa_q != 0.0) {  // with the surface-tension source
    switch (a.kind) {
      case kUnitTau: k_collide<kUnitTau, false, true><<<collide_grid(a), block, 0, s>>>(a, 0, 0, 0, 0); break;
      case kShearTau: k_collide<kShearTau, false, true><<<collide_grid(a), block, 0, s>>>(a, 0, 0, 0, 0); break;
      default: k_collide<kFullMrt, false, true><<<collide_grid(a), block, 0, s>>>(a, 0, 0, 0, 0); break;
    }
    return;
  }
  switch (a.kind) {
    case kUnitTau: k_collide<kUnitTau, false><<<collide_grid(a), block, 0, s>>>(a, 0, 0, 0, 0); break;
    case kShearTau: k_collide<kShearTau, false><<<collide_grid(a), block, 0, s>>>(a, 0, 0, 0, 0); break;
    default: k_collide<kFullMrt, false><<<collide_grid(a), block, 0, s>>>(a, 0, 0, 0, 0); break;
  }
}

void launch_fields(const StepArgs& a, double* rho, double* ux, double* uy, double* psi_out, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const dim3 block(kTX, kTY);
  switch (a.kind) {
    case kUnitTau: k_collide<kUnitTau, true><<<collide_grid(a), block, 0, s>>>(a, rho, ux, uy, psi_out); break;
    case kShearTau: k_collide<kShearTau, true><<<collide_grid(a), block, 0, s>>>(a, rho, ux, uy, psi_out); break;
    default: k_collide<kFullMrt, true><<<collide_grid(a), block, 0, s>>>(a, rho, ux, uy, psi_out); break;
  }
}

void launch_init_eq(const StepArgs& a, double* f, const double* rho0, const double* ux0, const double* uy0,
                    void* stream) {
  const unsigned blocks = (unsigned)((a.n + 255) / 256);
  k_init_eq<<<blocks, 256, 0, (cudaStream_t)stream>>>(a.n, f, rho0, ux0, uy0, a.err);
}

int guard_blocks() { return kGuardBlocks; }

void launch_guard(const StepArgs& a, double* snap, int snap_valid, double* partials, double* out, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  launch_rho_psi(a, stream);
  k_guard_partial<<<kGuardBlocks, kGuardThreads, 0, s>>>(a, snap, snap_valid, partials);
  k_guard_final<<<1, kGuardThreads, 0, s>>>(partials, kGuardBlocks, snap_valid, out);
}

}  // namespace pplbm
