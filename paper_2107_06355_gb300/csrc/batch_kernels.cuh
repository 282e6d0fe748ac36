// Device code of the batched engine (batch.cu): the per-instance argument table, the
// work-item kernels of the two passes, the persistent kernel with its bounded grid
// barrier, the per-instance guard, and their launchers. The per-node arithmetic is
// step_device.cuh's, shared with the single-lattice kernels.
#pragma once

#include <cuda_runtime.h>

#include "step_device.cuh"

namespace pplbm {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxTileSmem = (256 + 2) * (1 + 2);  // largest (tw + 2)(th + 2) over tw*th = 256
constexpr unsigned kSpinLimit = 1u << 24;           // x ~100 ns sleeps: ~1.7 s per barrier wait
constexpr int kErrTimeout = 2;  // batch error word; divergence is flagged per instance

struct BatchInst {
  StepArgs a[2];  // a[p] reads f from buffer p and writes buffer 1 - p
  double* snap;   // density at the previous guard call (one plane)
  int tw, th, log2tw, tiles_x;
  int k1_start, k2_start;
};

struct GridBarrier {
  unsigned int count;
  unsigned int generation;
};

// Bounded grid-wide barrier for a cooperative launch; false if a wait gave up.
__device__ bool grid_barrier(GridBarrier* b, int* err, unsigned spin_limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = &b->generation;
    const unsigned int g = *gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&b->count, 1u) + 1u;
    if (arrived == gridDim.x) {
      b->count = 0u;
      __threadfence();
      atomicAdd(&b->generation, 1u);
    } else {
      unsigned int it = 0;
      while (*gen == g) {
        if (++it > spin_limit) {
          atomicOr(err, kErrTimeout);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return (*(volatile int*)err & kErrTimeout) == 0;
}

// Copies instance id's StepArgs for `parity` into shared memory (uniform across
// the block, so every later field read is a shared-memory broadcast).
__device__ __forceinline__ void stage_args(const BatchInst* __restrict__ inst, int id, int parity, StepArgs* sa) {
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&inst[id].a[parity]);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(sa);
  for (int k = threadIdx.x; k < (int)(sizeof(StepArgs) / 8); k += blockDim.x) dst[k] = src[k];
  __syncthreads();
}

// density/psi pass over block `local` (256 nodes) of instance id; REUSE: the block
// takes another item afterwards (persistent kernel), so it waits until every thread is
// done with the shared arguments
template <int KIND, bool REUSE>
__device__ __forceinline__ void batch_rho_psi_local(const BatchInst* __restrict__ inst, int id, int local,
                                                    int parity, StepArgs* sa) {
  stage_args(inst, id, parity, sa);
  const int64_t i = (int64_t)local * kThreads + threadIdx.x;
  if (i < sa->n) rho_psi_node<KIND>(*sa, sa->f_in, i);
  if (REUSE) __syncthreads();
}

template <int KIND, bool REUSE>
__device__ __forceinline__ void batch_rho_psi_item(const BatchInst* __restrict__ inst, const int* __restrict__ owner,
                                                   int w, int parity, StepArgs* sa) {
  const int id = owner[w];
  batch_rho_psi_local<KIND, REUSE>(inst, id, w - inst[id].k1_start, parity, sa);
}

// collision pass over tile t of instance id; org: two shared ints for the tile
// origin, which one thread computes per item; REUSE as for the density pass
template <int KIND, bool ST, bool REUSE>
__device__ __forceinline__ void batch_collide_local(const BatchInst* __restrict__ inst, int id, int t, int parity,
                                                    double* sp, StepArgs* sa, int* org) {
  const BatchInst& I = inst[id];
  if (threadIdx.x == 0) {
    const int tyi = t / I.tiles_x;
    org[0] = (t - tyi * I.tiles_x) * I.tw;
    org[1] = tyi * I.th;
  }
  stage_args(inst, id, parity, sa);  // ends with a barrier: org is visible
  const StepArgs& a = *sa;
  const int tw = I.tw, th = I.th, log2tw = I.log2tw;
  const int x0 = org[0], y0 = org[1];
  const int lx = threadIdx.x & (tw - 1), ly = threadIdx.x >> log2tw;
  load_psi_tile(a, sp, x0, y0, tw, th, lx, ly, threadIdx.x, kThreads);
  __syncthreads();
  const int x = x0 + lx, y = y0 + ly;
  if (x < a.nx && y < a.ny)
    collide_node<KIND, false, ST>(a, x, y, sp, (ly + 1) * (tw + 2) + lx + 1, tw + 2, nullptr, nullptr, nullptr,
                                  nullptr);
  if (REUSE) __syncthreads();
}

template <int KIND, bool ST, bool REUSE>
__device__ __forceinline__ void batch_collide_item(const BatchInst* __restrict__ inst, const int* __restrict__ owner,
                                                   int w, int parity, double* sp, StepArgs* sa, int* org) {
  const int id = owner[w];
  batch_collide_local<KIND, ST, REUSE>(inst, id, w - inst[id].k2_start, parity, sp, sa, org);
}

template <int KIND>
__global__ void __launch_bounds__(kThreads) k_batch_rho_psi(const BatchInst* inst, const int* owner, int parity) {
  __shared__ StepArgs sa;
  batch_rho_psi_item<KIND, false>(inst, owner, blockIdx.x, parity, &sa);
}

// ST: some instance has the surface-tension source (kappa != 0); for the others
// kappa_q = 0 makes the source exactly zero, so their results do not change
// Unit relaxation times: 5 resident blocks per SM (at most 48 registers); the
// integer-bound collision pass issues faster with the extra warps than it loses to
// the 8-20 bytes of spilled registers. The other kinds keep 4 (they would spill more).
constexpr int collide_min_blocks(int kind) { return kind == kUnitTau ? 5 : 4; }

template <int KIND, bool ST>
__global__ void __launch_bounds__(kThreads, collide_min_blocks(KIND))
    k_batch_collide(const BatchInst* inst, const int* owner, int parity) {
  __shared__ double sp[kMaxTileSmem];
  __shared__ StepArgs sa;
  __shared__ int org[2];
  batch_collide_item<KIND, ST, false>(inst, owner, blockIdx.x, parity, sp, &sa, org);
}

// Work items of both passes in one launch (the pipelined plan): item.x is the
// instance, with the top bit set for a collision tile; item.y the item's index within
// its instance. Density items read buffer p1, collision items p2. Lattices of one
// group run their density pass while those of the other run their collision pass, so
// the FP64 pipe (the density pass's bound) and the integer pipe (the collision pass's)
// work at the same time on every SM.
template <int KIND, bool ST>
__global__ void __launch_bounds__(kThreads, collide_min_blocks(KIND))
    k_batch_mixed(const BatchInst* inst, const int2* items, int p1, int p2) {
  __shared__ double sp[kMaxTileSmem];
  __shared__ StepArgs sa;
  __shared__ int org[2];
  const int2 it = items[blockIdx.x];
  if (it.x >= 0)
    batch_rho_psi_local<KIND, false>(inst, it.x, it.y, p1, &sa);
  else
    batch_collide_local<KIND, ST, false>(inst, it.x & 0x7FFFFFFF, it.y, p2, sp, &sa, org);
}

template <int KIND, bool ST>
__global__ void __launch_bounds__(kThreads) k_batch_persistent(const BatchInst* inst, const int* owner1, int n1,
                                                               const int* owner2, int n2, int parity0, long long nsteps,
                                                               GridBarrier* bar, int* err, unsigned spin_limit,
                                                               int absent_block) {
  __shared__ double sp[kMaxTileSmem];
  __shared__ StepArgs sa;
  __shared__ int org[2];
  // barrier self-test only: one block leaves without arriving, so the others' waits run out
  if ((int)blockIdx.x == absent_block) return;
  for (long long s = 0; s < nsteps; ++s) {
    const int parity = (int)((parity0 + s) & 1);
    for (int w = blockIdx.x; w < n1; w += gridDim.x) batch_rho_psi_item<KIND, true>(inst, owner1, w, parity, &sa);
    if (!grid_barrier(bar, err, spin_limit)) return;
    for (int w = blockIdx.x; w < n2; w += gridDim.x)
      batch_collide_item<KIND, ST, true>(inst, owner2, w, parity, sp, &sa, org);
    if (!grid_barrier(bar, err, spin_limit)) return;
  }
}

// Guard, pass 1: one block per 256-node work item of the density pass; per block
// (mass, max |u|, bad count, sum |rho - rho'|), reduced in a fixed tree order
// (guard_node, the same terms as the single-lattice guard). Runs after a density
// pass over the current state, so rho, j and psi are those the next step starts
// from. Refreshes the snapshot rho'.
__global__ void __launch_bounds__(kThreads) k_batch_guard_partial(const BatchInst* inst, const int* owner, int parity,
                                                                  const int* snap_valid, double* partials) {
  __shared__ double s[kGuardQ][kThreads];
  const int w = blockIdx.x;
  const int id = owner[w];
  const BatchInst& I = inst[id];
  const StepArgs& a = I.a[parity];
  const int64_t i = (int64_t)(w - I.k1_start) * kThreads + threadIdx.x;
  double v[kGuardQ] = {0.0, 0.0, 0.0, 0.0};
  if (i < a.n) guard_node(a, i, I.snap, snap_valid[id] != 0, v);
  guard_block_reduce<kThreads>(v, s);
  if (threadIdx.x < kGuardQ) partials[kGuardQ * (int64_t)w + threadIdx.x] = s[threadIdx.x][0];
}

// Guard, pass 2: one block per instance over its work items, in a fixed order.
__global__ void __launch_bounds__(kThreads) k_batch_guard_final(const BatchInst* inst, const double* partials,
                                                                int* snap_valid, double* out) {
  __shared__ double s[kGuardQ][kThreads];
  const int id = blockIdx.x;
  const BatchInst& I = inst[id];
  const int nb = (int)((I.a[0].n + kThreads - 1) / kThreads);
  double v[kGuardQ] = {0.0, 0.0, 0.0, 0.0};
  for (int k = threadIdx.x; k < nb; k += kThreads) {
    const double* p = partials + kGuardQ * (int64_t)(I.k1_start + k);
    v[0] += p[0];
    v[1] = fmax(v[1], p[1]);
    v[2] += p[2];
    v[3] += p[3];
  }
  guard_block_reduce<kThreads>(v, s);
  if (threadIdx.x == 0) {
    out[kGuardQ * id + 0] = s[0][0];
    out[kGuardQ * id + 1] = s[1][0];
    out[kGuardQ * id + 2] = s[2][0];
    out[kGuardQ * id + 3] = snap_valid[id] ? s[3][0] / s[0][0] : -1.0;
    snap_valid[id] = 1;
  }
}

template <bool ST>
const void* persistent_kernel_t(int kind) {
  switch (kind) {
    case kUnitTau: return (const void*)k_batch_persistent<kUnitTau, ST>;
    case kShearTau: return (const void*)k_batch_persistent<kShearTau, ST>;
    default: return (const void*)k_batch_persistent<kFullMrt, ST>;
  }
}

const void* persistent_kernel(int kind, bool st) {
  return st ? persistent_kernel_t<true>(kind) : persistent_kernel_t<false>(kind);
}

template <bool ST>
void launch_pair_t(int kind, const BatchInst* inst, const int* o1, int n1, const int* o2, int n2, int parity,
                   cudaStream_t s) {
  switch (kind) {
    case kUnitTau:
      k_batch_rho_psi<kUnitTau><<<n1, kThreads, 0, s>>>(inst, o1, parity);
      k_batch_collide<kUnitTau, ST><<<n2, kThreads, 0, s>>>(inst, o2, parity);
      break;
    case kShearTau:
      k_batch_rho_psi<kShearTau><<<n1, kThreads, 0, s>>>(inst, o1, parity);
      k_batch_collide<kShearTau, ST><<<n2, kThreads, 0, s>>>(inst, o2, parity);
      break;
    default:
      k_batch_rho_psi<kFullMrt><<<n1, kThreads, 0, s>>>(inst, o1, parity);
      k_batch_collide<kFullMrt, ST><<<n2, kThreads, 0, s>>>(inst, o2, parity);
      break;
  }
}

void launch_pair(int kind, bool st, const BatchInst* inst, const int* o1, int n1, const int* o2, int n2, int parity,
                 cudaStream_t s) {
  if (st)
    launch_pair_t<true>(kind, inst, o1, n1, o2, n2, parity, s);
  else
    launch_pair_t<false>(kind, inst, o1, n1, o2, n2, parity, s);
}

// one launch of the mixed kernel over n items
void launch_mixed(int kind, bool st, const BatchInst* inst, const int2* items, int n, int p1, int p2, cudaStream_t s) {
  if (n <= 0) return;
#define PPLBM_KM(K)                                                                   \
  do {                                                                                \
    if (st)                                                                           \
      k_batch_mixed<K, true><<<n, kThreads, 0, s>>>(inst, items, p1, p2);             \
    else                                                                              \
      k_batch_mixed<K, false><<<n, kThreads, 0, s>>>(inst, items, p1, p2);            \
  } while (0)
  switch (kind) {
    case kUnitTau: PPLBM_KM(kUnitTau); break;
    case kShearTau: PPLBM_KM(kShearTau); break;
    default: PPLBM_KM(kFullMrt); break;
  }
#undef PPLBM_KM
}

// the collision pass alone, over every instance
void launch_collision_pass(int kind, bool st, const BatchInst* inst, const int* o2, int n2, int parity,
                           cudaStream_t s) {
#define PPLBM_K2(K)                                                                   \
  do {                                                                                \
    if (st)                                                                           \
      k_batch_collide<K, true><<<n2, kThreads, 0, s>>>(inst, o2, parity);             \
    else                                                                              \
      k_batch_collide<K, false><<<n2, kThreads, 0, s>>>(inst, o2, parity);            \
  } while (0)
  switch (kind) {
    case kUnitTau: PPLBM_K2(kUnitTau); break;
    case kShearTau: PPLBM_K2(kShearTau); break;
    default: PPLBM_K2(kFullMrt); break;
  }
#undef PPLBM_K2
}

// the density/psi pass alone, over every instance (refreshes psi and the moments)
void launch_density_pass(int kind, const BatchInst* inst, const int* o1, int n1, int parity, cudaStream_t s) {
  switch (kind) {
    case kUnitTau: k_batch_rho_psi<kUnitTau><<<n1, kThreads, 0, s>>>(inst, o1, parity); break;
    case kShearTau: k_batch_rho_psi<kShearTau><<<n1, kThreads, 0, s>>>(inst, o1, parity); break;
    default: k_batch_rho_psi<kFullMrt><<<n1, kThreads, 0, s>>>(inst, o1, parity); break;
  }
}

}  // namespace
}  // namespace pplbm
