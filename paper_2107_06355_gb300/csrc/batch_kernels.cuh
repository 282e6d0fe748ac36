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

// ---- the pipelined plan's mixed kernel ----------------------------------------------

// 8- and 16-byte asynchronous copies global -> shared (cp.async, cached in L1); the
// data is visible to the block after cp_async_wait_all and a barrier. Both addresses
// are aligned to the copy size.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// A work item of the pipelined plan (int4): x = the instance, with the top bit set for
// a collision tile; for a density item y = its 256-node block within the instance; for
// a collision tile y = log2 of the tile width tw (tile height 256 / tw) and (z, w) the
// tile's origin (x0, y0).
__device__ __forceinline__ bool is_collision_item(const int4& h) { return h.x < 0; }

// Starts the copy of the item's StepArgs (density items: parity p1, collision tiles:
// p2) into dst.
__device__ __forceinline__ void fetch_item_args(const BatchInst* __restrict__ inst, const int4& h, int p1, int p2,
                                                StepArgs* dst) {
  const int id = h.x & 0x7FFFFFFF;
  const unsigned long long* src =
      reinterpret_cast<const unsigned long long*>(&inst[id].a[is_collision_item(h) ? p2 : p1]);
  unsigned long long* d = reinterpret_cast<unsigned long long*>(dst);
  for (int k = threadIdx.x; k < (int)(sizeof(StepArgs) / 8); k += kThreads) cp_async8(d + k, src + k);
}

// Starts the load of a collision tile's psi halo tile into sp (row stride tw + 2), as
// load_psi_tile does: psi values by asynchronous copies, the wall ghost values by
// plain stores.
__device__ __forceinline__ void fetch_item_tile(const StepArgs& a, const int4& h, double* sp) {
  const int log2tw = h.y, tw = 1 << log2tw, th = kThreads >> log2tw, sw = tw + 2;
  const int x0 = h.z, y0 = h.w;
  const int nh = 2 * sw + 2 * th;
  for (int k = (int)threadIdx.x - kThreads; k < nh; k += kThreads) {
    int tx, ty;
    if (k < 0) {  // the thread's own node
      tx = 1 + ((int)threadIdx.x & (tw - 1));
      ty = 1 + ((int)threadIdx.x >> log2tw);
    } else if (k < 2 * sw) {
      const bool top = k >= sw;
      ty = top ? th + 1 : 0;
      tx = top ? k - sw : k;
    } else {
      const int j = k - 2 * sw;
      ty = 1 + (j >> 1);
      tx = (j & 1) ? tw + 1 : 0;
    }
    const int gx = wrap_near(x0 + tx - 1, a.nx);
    int gy = y0 + ty - 1;
    double* d = sp + ty * sw + tx;
    if (a.walls && (gy < 0 || gy >= a.ny)) {
      *d = gy < 0 ? a.psi_ghost_bottom : a.psi_ghost_top;
    } else {
      if (!a.walls) gy = wrap_near(gy, a.ny);
      cp_async8(d, a.psi + (int64_t)gy * a.nx + gx);
    }
  }
}

// The item's pass from its staged arguments (and tile)
template <int KIND, bool ST>
__device__ __forceinline__ void run_item(const StepArgs& a, const int4& h, const double* sp) {
  if (!is_collision_item(h)) {
    const int64_t i = (int64_t)h.y * kThreads + threadIdx.x;
    if (i < a.n) rho_psi_node<KIND>(a, a.f_in, i);
    return;
  }
  const int log2tw = h.y, tw = 1 << log2tw;
  const int lx = (int)threadIdx.x & (tw - 1), ly = (int)threadIdx.x >> log2tw;
  const int x = h.z + lx, y = h.w + ly;
  if (x < a.nx && y < a.ny)
    collide_node<KIND, false, ST>(a, x, y, sp, (ly + 1) * (tw + 2) + lx + 1, tw + 2, nullptr,
                                  nullptr, nullptr, nullptr);
}

// Work items of both passes in one launch (the pipelined plan): density items read
// buffer p1, collision tiles p2. Lattices of one group run their density pass while
// those of the other run their collision pass, so the FP64 pipe (the density pass's
// bound) and the integer pipe (the collision pass's) work at the same time on every
// SM. The grid is the resident block count G (at most n). Block b starts with item b;
// later items come in table order from the queue counter queue[0] (item G + the
// counter's old value), taken four items ahead: while a block computes item k it
// copies in the psi tile of item k + 1, the arguments of item k + 2 and the header of
// item k + 3 (rings of 2 tiles, 4 argument blocks, 4 headers and 4 table indices), so
// that no item waits on its set-up loads. The last block to finish resets queue[0]
// and the finished-block count queue[1] for the next launch.
template <int KIND, bool ST>
__global__ void __launch_bounds__(kThreads, collide_min_blocks(KIND))
    k_batch_mixed(const BatchInst* inst, const int4* items, int n, int p1, int p2, unsigned* queue) {
  __shared__ double sp[2][kMaxTileSmem];
  __shared__ StepArgs sa[4];
  __shared__ int4 hdr[4];
  __shared__ int qi[4];  // table index of the ring slot's item; -1: none
  const int G = gridDim.x;
  if (threadIdx.x == 0) {
    const int t = G + (int)atomicAdd(&queue[0], 3u);
    qi[0] = blockIdx.x;
    qi[1] = t < n ? t : -1;
    qi[2] = t + 1 < n ? t + 1 : -1;
    qi[3] = t + 2 < n ? t + 2 : -1;
  }
  __syncthreads();
  if (threadIdx.x < 3 && qi[threadIdx.x] >= 0) cp_async16(&hdr[threadIdx.x], items + qi[threadIdx.x]);
  cp_async_wait_all();
  __syncthreads();
  fetch_item_args(inst, hdr[0], p1, p2, &sa[0]);
  if (qi[1] >= 0) fetch_item_args(inst, hdr[1], p1, p2, &sa[1]);
  cp_async_wait_all();
  __syncthreads();
  if (is_collision_item(hdr[0])) fetch_item_tile(sa[0], hdr[0], sp[0]);
  cp_async_wait_all();
  __syncthreads();
  // qi[c] is rewritten during iteration k (thread 0, for item k + 4), so whether item
  // k + 1 exists is read from its slot c1 before the iteration's barrier: slot c1 is
  // not written during iteration k, and every thread reads the same value
  for (int k = 0;; ++k) {
    const int c = k & 3, c1 = (k + 1) & 3, c2 = (k + 2) & 3, c3 = (k + 3) & 3;
    if (qi[c1] >= 0 && is_collision_item(hdr[c1])) fetch_item_tile(sa[c1], hdr[c1], sp[(k + 1) & 1]);
    if (qi[c2] >= 0) fetch_item_args(inst, hdr[c2], p1, p2, &sa[c2]);
    int next = -1;
    if (threadIdx.x == 0) {
      if (qi[c3] >= 0) cp_async16(&hdr[c3], items + qi[c3]);
      const int t = G + (int)atomicAdd(&queue[0], 1u);
      next = t < n ? t : -1;
    }
    run_item<KIND, ST>(sa[c], hdr[c], sp[k & 1]);
    if (threadIdx.x == 0) qi[c] = next;  // slot c now names item k + 4
    const bool more = qi[c1] >= 0;
    cp_async_wait_all();
    __syncthreads();
    if (!more) break;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&queue[1], 1u) == (unsigned)G - 1u) {
      queue[0] = 0u;
      queue[1] = 0u;
      __threadfence();
    }
  }
}

template <bool ST>
const void* mixed_kernel_t(int kind) {
  switch (kind) {
    case kUnitTau: return (const void*)k_batch_mixed<kUnitTau, ST>;
    case kShearTau: return (const void*)k_batch_mixed<kShearTau, ST>;
    default: return (const void*)k_batch_mixed<kFullMrt, ST>;
  }
}

const void* mixed_kernel(int kind, bool st) { return st ? mixed_kernel_t<true>(kind) : mixed_kernel_t<false>(kind); }

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

// one launch of the mixed kernel over n items with `grid` blocks (at most n); queue:
// the kernel's two counters, zero before the launch (and after it)
void launch_mixed(int kind, bool st, const BatchInst* inst, const int4* items, int n, int grid, int p1, int p2,
                  unsigned* queue, cudaStream_t s) {
  if (n <= 0) return;
  grid = grid < n ? grid : n;
#define PPLBM_KM(K)                                                                   \
  do {                                                                                \
    if (st)                                                                           \
      k_batch_mixed<K, true><<<grid, kThreads, 0, s>>>(inst, items, n, p1, p2, queue);\
    else                                                                              \
      k_batch_mixed<K, false><<<grid, kThreads, 0, s>>>(inst, items, n, p1, p2, queue);\
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
