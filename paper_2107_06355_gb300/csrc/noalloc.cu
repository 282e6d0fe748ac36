// pplbm_step_noalloc: one time step with no device allocation.
//
// For callers that cannot allocate device memory: code running under a host
// application or framework that owns every byte of device memory (its own pool
// allocator, a fixed memory budget), and code on a latency-critical stream that
// must not let cudaMalloc/cudaFree synchronise the device. Such callers pass the
// input and output distributions; the intermediate psi and moment planes the two
// step kernels exchange live in a static device array compiled into this library.
//
// The array is file-scope `static __device__`, so every GPU that loads the library
// holds it (5.2 MB) until the process exits. Host code cannot use its name as a
// device address; the address is taken once per device with cudaGetSymbolAddress
// on the first call made while that device is current, and kept for the life of
// the process (a cudaDeviceReset() ends the context that address belongs to, so
// the entry point must not be called after one).
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>

#include "../../include/pplbm.h"
#include "internal.h"

namespace pplbm {
namespace {

constexpr int64_t kNoAllocMaxNodes = 65536;  // largest lattice nx*ny this entry point accepts
constexpr int kNoAllocPlanes = 10;           // psi + up to 9 moment planes
constexpr int64_t kHeaderDoubles = 32;       // first 256 bytes: the error word

static __device__ __align__(256) double g_noalloc_scratch[kHeaderDoubles + kNoAllocPlanes * kNoAllocMaxNodes];

constexpr int kMaxDevices = 64;
std::atomic<double*> g_scratch_addr[kMaxDevices];

const char* kMsgTooLarge = "pplbm_step_noalloc: nx*ny exceeds the static scratch limit of 65536 nodes";
const char* kMsgArgs = "pplbm_step_noalloc: invalid lattice, relaxation set, EOS block or buffer";
const char* kMsgOverlap = "pplbm_step_noalloc: f_in and f_out overlap (they must be distinct 9*nx*ny buffers)";
const char* kMsgSymbol = "pplbm_step_noalloc: cudaGetSymbolAddress of the static scratch failed";
const char* kMsgCuda = "pplbm_step_noalloc: a CUDA call failed";
const char* kMsgDiverged = "pplbm_step_noalloc: non-finite or non-positive density, or psi^2 <= 0";

pplbm_status noalloc_fail(const char** message, pplbm_status s, const char* text) {
  if (message) *message = text;
  return s;
}

}  // namespace
}  // namespace pplbm

using namespace pplbm;

extern "C" pplbm_status pplbm_step_noalloc(const pplbm_lattice* lattice, const pplbm_eos_derived* eos,
                                           const pplbm_relax* relax, const double* f_in, double* f_out,
                                           void* stream, const char** message) {
  if (message) *message = "";
  const int kind = collision_kind(relax);
  if (!lattice || !eos || !f_in || !f_out || kind < 0 || lattice->nx < 1 || lattice->ny < 1 ||
      lattice->reserved != 0 || !(eos->G < 0.0) || eos->mode < PPLBM_EOS_CS || eos->mode > PPLBM_EOS_SMOOTH_MOD)
    return noalloc_fail(message, PPLBM_ERR_ARG, kMsgArgs);
  const uint32_t bc = lattice->bc, walls_bits = bc & (PPLBM_BC_WALL_BOTTOM | PPLBM_BC_WALL_TOP);
  const bool per_y = (bc & PPLBM_BC_PERIODIC_Y) != 0;
  if (!(bc & PPLBM_BC_PERIODIC_X) || (per_y && walls_bits) ||
      (!per_y && walls_bits != (PPLBM_BC_WALL_BOTTOM | PPLBM_BC_WALL_TOP)))
    return noalloc_fail(message, PPLBM_ERR_ARG, kMsgArgs);
  const int64_t n = (int64_t)lattice->nx * lattice->ny;
  if (n > kNoAllocMaxNodes) return noalloc_fail(message, PPLBM_ERR_ARG, kMsgTooLarge);
  // f_in and f_out are two separate buffers, as in the context path: reject any overlap
  const uintptr_t in0 = (uintptr_t)f_in, out0 = (uintptr_t)f_out, bytes = (uintptr_t)(9 * n) * sizeof(double);
  if (in0 < out0 + bytes && out0 < in0 + bytes) return noalloc_fail(message, PPLBM_ERR_ARG, kMsgOverlap);

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(message, PPLBM_ERR_CUDA, kMsgCuda);
  double* base = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!base) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return noalloc_fail(message, PPLBM_ERR_CUDA, kMsgSymbol);
    }
    base = (double*)p;
    g_scratch_addr[dev].store(base, std::memory_order_release);
  }
  cudaStream_t s = (cudaStream_t)stream;
  int* err = (int*)base;

  StepArgs a;
  std::memset(&a, 0, sizeof(a));
  a.f_in = f_in;
  a.f_out = f_out;
  a.psi = base + kHeaderDoubles;
  a.mom = base + kHeaderDoubles + n;
  a.err = err;
  a.nx = lattice->nx;
  a.ny = lattice->ny;
  a.n = n;
  a.walls = per_y ? 0 : 1;
  a.kind = kind;
  a.eos = make_eos_const(*eos);
  a.G = eos->G;
  a.half_force = -eos->G / 24.0;
  a.psi_ghost_bottom = eos->psi_l;
  a.psi_ghost_top = eos->psi_v;
  set_collision_args(a, kind, *relax, *eos, eos->G);

  // the error word keeps the previous call's value: clear it first
  if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return noalloc_fail(message, PPLBM_ERR_CUDA, kMsgCuda);
  launch_rho_psi(a, s);
  launch_collide(a, s);
  int h = 0;
  if (cudaGetLastError() != cudaSuccess || cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return noalloc_fail(message, PPLBM_ERR_CUDA, kMsgCuda);
  if (h != 0) return noalloc_fail(message, PPLBM_ERR_DIVERGED, kMsgDiverged);
  return PPLBM_OK;
}
