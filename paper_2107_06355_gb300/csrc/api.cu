// C ABI of the library: context life cycle, argument checking, stream-ordered
// launches of the step kernels, host/device staging and sticky error handling.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "../../include/pplbm.h"
#include "internal.h"

using namespace pplbm;

#include "ctx.h"

namespace {

pplbm_status fail(pplbm_ctx* c, pplbm_status s, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
pplbm_status fail(pplbm_ctx* c, pplbm_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->msg = buf;
  }
  return s;
}

pplbm_status cuda_fail(pplbm_ctx* c, cudaError_t e, const char* what) {
  return fail(c, PPLBM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CUDA_TRY(c, call)                                   \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail((c), e_, #call); \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// 8-node rows of tiles on a grid's y axis, at most 65,535 of them
constexpr int kMaxRows = 65535 * 8;

bool valid_lattice(const pplbm_lattice* l) {
  if (!l || l->nx < 1 || l->ny < 1 || l->reserved != 0) return false;
  const int64_t n = (int64_t)l->nx * l->ny;
  if (9 * n >= (int64_t)1 << 31) return false;
  if (l->ny > kMaxRows) return false;  // the 2-D grids of the collision and adjoint passes
  if (!(l->bc & PPLBM_BC_PERIODIC_X)) return false;
  const uint32_t walls = l->bc & (PPLBM_BC_WALL_BOTTOM | PPLBM_BC_WALL_TOP);
  if (l->bc & PPLBM_BC_PERIODIC_Y) return walls == 0;
  return walls == (PPLBM_BC_WALL_BOTTOM | PPLBM_BC_WALL_TOP);
}

pplbm_status check_sticky(pplbm_ctx* c) {
  if (c->sticky != PPLBM_OK) return c->sticky;
  return PPLBM_OK;
}

// Reads the device error word (synchronises the stream).
pplbm_status poll_error(pplbm_ctx* c) {
  int h = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (h != 0 && c->sticky == PPLBM_OK) {
    c->sticky = PPLBM_ERR_DIVERGED;
    c->msg = "a kernel met a non-finite or non-positive density, or psi^2 <= 0";
  }
  return c->sticky;
}

// device pointer for an n-value input: `p` itself, or a staged copy in plane `plane` of fB
pplbm_status stage_in(pplbm_ctx* c, const double* p, int plane, const double** out) {
  if (!p) {
    *out = nullptr;
    return PPLBM_OK;
  }
  if (is_device_ptr(p)) {
    *out = p;
    return PPLBM_OK;
  }
  double* dst = c->fB + (int64_t)plane * c->n;
  CUDA_TRY(c, cudaMemcpyAsync(dst, p, sizeof(double) * c->n, cudaMemcpyHostToDevice, c->stream));
  *out = dst;
  return PPLBM_OK;
}

pplbm_status grow_events(pplbm_ctx* c, int k, size_t need) {
  while (c->ev[k].size() < need) {
    cudaEvent_t e;
    CUDA_TRY(c, cudaEventCreate(&e));
    c->ev[k].push_back(e);
  }
  return PPLBM_OK;
}

// launches kernel k (0: density/psi, 1: collision) with optional timing events
pplbm_status timed_launch(pplbm_ctx* c, int k) {
  if (c->timing) {
    if (pplbm_status s = grow_events(c, k, c->ev_used[k] + 2)) return s;
    cudaEventRecord(c->ev[k][c->ev_used[k]], c->stream);
  }
  if (k == 0) launch_rho_psi(c->args, c->stream);
  else launch_collide(c->args, c->stream);
  if (c->timing) {
    cudaEventRecord(c->ev[k][c->ev_used[k] + 1], c->stream);
    c->ev_used[k] += 2;
  }
  return PPLBM_OK;
}

}  // namespace

extern "C" {

const char* pplbm_status_string(pplbm_status s) {
  switch (s) {
    case PPLBM_OK: return "ok";
    case PPLBM_ERR_ARG: return "invalid argument";
    case PPLBM_ERR_EOS_SETUP: return "equation-of-state set-up failed";
    case PPLBM_ERR_CUDA: return "CUDA error";
    case PPLBM_ERR_DIVERGED: return "simulation diverged";
    case PPLBM_ERR_TIMEOUT: return "device wait timed out";
    case PPLBM_ERR_STATE: return "invalid state";
  }
  return "unknown status";
}

size_t pplbm_workspace_bytes(const pplbm_lattice* lattice, const pplbm_relax* relax) {
  if (!valid_lattice(lattice)) return 0;
  const int kind = collision_kind(relax);
  if (kind < 0) return 0;
  const size_t n = (size_t)lattice->nx * lattice->ny;
  return sizeof(double) * n * (9 + 9 + 1 + (size_t)moment_planes(kind) + 1);
}

pplbm_status pplbm_create(pplbm_ctx** out, const pplbm_lattice* lattice, const pplbm_eos_params* eos,
                          const pplbm_relax* relax, double G, void* workspace, size_t workspace_bytes,
                          void* stream) {
  if (!out) return PPLBM_ERR_ARG;
  *out = nullptr;
  if (!valid_lattice(lattice) || !eos || !workspace) return PPLBM_ERR_ARG;
  const int kind = collision_kind(relax);
  if (kind < 0) return PPLBM_ERR_ARG;
  if (workspace_bytes < pplbm_workspace_bytes(lattice, relax)) return PPLBM_ERR_ARG;
  if (((uintptr_t)workspace & 15u) != 0) return PPLBM_ERR_ARG;
  pplbm_eos_derived d;
  const pplbm_status st = pplbm_eos_setup(eos, G, &d);
  if (st != PPLBM_OK) return st;
  pplbm_ctx* c = new (std::nothrow) pplbm_ctx();
  if (!c) return PPLBM_ERR_ARG;
  c->lat = *lattice;
  c->relax = *relax;
  c->eos_params = *eos;
  c->eos = d;
  c->G = G;
  c->n = (int64_t)lattice->nx * lattice->ny;
  c->nmom = moment_planes(kind);
  double* w = (double*)workspace;
  c->fA = w;
  c->fB = w + 9 * c->n;
  c->psi = w + 18 * c->n;
  c->mom = w + 19 * c->n;
  c->snap = w + (19 + c->nmom) * c->n;
  c->snap_valid = false;
  c->stream = (cudaStream_t)stream;
  c->sticky = PPLBM_OK;
  const size_t partial_bytes = sizeof(double) * 4 * guard_blocks();
  const size_t block_bytes = 256 + partial_bytes + 256;
  cudaError_t e = cudaMalloc(&c->dev_block, block_bytes);
  if (e != cudaSuccess) {
    delete c;
    return PPLBM_ERR_CUDA;
  }
  c->d_err = (int*)c->dev_block;
  c->d_partials = (double*)((char*)c->dev_block + 256);
  c->d_guard = (double*)((char*)c->dev_block + 256 + partial_bytes);
  e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
  if (e != cudaSuccess) {
    cudaFree(c->dev_block);
    delete c;
    return PPLBM_ERR_CUDA;
  }

  StepArgs& a = c->args;
  std::memset(&a, 0, sizeof(a));
  a.f_in = c->fA;
  a.f_out = c->fB;
  a.psi = c->psi;
  a.mom = c->mom;
  a.err = c->d_err;
  a.nx = lattice->nx;
  a.ny = lattice->ny;
  a.n = c->n;
  a.walls = (lattice->bc & PPLBM_BC_PERIODIC_Y) ? 0 : 1;
  a.kind = kind;
  a.eos = make_eos_const(d);
  a.G = G;
  a.half_force = -G / 24.0;
  a.psi_ghost_bottom = d.psi_l;  // liquid below the bottom wall (Sec. IV)
  a.psi_ghost_top = d.psi_v;     // vapour above the top wall
  set_collision_args(a, kind, *relax, d, G);
  *out = c;
  return PPLBM_OK;
}

pplbm_status pplbm_set_stream(pplbm_ctx* c, void* stream) {
  if (!c) return PPLBM_ERR_ARG;
  c->stream = (cudaStream_t)stream;
  return PPLBM_OK;
}

pplbm_status pplbm_init_equilibrium(pplbm_ctx* c, const double* rho0, const double* ux0, const double* uy0) {
  if (!c || !rho0) return fail(c, PPLBM_ERR_ARG, "rho0 is NULL");
  if (pplbm_status s = check_sticky(c)) return s;
  const double *r, *u, *v;
  pplbm_status s;
  if ((s = stage_in(c, rho0, 0, &r)) || (s = stage_in(c, ux0, 1, &u)) || (s = stage_in(c, uy0, 2, &v))) return s;
  launch_init_eq(c->args, c->fA, r, u, v, c->stream);
  CUDA_TRY(c, cudaGetLastError());
  c->steps = 0;
  c->snap_valid = false;
  return poll_error(c);
}

pplbm_status pplbm_step(pplbm_ctx* c, int64_t nsteps) {
  if (!c || nsteps < 0) return fail(c, PPLBM_ERR_ARG, "nsteps < 0");
  if (pplbm_status s = check_sticky(c)) return s;
  for (int64_t k = 0; k < nsteps; ++k) {
    StepArgs& a = c->args;
    a.f_in = c->fA;
    a.f_out = c->fB;
    if (pplbm_status s = timed_launch(c, 0)) return s;
    if (pplbm_status s = timed_launch(c, 1)) return s;
    double* t = c->fA;
    c->fA = c->fB;
    c->fB = t;
  }
  CUDA_TRY(c, cudaGetLastError());
  c->steps += nsteps;
  return PPLBM_OK;
}

pplbm_status pplbm_get_fields(pplbm_ctx* c, double* rho, double* ux, double* uy, double* psi) {
  if (!c) return PPLBM_ERR_ARG;
  if (pplbm_status s = check_sticky(c)) return s;
  StepArgs a = c->args;
  a.f_in = c->fA;
  a.f_out = c->fB;
  launch_rho_psi(a, c->stream);
  double* outs[4] = {rho, ux, uy, psi};
  double* dst[4];
  bool host[4];
  for (int k = 0; k < 4; ++k) {
    host[k] = outs[k] && !is_device_ptr(outs[k]);
    dst[k] = host[k] ? c->fB + (int64_t)k * c->n : outs[k];
  }
  launch_fields(a, dst[0], dst[1], dst[2], dst[3], c->stream);
  CUDA_TRY(c, cudaGetLastError());
  for (int k = 0; k < 4; ++k)
    if (host[k])
      CUDA_TRY(c, cudaMemcpyAsync(outs[k], dst[k], sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->stream));
  return poll_error(c);
}

pplbm_status pplbm_get_f(pplbm_ctx* c, double* f) {
  if (!c || !f) return fail(c, PPLBM_ERR_ARG, "f is NULL");
  CUDA_TRY(c, cudaMemcpyAsync(f, c->fA, sizeof(double) * 9 * c->n, cudaMemcpyDefault, c->stream));
  if (!is_device_ptr(f)) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return PPLBM_OK;
}

pplbm_status pplbm_set_f(pplbm_ctx* c, const double* f) {
  if (!c || !f) return fail(c, PPLBM_ERR_ARG, "f is NULL");
  if (pplbm_status s = check_sticky(c)) return s;
  CUDA_TRY(c, cudaMemcpyAsync(c->fA, f, sizeof(double) * 9 * c->n, cudaMemcpyDefault, c->stream));
  if (!is_device_ptr(f)) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->snap_valid = false;
  return PPLBM_OK;
}

pplbm_status pplbm_sync(pplbm_ctx* c, int64_t* steps_done) {
  if (!c) return PPLBM_ERR_ARG;
  const pplbm_status s = poll_error(c);
  if (steps_done) *steps_done = c->steps;
  return s;
}

pplbm_status pplbm_guard(pplbm_ctx* c, double out[4]) {
  if (!c || !out) return fail(c, PPLBM_ERR_ARG, "out is NULL");
  if (pplbm_status s = check_sticky(c)) return s;
  StepArgs a = c->args;
  a.f_in = c->fA;
  a.f_out = c->fB;
  launch_guard(a, c->snap, c->snap_valid ? 1 : 0, c->d_partials, c->d_guard, c->stream);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaMemcpyAsync(out, c->d_guard, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  const pplbm_status s = poll_error(c);
  c->snap_valid = true;
  if (s == PPLBM_OK && out[2] > 0) {
    c->sticky = PPLBM_ERR_DIVERGED;
    c->msg = "non-finite or non-positive density in the state";
    return c->sticky;
  }
  return s;
}

pplbm_status pplbm_get_derived(const pplbm_ctx* c, pplbm_eos_derived* out) {
  if (!c || !out) return PPLBM_ERR_ARG;
  *out = c->eos;
  return PPLBM_OK;
}

pplbm_status pplbm_run_host(pplbm_ctx* c, const double* rho0, const double* ux0, const double* uy0,
                            int64_t nsteps, double* rho_out) {
  if (!c || !rho0 || !rho_out) return fail(c, PPLBM_ERR_ARG, "NULL host buffer");
  pplbm_status s = pplbm_init_equilibrium(c, rho0, ux0, uy0);
  if (s != PPLBM_OK) return s;
  if ((s = pplbm_step(c, nsteps)) != PPLBM_OK) return s;
  return pplbm_get_fields(c, rho_out, nullptr, nullptr, nullptr);
}

pplbm_status pplbm_enable_kernel_timing(pplbm_ctx* c, int64_t capacity) {
  if (!c || capacity < 0) return PPLBM_ERR_ARG;
  c->timing = capacity > 0;
  if (c->timing) {
    for (int k = 0; k < 2; ++k)
      if (pplbm_status s = grow_events(c, k, 2 * (size_t)capacity)) return s;
  }
  c->ev_used[0] = c->ev_used[1] = 0;
  return PPLBM_OK;
}

pplbm_status pplbm_kernel_times(pplbm_ctx* c, double ms[2], int64_t launches[2]) {
  if (!c || !ms || !launches) return PPLBM_ERR_ARG;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  for (int k = 0; k < 2; ++k) {
    double acc = 0.0;
    for (size_t i = 0; i + 1 < c->ev_used[k]; i += 2) {
      float t = 0.f;
      CUDA_TRY(c, cudaEventElapsedTime(&t, c->ev[k][i], c->ev[k][i + 1]));
      acc += t;
    }
    ms[k] = acc;
    launches[k] = (int64_t)(c->ev_used[k] / 2);
    c->ev_used[k] = 0;
  }
  return PPLBM_OK;
}

const char* pplbm_last_error(const pplbm_ctx* c) { return c ? c->msg.c_str() : ""; }

void pplbm_destroy(pplbm_ctx* c) {
  if (!c) return;
  if (c->dev_block) cudaFree(c->dev_block);
  for (int k = 0; k < 2; ++k)
    for (cudaEvent_t e : c->ev[k]) cudaEventDestroy(e);
  delete c;
}

}  // extern "C"
