// The context behind pplbm_ctx (shared by the library's translation units).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "internal.h"

using pplbm::StepArgs;

struct pplbm_ctx {
  pplbm_lattice lat;
  pplbm_relax relax;
  pplbm_eos_params eos_params;  // as given to pplbm_create (the adjoint's chain rule needs them)
  pplbm_eos_derived eos;
  double G;
  int64_t n;
  int nmom;
  double* fA;  // current f(t)
  double* fB;  // next f(t+1); scratch between steps (host staging)
  double* psi;
  double* mom;
  double* snap;     // density at the previous pplbm_guard call (workspace plane)
  bool snap_valid;  // snap holds a density of this state's history
  cudaStream_t stream;
  void* dev_block;  // owned: error word + guard partials + guard output (4 values)
  int* d_err;
  double* d_partials;
  double* d_guard;
  int64_t steps;
  pplbm_status sticky;
  std::string msg;
  StepArgs args;
  // kernel timing: event pairs recorded around each launch while enabled
  bool timing;
  std::vector<cudaEvent_t> ev[2];  // per kernel: start/stop interleaved
  size_t ev_used[2];
  uint32_t adj_slots = ~0u;  // adjoint: bit k set = gradient slot k is accumulated
  // adjoint chain rule: dc_k/dtheta of the parameter chosen by pplbm_adjoint_set_param
  double adj_dc[PPLBM_NGRAD] = {};
  int adj_param = -1;  // -1: none chosen
};
