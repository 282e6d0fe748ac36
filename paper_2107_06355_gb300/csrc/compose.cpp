// Entry points that state the problem in one call (Sec. III.A set-up: lattice,
// EOS and shaping parameters, relaxation set, G, boundary flags, initial fields),
// composed from the finer-grained calls of include/pplbm.h. Host code only.
#include <cstddef>
#include <cstdint>

#include "../../include/pplbm.h"

extern "C" {

pplbm_status pplbm_init(pplbm_ctx** out, const pplbm_lattice* lattice, const pplbm_eos_params* eos,
                        const pplbm_relax* relax, double G, const double* rho0, const double* ux0, const double* uy0,
                        void* f_workspace, size_t workspace_bytes, void* stream) {
  if (!out) return PPLBM_ERR_ARG;
  *out = nullptr;
  if (!rho0) return PPLBM_ERR_ARG;
  pplbm_ctx* c = nullptr;
  pplbm_status st = pplbm_create(&c, lattice, eos, relax, G, f_workspace, workspace_bytes, stream);
  if (st != PPLBM_OK) return st;
  st = pplbm_init_equilibrium(c, rho0, ux0, uy0);
  if (st != PPLBM_OK) {
    pplbm_destroy(c);
    return st;
  }
  *out = c;
  return PPLBM_OK;
}

pplbm_status pplbm_batch_init(pplbm_batch** out, int32_t n, const pplbm_lattice* lattices,
                              const pplbm_eos_params* eos, const pplbm_relax* relax, double G,
                              const double* const* rho0, const double* const* ux0, const double* const* uy0,
                              void* workspace, size_t workspace_bytes, void* stream) {
  if (!out) return PPLBM_ERR_ARG;
  *out = nullptr;
  if (!rho0 || n < 1) return PPLBM_ERR_ARG;
  for (int32_t i = 0; i < n; ++i)
    if (!rho0[i]) return PPLBM_ERR_ARG;
  pplbm_batch* b = nullptr;
  pplbm_status st = pplbm_batch_create(&b, n, lattices, eos, relax, G, workspace, workspace_bytes, stream);
  if (st != PPLBM_OK) return st;
  for (int32_t i = 0; i < n; ++i) {
    st = pplbm_batch_init_equilibrium(b, i, rho0[i], ux0 ? ux0[i] : nullptr, uy0 ? uy0[i] : nullptr);
    if (st != PPLBM_OK) {
      pplbm_batch_destroy(b);
      return st;
    }
  }
  *out = b;
  return PPLBM_OK;
}

pplbm_status pplbm_adjoint_segment(pplbm_ctx* ctx, const double* f_start, int64_t nsteps, double* states,
                                   const double* lambda_end, double* lambda_start, double* grad,
                                   void* adj_workspace, size_t adj_workspace_bytes) {
  if (nsteps < 1) return PPLBM_ERR_ARG;
  return pplbm_backward_checkpointed(ctx, nsteps, nsteps, f_start, states, lambda_end, lambda_start, grad,
                                     adj_workspace, adj_workspace_bytes);
}

}  // extern "C"
