/*
 * pplbm.h -- C ABI of the GB300 pseudopotential D2Q9 lattice Boltzmann step.
 *
 * One time step of the method of Czelusniak, Mapelli, Cabezas Gomez and Wagner,
 * "Shaping the equation of state to improve numerical accuracy and stability of
 * the pseudopotential lattice Boltzmann method":
 *   density moment (Eq. Density) -> shaped equation of state (Sec. III.D, the
 *   "Smooth C-S" EOS, or plain Carnahan-Starling, Eq. CS) -> psi(rho)
 *   (Eq. InteractionPotential) -> Shan-Chen force (Eq. ShanChenForce) ->
 *   MRT collision (Eqs. OperatorMRT, MatrixMRT, RelaxationMatrix) with the Li
 *   forcing scheme (Eq. LiFS; sigma = 0 is the Guo scheme, Eq. GFS) ->
 *   streaming (Eq. LBE), periodic or half-way bounce-back walls (Sec. IV).
 * All arithmetic is IEEE double precision.
 *
 * Conventions
 *   - Fields are row-major, x fastest: element (x, y) of an nx-by-ny field is at
 *     index y*nx + x. Distributions f are 9 such planes (i = 0..8, the D2Q9
 *     order of Eq. VelocitySet), plane i at offset i*nx*ny.
 *   - The stored distribution is the pre-collision f(t) of Eq. LBE.
 *   - Every call returns a pplbm_status; PPLBM_OK is 0. On error the context
 *     (if any) keeps a message readable with pplbm_last_error(). Errors raised
 *     by kernels (non-finite or non-positive density, psi^2 <= 0) are sticky:
 *     they are read by pplbm_sync() / pplbm_guard() and returned by every later
 *     call until pplbm_destroy().
 *   - Device work is issued on the context's CUDA stream and is asynchronous
 *     unless a call says otherwise. Pointers named "device or host" are checked
 *     with cudaPointerGetAttributes: device memory is used in place; host memory
 *     is staged through the workspace and the call synchronises the stream.
 *   - Memory: the caller allocates the workspace (pplbm_workspace_bytes) and
 *     every input/output buffer; the library never frees caller memory. The
 *     context owns only a small device block for the error word and reduction
 *     partials, allocated in pplbm_create and freed in pplbm_destroy.
 */
#ifndef PPLBM_H
#define PPLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PPLBM_API_VERSION 1

typedef enum pplbm_status {
  PPLBM_OK = 0,
  PPLBM_ERR_ARG = 1,        /* invalid argument (size, flag, tau <= 1/2, null pointer ...) */
  PPLBM_ERR_EOS_SETUP = 2,  /* no Maxwell root, a_1^2 or a_3^2 <= 0, psi^2 <= 0 at set-up */
  PPLBM_ERR_CUDA = 3,       /* a CUDA runtime call failed */
  PPLBM_ERR_DIVERGED = 4,   /* a kernel met a non-finite or non-positive density or psi^2 <= 0 */
  PPLBM_ERR_TIMEOUT = 5,    /* a bounded device wait gave up */
  PPLBM_ERR_STATE = 6       /* call not valid in the context's state */
} pplbm_status;

/* Boundary flags (Sec. III.A: periodic planar tests; Sec. IV: periodic in x,
 * half-way bounce-back walls at bottom and top). x must be periodic; y is either
 * periodic or walled on both sides. */
#define PPLBM_BC_PERIODIC_X 1u
#define PPLBM_BC_PERIODIC_Y 2u
#define PPLBM_BC_WALL_BOTTOM 4u
#define PPLBM_BC_WALL_TOP 8u

/* Equation of state in use. */
#define PPLBM_EOS_CS 0      /* Carnahan-Starling with a_liq everywhere (Eq. CS) */
#define PPLBM_EOS_SMOOTH 1  /* Smooth C-S of Sec. III.D: vapour branch C-S(a_vap),
                               liquid branch C-S(a_liq) + Delta P (Sec. III.D, last part) */
#define PPLBM_EOS_PENG 2    /* Peng et al. loop (Eqs. PengEOS, PengTheta) on C-S(a_liq): the cubic
                               p_sat + theta (rho - rho_v)(rho - rho_l)(rho - rho_m), rho_m from Eq.
                               VaporLiqEq with eps = 0, theta from r_theta; meant for Guo forcing */
#define PPLBM_EOS_SMOOTH_MOD 3  /* "Modified Smooth" (Sec. IV.C): the Smooth C-S shape with p_max
                                   from Eq. VaporLiqEq with eps = 0 instead of the Maxwell rule;
                                   meant for Guo forcing */

/* Relaxation set. */
#define PPLBM_RELAX_MRT 0        /* six constant relaxation times, Eq. RelaxationMatrix */
#define PPLBM_RELAX_TWO_PHASE 1  /* Lambda = diag(1,1,1,1,1,1,1,1/tau,1/tau) with tau(rho) of
                                    Eq. RelaxationTime, tau_v = 1/2 + v_r (tau_l - 1/2) (Sec. IV) */

/* Forcing scheme. */
#define PPLBM_FORCING_GUO 0  /* Eq. GFS (the Li scheme with sigma = 0) */
#define PPLBM_FORCING_LI 1   /* Eq. LiFS */

typedef struct pplbm_lattice {
  int32_t nx, ny;   /* nodes along x and y, each >= 1; 9*nx*ny < 2^31; a single
                       lattice (pplbm_create) and the FD solver also need
                       ny <= 524,280 (their 2-D grids); a batch does not */
  uint32_t bc;      /* PPLBM_BC_* flags */
  int32_t reserved; /* must be 0 */
} pplbm_lattice;

typedef struct pplbm_eos_params {
  int32_t mode;     /* PPLBM_EOS_* */
  int32_t reserved; /* must be 0 */
  double Tr;        /* reduced temperature T/T_c, 0 < Tr < 1 */
  double a_liq;     /* C-S attraction a of the liquid branch (and of the whole EOS for PPLBM_EOS_CS) */
  double a_vap;     /* C-S attraction a of the vapour branch (PPLBM_EOS_SMOOTH) */
  double b, R;      /* C-S co-volume and gas constant (paper: b = 4, R = 1) */
  double alpha;     /* shaping parameter: p_min = p_sat - alpha (p_sat^CS - p_min^CS) (Sec. III.D) */
  double r_theta;   /* PPLBM_EOS_PENG: weight of the liquid slope in theta (Eq. PengTheta) */
} pplbm_eos_params;

typedef struct pplbm_relax {
  int32_t kind;     /* PPLBM_RELAX_* */
  int32_t forcing;  /* PPLBM_FORCING_* */
  /* PPLBM_RELAX_MRT: tau_rho, tau_e, tau_zeta (varsigma), tau_j, tau_q, tau_nu, each > 1/2 */
  double tau_rho, tau_e, tau_zeta, tau_j, tau_q, tau_nu;
  /* PPLBM_RELAX_TWO_PHASE: liquid relaxation time (> 1/2) and kinematic viscosity ratio v_r (> 0) */
  double tau_l, visc_ratio;
  double sigma;        /* Li forcing parameter, used when sigma_auto == 0 */
  int32_t sigma_auto;  /* 1: sigma = -eps/(16 G) with eps solving Eq. VaporLiqEq at the
                          Maxwell densities for the EOS in use (Sec. III.A) */
  int32_t reserved;    /* must be 0 */
  /* Surface-tension control, the technique the discussion (Sec. V) names for
     keeping the Weber number when alpha lowers the surface tension (Li & Luo,
     Phys. Rev. E 88, 053307, 2013): the source
       C = [0, 1.5 l_e tr Q, -1.5 l_zeta tr Q, 0, 0, 0, 0, -l_nu (Q_xx - Q_yy), -l_nu Q_xy]
     (rows of Eq. MatrixMRT, l_k the relaxation rates of Eq. RelaxationMatrix) is
     added to m*, with Q_ab = kappa (G/2) psi(x) sum_i w_i [psi(x + c_i) - psi(x)] c_ia c_ib
     over the Shan-Chen stencil (wall ghosts as for the force). The coexistence
     densities (Eq. VaporLiqEq) are unchanged and the surface tension of Eq.
     IntegralSurfaceTension scales by (1 - kappa). 0 = off (the step is then
     bitwise the plain one); finite and < 1, else PPLBM_ERR_ARG. The adjoint
     (unit relaxation times) differentiates through it. */
  double kappa;
} pplbm_relax;

/* Everything the device needs about the EOS, computed by pplbm_eos_setup. */
typedef struct pplbm_eos_derived {
  int32_t mode, reserved;
  double G;                  /* interaction parameter (paper: -1) */
  double b, R;
  double a_l, a_v;           /* C-S a of the liquid / vapour branch */
  double Tc_l, Tc_v;         /* exact C-S critical temperatures for a_l, a_v */
  double T_l, T_v;           /* Tr * Tc_l, Tr * Tc_v */
  double rho_v, rho_l;       /* Maxwell coexistence densities (Eq. MaxwellRule) */
  double p_sat;              /* saturation pressure of the EOS in use */
  double p_sat_cs;           /* Maxwell pressure of C-S(a_l) */
  double rho_max, rho_min;   /* C-S spinodal densities (extrema of the vdW loop) */
  double p_min_cs;           /* C-S(a_l) pressure at rho_min */
  double p_max, p_min;       /* shaped-loop extrema (Sec. III.D) */
  double dP;                 /* liquid-branch shift p_sat(a_v) - p_sat(a_l) */
  double dpdrho_v, dpdrho_l; /* bulk-branch slopes at rho_v and rho_l */
  double a1sq, b1;           /* region-1 ellipse */
  double a3sq, b3;           /* region-3 ellipse */
  double eps;                /* mechanical-stability exponent solving Eq. VaporLiqEq (0 for the
                                Peng and Modified Smooth EOS, built for eps = 0) */
  double psi_v, psi_l;       /* psi(rho_v), psi(rho_l): wall ghost values (Sec. IV) */
  double rho_m, theta;       /* PPLBM_EOS_PENG: cubic root and coefficient */
} pplbm_eos_derived;

typedef struct pplbm_ctx pplbm_ctx;

/* Host-only, pure. Builds the EOS at one reduced temperature: exact critical
 * point of Eq. CS, Maxwell densities (Eq. MaxwellRule), spinodal densities,
 * p_min from alpha and p_max from the Maxwell rule of the shaped EOS
 * (Sec. III.D), and eps of Eq. VaporLiqEq by Newton's method from eps = 2
 * (Sec. III.A). G must be negative (Sec. II.B). Returns PPLBM_ERR_EOS_SETUP if
 * any step has no solution. */
pplbm_status pplbm_eos_setup(const pplbm_eos_params* params, double G, pplbm_eos_derived* out);

/* Bytes of caller-owned device workspace a lattice needs with the given
 * relaxation set: two distribution buffers (9 planes each), psi (1 plane), the
 * moments the collision pass reads (3, 5 or 9 planes) and the guard's density
 * snapshot (1 plane). 0 on invalid input. */
size_t pplbm_workspace_bytes(const pplbm_lattice* lattice, const pplbm_relax* relax);

/* Creates a context for one lattice. `workspace` is device memory of at least
 * pplbm_workspace_bytes() bytes, 16-byte aligned, owned by the caller and kept
 * alive until pplbm_destroy. `stream` is a cudaStream_t (NULL = legacy default
 * stream). The distributions are undefined until pplbm_init_equilibrium or
 * pplbm_set_f. On error *out is NULL. */
pplbm_status pplbm_create(pplbm_ctx** out, const pplbm_lattice* lattice, const pplbm_eos_params* eos,
                          const pplbm_relax* relax, double G, void* workspace, size_t workspace_bytes,
                          void* stream);

/* Replaces the stream later calls are issued on. */
pplbm_status pplbm_set_stream(pplbm_ctx* ctx, void* stream);

/* f_i = f_i^eq(rho0, u0) (Sec. III.A, Eq. EquilibriumDistribution). rho0 (nx*ny
 * values, > 0) is device or host memory; ux0, uy0 likewise or NULL for zero. */
pplbm_status pplbm_init_equilibrium(pplbm_ctx* ctx, const double* rho0, const double* ux0, const double* uy0);

/* One call for the set-up of Sec. III.A: pplbm_create followed by
 * pplbm_init_equilibrium(rho0, ux0, uy0) (rho0 required; ux0, uy0 may be NULL;
 * host or device arrays of nx*ny). On failure nothing is left allocated and *out
 * is NULL. The workspace rules are those of pplbm_create. */
pplbm_status pplbm_init(pplbm_ctx** out, const pplbm_lattice* lattice, const pplbm_eos_params* eos,
                        const pplbm_relax* relax, double G, const double* rho0, const double* ux0, const double* uy0,
                        void* f_workspace, size_t workspace_bytes, void* stream);

/* Advances nsteps >= 0 time steps of Eq. LBE on the stream (asynchronous). */
pplbm_status pplbm_step(pplbm_ctx* ctx, int64_t nsteps);

/* Macroscopic fields of the current state: rho (Eq. Density), u with the F/2
 * correction (Eq. Momentum) and psi (Eq. InteractionPotential). Each output
 * (nx*ny values) is device or host memory, or NULL to skip. Overwrites the
 * moment planes of the workspace (they are rebuilt by the next step). */
pplbm_status pplbm_get_fields(pplbm_ctx* ctx, double* rho, double* ux, double* uy, double* psi);

/* Copies the current distributions (9*nx*ny values, plane-major) out of / into
 * the context; device or host memory. For checkpoint/resume. */
pplbm_status pplbm_get_f(pplbm_ctx* ctx, double* f);
pplbm_status pplbm_set_f(pplbm_ctx* ctx, const double* f);

/* Synchronises the stream, then reports the sticky device error and the number
 * of steps issued so far (steps_done may be NULL). */
pplbm_status pplbm_sync(pplbm_ctx* ctx, int64_t* steps_done);

/* Per-M-step guard (Sec. III.A: the convergence criterion of the planar tests, the
 * paragraph after Eq. PlanarIntDensity; mass; the stability test of the dynamic
 * runs, Sec. IV). First runs the density/psi pass over the current state (as the
 * next step would; the psi and moment planes are rebuilt by every step anyway),
 * then writes to the host array out[4]:
 *   out[0] = mass sum(rho) over the nodes with a finite, positive density;
 *   out[1] = max |u| with u = (j + F/2)/rho the fluid velocity of Eq. Momentum (F the
 *            Shan-Chen force of the collision pass: same stencil, wrap and wall
 *            ghosts), the same quantity pplbm_batch_guard reports;
 *   out[2] = number of nodes with a non-finite or non-positive density (excluded
 *            from the other three);
 *   out[3] = sum |rho - rho'| / sum rho, rho' the density at the previous
 *            pplbm_guard call (a snapshot plane in the workspace): called every
 *            100 steps this is the paper's residual, converged below 1e-6. -1 on the
 *            first call and after pplbm_init_equilibrium / pplbm_set_f.
 * Deterministic (fixed partition, fixed-order reduction). Synchronises the stream.
 * Returns PPLBM_ERR_DIVERGED (sticky) when out[2] > 0. */
pplbm_status pplbm_guard(pplbm_ctx* ctx, double out[4]);

/* The EOS block the context uses. */
pplbm_status pplbm_get_derived(const pplbm_ctx* ctx, pplbm_eos_derived* out);

/* One call from host data to host data: rho0 (and optional ux0, uy0) are host
 * arrays; initialises f = f^eq, advances nsteps and writes the final density to
 * the host array rho_out. Synchronous. */
pplbm_status pplbm_run_host(pplbm_ctx* ctx, const double* rho0, const double* ux0, const double* uy0,
                            int64_t nsteps, double* rho_out);

/* ---- Adjoint (reverse-mode gradients) -----------------------------------------
 * A hand-written adjoint of pplbm_step for contexts whose relaxation times are
 * all 1 (Sec. III.A) or the two-phase set of the dynamic runs (Sec. IV: rows 7, 8
 * relax with 1/tau(rho), Eq. RelaxationTime, differentiated through tau(rho) too);
 * the general six-time MRT set returns PPLBM_ERR_STATE. Gradients flow to the state and to
 * the EOS constants that the shaping parameters move (Sec. III.D):
 * grad[PPLBM_NGRAD] = dL/d{p_max, b1, 1/a1^2, a2, b2, p_min, b3, 1/a3^2, z,
 *                          k1_v, k2_v, k1_l, k2_l, k4_l, kappa},
 * with a2, b2 the cubic's coefficients, z = sigma G^2/432 the Li term's scale
 * (Eq. LiFS), and k1 = (2/G) R T, k2 = -(2/G) a, k4 = (2/G) Delta P the constants of
 * psi^2 = rho (k1 Z(rho) + k2 rho - 2/(3G)) + k4 on the vapour (v) and liquid (l)
 * C-S branches (Eq. CS, Eq. InteractionPotential), and kappa the surface-tension
 * control, pplbm_relax.kappa; its slot is computed also at kappa = 0, through the
 * source's kernels with a zero scale. pplbm_eos_constant_sensitivity
 * gives their derivatives with respect to alpha, a_vap or a_liq, so dL/dtheta =
 * sum_k grad[k] dc[k]. At fixed T_r the branch boundaries (rho_v, rho_l, rho_max,
 * rho_min) do not depend on these parameters, so the chain is exact. All pointers
 * are device memory unless noted. */
#define PPLBM_NGRAD 15

/* Bytes of the adjoint workspace (adjoint planes, lambda ping-pong, per-block partials). */
size_t pplbm_adjoint_workspace_bytes(const pplbm_lattice* lattice);
/* One adjoint step at the state f_t (9 planes): lambda_t = (d f^{t+1}/d f^t)^T lambda_next,
 * grad += (d f^{t+1}/d constants)^T lambda_next. Uses the context's psi/moment planes.
 * Asynchronous; the reduction into grad is deterministic. */
pplbm_status pplbm_adjoint_step(pplbm_ctx* ctx, const double* f_t, const double* lambda_next, double* lambda_t,
                                double* grad, void* adj_workspace, size_t adj_workspace_bytes);
/* Advances nsteps from the current state, copying f into checkpoints[k] (9*nx*ny
 * values each) before steps k*interval; ceil(nsteps/interval) slots. */
pplbm_status pplbm_forward_checkpointed(pplbm_ctx* ctx, int64_t nsteps, int64_t interval, double* checkpoints);
/* Reverse pass of a checkpointed rollout: for each segment, last first, recomputes
 * its states from the checkpoint into `segment` (interval slots of 9*nx*ny) and runs
 * the adjoint steps back through it. lambda_N = dL/df^nsteps (device or host),
 * lambda_0 = dL/df^0 (device or host); grad accumulates. sqrt(N) checkpointing:
 * interval ~ sqrt(nsteps) keeps 2 sqrt(nsteps) states and costs one extra forward pass. */
pplbm_status pplbm_backward_checkpointed(pplbm_ctx* ctx, int64_t nsteps, int64_t interval, const double* checkpoints,
                                         double* segment, const double* lambda_N, double* lambda_0, double* grad,
                                         void* adj_workspace, size_t adj_workspace_bytes);
/* The adjoint over one segment of a checkpointed rollout: from the segment's first
 * state f_start (device, 9 planes), recomputes its nsteps states into `states`
 * (nsteps slots of 9*nx*ny, device) and runs the adjoint steps back through them:
 * lambda_start = (d f^{t0+nsteps} / d f^{t0})^T lambda_end, grad += the constants'
 * adjoints. Equal to pplbm_backward_checkpointed with interval = nsteps. */
pplbm_status pplbm_adjoint_segment(pplbm_ctx* ctx, const double* f_start, int64_t nsteps, double* states,
                                   const double* lambda_end, double* lambda_start, double* grad,
                                   void* adj_workspace, size_t adj_workspace_bytes);
/* Rollouts whose fields fit in device memory (P planes per step: psi and the moment
 * planes, P = 4 with unit relaxation times -- psi, rho, jx, jy -- and P = 6 with the
 * two-phase set, which adds the stress moments of rows 7, 8; 2,000 steps of a 256^2
 * lattice with P = 4 take 4.2 GB): pplbm_forward_stored advances nsteps
 * like pplbm_step, its density passes writing psi and the moments of f^t into
 * fields + P*nx*ny*t (nsteps slots, device); pplbm_backward_stored then runs the
 * adjoint steps t = nsteps-1 ... 0 from those slots, with no recomputation and no
 * density pass of its own. Results are bitwise those of the checkpointed pair. */
pplbm_status pplbm_forward_stored(pplbm_ctx* ctx, int64_t nsteps, double* fields);
pplbm_status pplbm_backward_stored(pplbm_ctx* ctx, int64_t nsteps, const double* fields, const double* lambda_N,
                                   double* lambda_0, double* grad, void* adj_workspace, size_t adj_workspace_bytes);
/* Selects the gradient slots the adjoint calls accumulate: bit k of mask set =
 * slot k (of PPLBM_NGRAD) is computed; the others are left unchanged (0 when grad
 * starts at 0). Default: all slots. A caller that chains to one parameter can
 * clear the slots whose dc/dtheta is 0 (for alpha: the five C-S branch constants)
 * and skip their reductions. PPLBM_ERR_ARG for bits at or above PPLBM_NGRAD. */
pplbm_status pplbm_adjoint_set_slots(pplbm_ctx* ctx, uint32_t mask);
/* The chain rule to one parameter theta, behind the ABI. pplbm_adjoint_set_param
 * chooses theta (which: 0 alpha, 1 a_vap, 2 a_liq, 3 kappa, as in
 * pplbm_eos_constant_sensitivity), computes dc/dtheta at the context's own EOS
 * parameters and relaxation set with step h (host only), keeps it in the context and
 * sets the gradient slots to those with dc_k != 0 (as pplbm_adjoint_set_slots would);
 * PPLBM_ERR_ARG for another `which` or h <= 0. After the adjoint calls have filled
 * grad, pplbm_adjoint_param_gradient writes to the host out[0] = dL/dtheta =
 * sum_k grad[k] dc_k/dtheta over the selected slots, summed in slot order; grad is
 * PPLBM_NGRAD values in device or host memory (the call synchronises the stream).
 * PPLBM_ERR_STATE if no parameter was chosen. */
pplbm_status pplbm_adjoint_set_param(pplbm_ctx* ctx, int32_t which, double h);
pplbm_status pplbm_adjoint_param_gradient(pplbm_ctx* ctx, const double* grad, double* out);
/* rho0_bar = sum_i w_i lambda_0[i]: the gradient w.r.t. the initial density of
 * f^0 = f^eq(rho0, u = 0) (Sec. III.A). */
pplbm_status pplbm_adjoint_initial_density(pplbm_ctx* ctx, const double* lambda_0, double* rho0_bar);
/* Host only: the values of the PPLBM_NGRAD constants (z and kappa left 0). */
pplbm_status pplbm_eos_grad_constants(const pplbm_eos_derived* eos, double c[PPLBM_NGRAD]);
/* Host only: dc/dtheta of the PPLBM_NGRAD constants for theta = alpha (which = 0),
 * a_vap (1) or a_liq (2), including z through sigma(theta) when relax->sigma_auto,
 * by central differences of pplbm_eos_setup at steps h and h/2 combined by
 * Richardson extrapolation: D = (4 D(h/2) - D(h))/3. Error bound: the truncation
 * term is O(h^4) (the set-up is smooth in these parameters at fixed T_r); a
 * rounding or root-finding error delta in a constant adds at most 3 delta / h
 * (8 delta/h from D(h/2), delta/h from D(h), over 3). With the set-up's roots and
 * quadratures good to delta ~ 1e-15 |c| and the suggested h = 1e-4, the error is
 * about 3e-11 |c| (the tests compare h and h/2, and the oracle's own derivative).
 * For theta = kappa (3) exactly the unit vector of its slot. PPLBM_ERR_ARG for
 * another `which` or h <= 0. */
pplbm_status pplbm_eos_constant_sensitivity(const pplbm_eos_params* params, double G, const pplbm_relax* relax,
                                            int32_t which, double h, double dc[PPLBM_NGRAD]);

/* ---- Finite-difference solver of the same macroscopic equations (App. A) ----
 * The MacCormack scheme the paper uses as its reference for dynamics: predictor
 * with forward, corrector with backward first differences; central second
 * differences and central differences for every derivative of psi (Eqs.
 * FDmomentum, FDstressTensor, FDviscosityDerivative, FDforce). Periodic grids
 * only (App. B's wall conditions are not provided). State: rho, u_x, u_y planes
 * (x fastest); grid spacing dx in lattice units; eps is the EOS set-up's. */
typedef struct pplbm_fd pplbm_fd;
/* Caller-owned device workspace: 8 planes (state, predictor state, psi, p) of nx*ny
 * values, nx*(ny + 4) with walls; 0 for a grid or boundary flags pplbm_fd_create rejects. */
size_t pplbm_fd_workspace_bytes(const pplbm_lattice* lattice);
/* lattice->bc is PPLBM_BC_PERIODIC_X | PPLBM_BC_PERIODIC_Y, or PPLBM_BC_PERIODIC_X
 * with both walls (ny >= 2): the wall layers of the grid-dependency appendix (Eqs.
 * B1, B2) -- at the bottom a no-slip layer on the wall whose density and psi are
 * extrapolated linearly from the first two fluid rows and a layer in the solid with
 * psi_b2 = psi_b1 + 2 dx (psi_l - psi_b1); at the top reflexive layers (density and
 * psi mirrored, velocity reversed). The fluid rows are at y = 0, dx, ..., and the
 * bottom wall at y = -dx. tau_nu > 1/2 and tau_e > 0 give mu = rho (tau_nu - 1/2)/3
 * and mu_B = rho (tau_e - tau_nu)/3. The workspace holds 8 planes of nx*ny values,
 * nx*(ny + 4) with walls (pplbm_fd_workspace_bytes). */
pplbm_status pplbm_fd_create(pplbm_fd** out, const pplbm_lattice* lattice, const pplbm_eos_params* eos, double G,
                             double tau_nu, double tau_e, double dx, void* workspace, size_t workspace_bytes,
                             void* stream);
/* Replaces the constant tau_nu by tau_nu(rho) of Eq. RelaxationTime, linear in rho
 * from tau_v = 1/2 + visc_ratio (tau_l - 1/2) at rho_v to tau_l at rho_l (the Maxwell
 * densities), in the viscosities of Eq. DynamicViscosity and their density
 * derivatives (Eq. FDviscosityDerivative); tau_e stays. tau_l > 1/2, visc_ratio > 0. */
pplbm_status pplbm_fd_set_two_phase_viscosity(pplbm_fd* fd, double tau_l, double visc_ratio);
/* The surface-tension control of pplbm_relax.kappa, as the macroscopic equations
 * see it: the pressure tensor of Eq. FDforce gains its second-order counterpart
 * (kappa G/6) psi (delta_ab lap psi - d_a d_b psi), whose divergence
 * (kappa G/6) [(d_a psi) lap psi - (d_g psi)(d_a d_g psi)] has no third
 * derivative. kappa finite and < 1 (0 = off), else PPLBM_ERR_ARG. Applies from the
 * next pplbm_fd_step. */
pplbm_status pplbm_fd_set_surface_tension(pplbm_fd* fd, double kappa);
/* Copies the state in / out (device or host pointers; NULL skips an output). Synchronous. */
pplbm_status pplbm_fd_set_state(pplbm_fd* fd, const double* rho, const double* ux, const double* uy);
pplbm_status pplbm_fd_get_state(pplbm_fd* fd, double* rho, double* ux, double* uy);
/* nsteps MacCormack steps of size dt (the paper uses dt = 0.8 dx^2 for v_r = 1). Asynchronous. */
pplbm_status pplbm_fd_step(pplbm_fd* fd, int64_t nsteps, double dt);
pplbm_status pplbm_fd_sync(pplbm_fd* fd);
void pplbm_fd_destroy(pplbm_fd* fd);

/* ---- Batched engine: many independent lattices advanced together ----------
 * The instances may differ in size, boundary flags, EOS parameters (e.g. a sweep
 * of reduced temperatures) and relaxation times, but must share one collision
 * kind (all tau = 1; only tau_nu or the two-phase tau(rho) relaxing; or general
 * MRT). Work is partitioned by 256-node blocks and 256-thread tiles across all
 * instances, so one launch per pass covers the whole batch; the per-node
 * arithmetic is the single-lattice step's, and a batched step is bitwise equal
 * to stepping each lattice alone. */
typedef struct pplbm_batch pplbm_batch;

#define PPLBM_PLAN_LAUNCHES 0    /* two launches per step covering all instances */
#define PPLBM_PLAN_GRAPH 1       /* the same launches, two steps per replayed CUDA graph */
#define PPLBM_PLAN_PERSISTENT 2  /* one cooperative launch per call; bounded grid barriers
                                    between the passes (PPLBM_ERR_TIMEOUT if a wait gives up) */
#define PPLBM_PLAN_PIPELINED 3   /* the instances in two groups of about equal node counts, the
                                    second half a step behind the first within a call: every
                                    launch runs one group's density pass with the other's
                                    collision pass (the FP64-bound and the integer-bound pass
                                    share the SMs); 2 nsteps + 1 launches per call, two-step
                                    CUDA graphs in between; every instance ends the call at the
                                    same step; each launch is a resident grid whose blocks take
                                    the work items in order from a device counter */

typedef struct pplbm_batch_plan {
  int32_t mode;        /* PPLBM_PLAN_* */
  int32_t tile_width;  /* collision tile width; 0 = per instance, the power of two in [4, 256]
                          wasting the fewest threads on partial tiles */
  int32_t k1_blocks;   /* work items of the density/psi pass */
  int32_t k2_tiles;    /* work items of the collision pass */
  double ms_launches, ms_graph, ms_persistent;  /* per-step times measured by the autotuner (0 if not) */
  double ms_chosen;
  double ms_pipelined;                          /* the pipelined plan's, likewise */
} pplbm_batch_plan;

/* Workspace bytes for n instances: per instance two f buffers, psi, the moment
 * planes of the collision kind and a density snapshot for pplbm_batch_guard
 * (each instance's block is 256-byte aligned);
 * 0 if any lattice or relaxation set is invalid or the collision kinds differ. */
size_t pplbm_batch_workspace_bytes(int32_t n, const pplbm_lattice* lattices, const pplbm_relax* relax);

/* Creates a batch over caller-owned device workspace (256-byte aligned). eos and
 * relax are arrays of n; each EOS is set up as in pplbm_eos_setup. The batch owns
 * a small device block (instance table, work-item tables, barrier, error word)
 * and a capture stream. Initial plan: PPLBM_PLAN_LAUNCHES, per-instance tiles. */
pplbm_status pplbm_batch_create(pplbm_batch** out, int32_t n, const pplbm_lattice* lattices,
                                const pplbm_eos_params* eos, const pplbm_relax* relax, double G, void* workspace,
                                size_t workspace_bytes, void* stream);
/* As pplbm_init_equilibrium, for instance i. Synchronises. */
pplbm_status pplbm_batch_init_equilibrium(pplbm_batch* b, int32_t i, const double* rho0, const double* ux0,
                                          const double* uy0);
/* pplbm_batch_create followed by pplbm_batch_init_equilibrium for every instance:
 * rho0[i] (required), ux0[i], uy0[i] (ux0, uy0 or their entries may be NULL) are
 * instance i's arrays. On failure nothing is left allocated and *out is NULL. */
pplbm_status pplbm_batch_init(pplbm_batch** out, int32_t n, const pplbm_lattice* lattices,
                              const pplbm_eos_params* eos, const pplbm_relax* relax, double G,
                              const double* const* rho0, const double* const* ux0, const double* const* uy0,
                              void* workspace, size_t workspace_bytes, void* stream);
/* Advances every instance by nsteps (asynchronous). */
pplbm_status pplbm_batch_step(pplbm_batch* b, int64_t nsteps);
/* As pplbm_get_fields / pplbm_get_f / pplbm_set_f, for instance i. */
pplbm_status pplbm_batch_get_fields(pplbm_batch* b, int32_t i, double* rho, double* ux, double* uy, double* psi);
pplbm_status pplbm_batch_get_f(pplbm_batch* b, int32_t i, double* f);
pplbm_status pplbm_batch_set_f(pplbm_batch* b, int32_t i, const double* f);
/* Fixes the plan: mode PPLBM_PLAN_*, tile_width 0 (per instance) or a power of two in [4, 256]. */
pplbm_status pplbm_batch_set_plan(pplbm_batch* b, int32_t mode, int32_t tile_width);
pplbm_status pplbm_batch_get_plan(const pplbm_batch* b, pplbm_batch_plan* out);
/* Times trial_steps (>= 2) steps of each mode with per-instance and width-32 tiles
 * on the current state, in three interleaved rounds keeping each candidate's best
 * time, keeps the fastest plan and restores the state (it allocates a temporary copy
 * of every instance's distributions). The plan's ms_* fields get each mode's best
 * per-step time. Synchronises. */
pplbm_status pplbm_batch_autotune(pplbm_batch* b, int32_t trial_steps, pplbm_batch_plan* chosen);
/* Synchronises; sticky device error (PPLBM_ERR_DIVERGED / PPLBM_ERR_TIMEOUT) and steps issued. */
pplbm_status pplbm_batch_sync(pplbm_batch* b, int64_t* steps_done);
pplbm_status pplbm_batch_get_derived(const pplbm_batch* b, int32_t i, pplbm_eos_derived* out);
/* Timing aid: with capacity > 0, each pplbm_batch_step call is bracketed by CUDA
 * events; pplbm_batch_times synchronises and returns the summed milliseconds and
 * steps since the previous call, then resets. */
pplbm_status pplbm_batch_enable_timing(pplbm_batch* b, int64_t capacity);
pplbm_status pplbm_batch_times(pplbm_batch* b, double* ms, int64_t* steps);
/* Per-pass timing aid (for the roofline of each kernel). With capacity > 0, every
 * launch of either pass is bracketed by CUDA events on the batch's stream: under the
 * launches plan as two plain launches per step (events for `capacity` steps are
 * created here, more on demand); under the graph plan by event-record nodes inside
 * ceil(capacity/2) two-step graphs per parity built here, each replayed at most once
 * between two pplbm_batch_pass_times calls (steps beyond them run as timed plain
 * launches). PPLBM_ERR_STATE under the persistent plan, whose passes share one
 * launch, and under the pipelined plan, whose launches mix the passes. capacity = 0
 * turns it off. The autotuner times every plan without these events and turns them
 * off if it keeps the persistent or the pipelined plan. pplbm_batch_pass_times
 * synchronises and returns, since the previous call, the summed milliseconds and
 * launch counts of the density/psi pass (index 0) and of the collision pass (index
 * 1), then resets them. */
pplbm_status pplbm_batch_enable_pass_timing(pplbm_batch* b, int64_t capacity);
pplbm_status pplbm_batch_pass_times(pplbm_batch* b, double ms[2], int64_t launches[2]);
/* Failure-detection self-test of the persistent kernel's bounded grid barrier:
 * launches one step in which one block leaves without arriving, with waits
 * limited to spin_limit sleeps of ~100 ns; returns PPLBM_ERR_TIMEOUT when the
 * others' waits ran out and were reported (the expected outcome). The waits give
 * up before the collision pass, so the distributions are not touched; the error
 * word is cleared and the batch stays usable. Synchronises. */
pplbm_status pplbm_batch_barrier_selftest(pplbm_batch* b, uint32_t spin_limit);
/* Divergence isolation for sweeps: with on != 0, an instance whose kernels meet a
 * non-finite or non-positive density (or psi^2 <= 0) is marked diverged but does
 * not make the batch's status sticky, so the other instances keep stepping (a
 * diverged instance keeps computing on its non-finite state, touching nothing
 * else). Off by default: any divergence stops the batch. */
pplbm_status pplbm_batch_set_isolation(pplbm_batch* b, int32_t on);
/* Synchronises and writes, per instance, PPLBM_OK or PPLBM_ERR_DIVERGED into
 * status[n] (host); returns the batch status. */
pplbm_status pplbm_batch_instance_status(pplbm_batch* b, int32_t* status);
/* One call from host data to host data for the whole batch: rho0[i] and
 * rho_out[i] are host arrays of instance i's nx*ny densities (pinned memory gives
 * the fastest copies). Sets f = f^eq(rho0[i], 0) for every instance, advances
 * nsteps with the current plan and writes the final densities (the density
 * pass's rho, Eq. Density) to rho_out. Synchronous; returns the batch status. */
pplbm_status pplbm_batch_run_host(pplbm_batch* b, const double* const* rho0, int64_t nsteps,
                                  double* const* rho_out);
/* Per-instance guard (Sec. III.A convergence check, mass and the stability test of
 * the dynamic runs, Sec. IV). First runs the density/psi pass over every
 * instance's current state (as the next step would), then writes to the host
 * array out[4 n], for instance i, out[4i] = mass sum(rho), out[4i+1] = max |u|
 * with u = (j + F/2)/rho the fluid velocity (Eq. Momentum; F the Shan-Chen force
 * of the collision pass), out[4i+2] = number of nodes with a non-finite or
 * non-positive density (excluded from the other three; such a node also marks
 * the instance diverged, as a step would), and
 * out[4i+3] = sum |rho - rho'| / sum rho, where rho' is the density at the
 * previous pplbm_batch_guard call, or -1 on the first call for the instance and
 * after its pplbm_batch_init_equilibrium / pplbm_batch_set_f. rho' lives in the
 * instance's workspace block. Deterministic (fixed-order) reduction; runs in the
 * batch's stream and synchronises it. Returns the batch status. */
pplbm_status pplbm_batch_guard(pplbm_batch* b, double* out);
const char* pplbm_batch_last_error(const pplbm_batch* b);
void pplbm_batch_destroy(pplbm_batch* b);

/* Self-test of the double-precision reciprocal and square root the step kernels
 * use in place of IEEE division and sqrt (a hardware seed refined by one
 * third-order series step). Evaluates n pseudo-random x = m 2^k (m in [1, 2),
 * |k| <= 60) and writes to the device array out[2] the largest relative error
 * against CUDA's correctly rounded 1/x (out[0]) and sqrt(x) (out[1]).
 * Asynchronous on `stream`. */
pplbm_status pplbm_fp64_selftest(long long n, unsigned long long seed, double* out, void* stream);

/* Self-test of the integer-pipe additions the step kernels use to unload the FP64
 * pipe (software IEEE 754 round-to-nearest-even adds, bitwise equal to the FP64
 * pipe's): the positive-operand sum of the density pass and the signed add of the
 * collision pass. Evaluates n seeded pairs (independent exponents, exponent gaps
 * 0..63, half-way ties, rounding carries; for the signed add every sign combination
 * and operands 0..7 ulp apart) and writes to the device array out[5]: out[0] = the
 * number of results that differ from the FP64 add in any bit, out[1..4] = the first
 * such pair and the two results (bit patterns). Asynchronous on `stream`. */
pplbm_status pplbm_int_add_selftest(long long n, unsigned long long seed, unsigned long long* out, void* stream);

/* The fixed-point sums of the step kernels, evaluated on caller data (a check of
 * the device build against other builds of the same source): the density moments
 * of Eqs. Density and Momentum and, for the two-phase set, rows 7 and 8 of Eq.
 * MatrixMRT, and the Shan-Chen stencil sums of Eq. ShanChenForce. Each sum is exact
 * in one 64-bit fixed-point frame anchored at its largest operand and rounded once
 * to nearest. Device arrays: f (n x 9 populations, row-major), p (n x 8 psi values
 * pE, pW, pN, pS, pNE, pNW, pSW, pSE), out (n x 8): rho, jx, jy, m7, m8, a flag,
 * gx, gy. The flag is 1.0 when the nine populations are positive normal doubles
 * below 2^1008 (the domain of the fixed-point moments); otherwise it is 0.0 and so
 * are the five moments. gx, gy are NaN for an infinite, NaN or negative psi.
 * PPLBM_ERR_ARG for n < 0, n > 2^31 * 255, or NULL pointers with n > 0.
 * Asynchronous on `stream`. */
pplbm_status pplbm_fixsum_eval(long long n, const double* f, const double* p, double* out, void* stream);

/* The fixed-point parts of the collision pass, evaluated on caller data (a check of
 * the device build against other builds of the same source): per row, the nine
 * post-collision populations of the reduced collision (Eqs. OperatorMRT, LiFS with
 * Lambda = I; with shear != 0 also the rows 7, 8 corrections of the two-phase set,
 * Eq. RelaxationTime) from q (n x 9: rho/36, Pi_xx/36, Pi_yy/36, Pi_xy/36, P_x/36,
 * P_y/36, the Li term zz, and the rows 7, 8 corrections, read only when shear != 0),
 * and the sums j + h, j + 2h, j + 3h, j - h of jh (n x 2: j, h). Device arrays;
 * out (n x 13): the nine populations, then the four sums. PPLBM_ERR_ARG for n < 0,
 * n > 2^31 * 255, or NULL pointers with n > 0. Asynchronous on `stream`. */
pplbm_status pplbm_fixsum_collision_eval(long long n, int32_t shear, const double* q, const double* jh, double* out,
                                         void* stream);

/* The reverse-mode counterparts of pplbm_fixsum_collision_eval's stages, and the
 * fixed-point sums of the adjoint's density pass, on caller data: per row, from mu
 * (n x 9, the adjoints of the nine post-collision populations) the adjoints of the
 * populations' nine inputs (rho/36, Pi_xx/36, Pi_yy/36, Pi_xy/36, P_x/36, P_y/36, zz
 * and, when shear != 0, the rows 7, 8 corrections; 0.0 otherwise); from a (n x 6: the
 * adjoints of j + h, j + 2h, j + 3h, j - h, and partial adjoints of j and h) the
 * adjoints of j and h; from gth (n x 13: a node's own psi adjoint, then gx_bar, gy_bar
 * at its W, E / S, N / SW, NE, NW, SE neighbours as x, y pairs) the gathered psi
 * adjoint (the transpose of the Shan-Chen stencil, Eq. ShanChenForce); from lam (n x
 * 5: rho_bar, jx_bar, jy_bar, m7_bar, m8_bar) the nine lambda_i = rho_bar + c_i . j_bar
 * (+ with shear the rows 7, 8 terms). Device arrays; out (n x 21): the nine, the two,
 * the gathered adjoint, the nine lambdas. PPLBM_ERR_ARG for n < 0, n > 2^31 * 255, or
 * NULL pointers with n > 0. Asynchronous on `stream`. */
pplbm_status pplbm_fixsum_adjoint_eval(long long n, int32_t shear, const double* mu, const double* a,
                                       const double* gth, const double* lam, double* out, void* stream);

/* FP64 issue-rate probe, the denominator of the step's arithmetic roofline (the
 * step's per-node arithmetic is double precision throughout, Sec. II; on this GPU
 * the FP64 pipe, not memory, bounds it). Launches blocks_per_sm x (SM count)
 * blocks of 256 threads; each thread runs `iters` rounds of `chains` (1, 2, 4, 8,
 * 16 or 32) independent chains of one FP64 operation: op 0 fused multiply-add,
 * 1 add, 2 multiply; op 3 runs chains of the integer-pipe addition the step kernels
 * use instead, op 4 one FMA and one integer-pipe addition per chain and round (the
 * same time as op 0 means the two pipes overlap); op 5 runs chains of 64-bit
 * integer to double conversions (round to nearest), op 6 of double to 64-bit
 * integer conversions (toward zero), each with a 64-bit integer add or XOR that
 * feeds the result back. Times the launch with CUDA events on `stream` and
 * synchronises it. Writes to host out[3]: out[0] = FP64 instructions per second
 * (op 3: integer-pipe additions, ops 5, 6: conversions per second; counted per
 * thread, as the step's per-node instruction counts are), out[1] = the launch's
 * milliseconds, out[2] = blocks launched. `sink` is one device double
 * the kernel may write (it never does for these inputs; it keeps the chains from
 * being optimised away). PPLBM_ERR_ARG for blocks_per_sm outside [1, 64], another
 * chain count or op, iters < 1 or NULL pointers. */
pplbm_status pplbm_fp64_peak(int32_t blocks_per_sm, int32_t chains, int32_t op, long long iters, double* sink,
                             double* out, void* stream);

/* Kernel timing, a profiling aid. With capacity > 0, pplbm_step records a CUDA
 * event pair around every launch of the two step kernels on the context's
 * stream; events for `capacity` launches of each kernel are created here, outside
 * any timed region (more are created on demand). capacity = 0 disables timing.
 * pplbm_kernel_times synchronises the stream and returns, since the previous
 * call, the summed device durations in milliseconds and the launch counts of the
 * density/psi pass (index 0) and the collision/streaming pass (index 1), then
 * resets them. */
pplbm_status pplbm_enable_kernel_timing(pplbm_ctx* ctx, int64_t capacity);
pplbm_status pplbm_kernel_times(pplbm_ctx* ctx, double ms[2], int64_t launches[2]);

/* One time step, f_out = step(f_in), that allocates no device memory. The paper
 * has no counterpart: this exists for callers that cannot call cudaMalloc, such
 * as code inside a host framework that owns all device memory through its own
 * pool or budget, or code on a latency-critical stream where cudaMalloc/cudaFree
 * would synchronise the device. There is no context: the caller passes the
 * lattice, an EOS block from pplbm_eos_setup (host only; any PPLBM_EOS_* mode),
 * the relaxation set and two non-overlapping device buffers of 9*nx*ny values
 * (plane-major; overlapping ranges return PPLBM_ERR_ARG); psi and the
 * moment planes live in a static device array inside the library, so
 * nx*ny <= 65536 (larger lattices return PPLBM_ERR_ARG with a message saying so).
 *  - The array (5.2 MB) is held by every GPU that loads the library until the
 *    process exits. Its address is looked up once per device, by the first call
 *    made while that device is current; make that first call before any stream
 *    capture. The address is kept for the life of the process: after a
 *    cudaDeviceReset() on that device this entry point must not be called.
 *  - Every call uses the same array: calls that overlap on the GPU (other
 *    streams, other threads) race and give undefined results. The error word in
 *    it is cleared at the start of each call.
 *  - Synchronises `stream` (cudaStream_t, NULL = legacy default stream) to read
 *    the error word; returns PPLBM_ERR_DIVERGED for a non-finite or non-positive
 *    density or psi^2 <= 0. `message` (may be NULL) receives a static string
 *    describing a failure, "" on success. */
pplbm_status pplbm_step_noalloc(const pplbm_lattice* lattice, const pplbm_eos_derived* eos,
                                const pplbm_relax* relax, const double* f_in, double* f_out, void* stream,
                                const char** message);

/* Message of the last error on this context ("" if none); valid until the next call. */
const char* pplbm_last_error(const pplbm_ctx* ctx);
const char* pplbm_status_string(pplbm_status status);

/* Frees the context's own device block. Does not touch caller memory. */
void pplbm_destroy(pplbm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* PPLBM_H */
