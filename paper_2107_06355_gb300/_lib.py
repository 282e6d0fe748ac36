"""ctypes binding of include/pplbm.h (argument marshalling only).

Every function of the C ABI is exposed under its C name on the object returned
by :func:`lib`. Struct layouts mirror the header exactly. Loading fails loudly if
the in-tree library has not been built; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpplbm.so")

PPLBM_OK = 0
PPLBM_ERR_ARG = 1
PPLBM_ERR_EOS_SETUP = 2
PPLBM_ERR_CUDA = 3
PPLBM_ERR_DIVERGED = 4
PPLBM_ERR_TIMEOUT = 5
PPLBM_ERR_STATE = 6

BC_PERIODIC_X = 1
BC_PERIODIC_Y = 2
BC_WALL_BOTTOM = 4
BC_WALL_TOP = 8
BC_PERIODIC = BC_PERIODIC_X | BC_PERIODIC_Y
BC_WALLS_Y = BC_PERIODIC_X | BC_WALL_BOTTOM | BC_WALL_TOP

EOS_CS = 0
EOS_SMOOTH = 1
EOS_PENG = 2
EOS_SMOOTH_MOD = 3
RELAX_MRT = 0
RELAX_TWO_PHASE = 1
FORCING_GUO = 0
FORCING_LI = 1


class pplbm_lattice(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("bc", C.c_uint32), ("reserved", C.c_int32)]


class pplbm_eos_params(C.Structure):
    _fields_ = [("mode", C.c_int32), ("reserved", C.c_int32), ("Tr", C.c_double), ("a_liq", C.c_double),
                ("a_vap", C.c_double), ("b", C.c_double), ("R", C.c_double), ("alpha", C.c_double),
                ("r_theta", C.c_double)]


class pplbm_relax(C.Structure):
    _fields_ = [("kind", C.c_int32), ("forcing", C.c_int32),
                ("tau_rho", C.c_double), ("tau_e", C.c_double), ("tau_zeta", C.c_double),
                ("tau_j", C.c_double), ("tau_q", C.c_double), ("tau_nu", C.c_double),
                ("tau_l", C.c_double), ("visc_ratio", C.c_double),
                ("sigma", C.c_double), ("sigma_auto", C.c_int32), ("reserved", C.c_int32),
                ("kappa", C.c_double)]


_DERIVED_DOUBLES = ["G", "b", "R", "a_l", "a_v", "Tc_l", "Tc_v", "T_l", "T_v", "rho_v", "rho_l", "p_sat",
                    "p_sat_cs", "rho_max", "rho_min", "p_min_cs", "p_max", "p_min", "dP", "dpdrho_v",
                    "dpdrho_l", "a1sq", "b1", "a3sq", "b3", "eps", "psi_v", "psi_l", "rho_m", "theta"]


class pplbm_eos_derived(C.Structure):
    _fields_ = [("mode", C.c_int32), ("reserved", C.c_int32)] + [(n, C.c_double) for n in _DERIVED_DOUBLES]

    def as_dict(self):
        d = {n: getattr(self, n) for n in _DERIVED_DOUBLES}
        d["mode"] = self.mode
        return d


class pplbm_batch_plan(C.Structure):
    _fields_ = [("mode", C.c_int32), ("tile_width", C.c_int32), ("k1_blocks", C.c_int32), ("k2_tiles", C.c_int32),
                ("ms_launches", C.c_double), ("ms_graph", C.c_double), ("ms_persistent", C.c_double),
                ("ms_chosen", C.c_double), ("ms_pipelined", C.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


NGRAD = 15
GRAD_NAMES = ("p_max", "b1", "inv_a1sq", "a2", "b2", "p_min", "b3", "inv_a3sq", "zz_scale",
              "k1_v", "k2_v", "k1_l", "k2_l", "k4_l", "kappa")
# parameters pplbm_eos_constant_sensitivity differentiates by (its `which`); kappa
# belongs to the relaxation set (Relax.kappa), the others to the EOS
SENS_PARAMS = {"alpha": 0, "a_vap": 1, "a_liq": 2, "kappa": 3}

PLAN_LAUNCHES = 0
PLAN_GRAPH = 1
PLAN_PERSISTENT = 2
PLAN_PIPELINED = 3

_P = C.c_void_p
_D = C.POINTER(C.c_double)
_SIGS = {
    "pplbm_eos_setup": (C.c_int, [C.POINTER(pplbm_eos_params), C.c_double, C.POINTER(pplbm_eos_derived)]),
    "pplbm_workspace_bytes": (C.c_size_t, [C.POINTER(pplbm_lattice), C.POINTER(pplbm_relax)]),
    "pplbm_create": (C.c_int, [C.POINTER(_P), C.POINTER(pplbm_lattice), C.POINTER(pplbm_eos_params),
                               C.POINTER(pplbm_relax), C.c_double, _P, C.c_size_t, _P]),
    "pplbm_set_stream": (C.c_int, [_P, _P]),
    "pplbm_init_equilibrium": (C.c_int, [_P, _P, _P, _P]),
    "pplbm_step": (C.c_int, [_P, C.c_int64]),
    "pplbm_get_fields": (C.c_int, [_P, _P, _P, _P, _P]),
    "pplbm_get_f": (C.c_int, [_P, _P]),
    "pplbm_set_f": (C.c_int, [_P, _P]),
    "pplbm_sync": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "pplbm_guard": (C.c_int, [_P, _D]),
    "pplbm_get_derived": (C.c_int, [_P, C.POINTER(pplbm_eos_derived)]),
    "pplbm_run_host": (C.c_int, [_P, _P, _P, _P, C.c_int64, _P]),
    "pplbm_enable_kernel_timing": (C.c_int, [_P, C.c_int64]),
    "pplbm_kernel_times": (C.c_int, [_P, _D, C.POINTER(C.c_int64)]),
    "pplbm_step_noalloc": (C.c_int, [C.POINTER(pplbm_lattice), C.POINTER(pplbm_eos_derived),
                                     C.POINTER(pplbm_relax), _P, _P, _P, C.POINTER(C.c_char_p)]),
    "pplbm_fp64_selftest": (C.c_int, [C.c_longlong, C.c_ulonglong, _P, _P]),
    "pplbm_fp64_peak": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_longlong, _P, _D, _P]),
    "pplbm_int_add_selftest": (C.c_int, [C.c_longlong, C.c_ulonglong, _P, _P]),
    "pplbm_fixsum_eval": (C.c_int, [C.c_longlong, _P, _P, _P, _P]),
    "pplbm_fixsum_collision_eval": (C.c_int, [C.c_longlong, C.c_int32, _P, _P, _P, _P]),
    "pplbm_fixsum_adjoint_eval": (C.c_int, [C.c_longlong, C.c_int32, _P, _P, _P, _P, _P, _P]),
    "pplbm_batch_workspace_bytes": (C.c_size_t, [C.c_int32, C.POINTER(pplbm_lattice), C.POINTER(pplbm_relax)]),
    "pplbm_batch_create": (C.c_int, [C.POINTER(_P), C.c_int32, C.POINTER(pplbm_lattice), C.POINTER(pplbm_eos_params),
                                     C.POINTER(pplbm_relax), C.c_double, _P, C.c_size_t, _P]),
    "pplbm_batch_init_equilibrium": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "pplbm_batch_step": (C.c_int, [_P, C.c_int64]),
    "pplbm_batch_get_fields": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P]),
    "pplbm_batch_get_f": (C.c_int, [_P, C.c_int32, _P]),
    "pplbm_batch_set_f": (C.c_int, [_P, C.c_int32, _P]),
    "pplbm_batch_set_plan": (C.c_int, [_P, C.c_int32, C.c_int32]),
    "pplbm_batch_get_plan": (C.c_int, [_P, C.POINTER(pplbm_batch_plan)]),
    "pplbm_batch_autotune": (C.c_int, [_P, C.c_int32, C.POINTER(pplbm_batch_plan)]),
    "pplbm_batch_sync": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "pplbm_batch_get_derived": (C.c_int, [_P, C.c_int32, C.POINTER(pplbm_eos_derived)]),
    "pplbm_batch_enable_timing": (C.c_int, [_P, C.c_int64]),
    "pplbm_batch_times": (C.c_int, [_P, _D, C.POINTER(C.c_int64)]),
    "pplbm_batch_enable_pass_timing": (C.c_int, [_P, C.c_int64]),
    "pplbm_batch_pass_times": (C.c_int, [_P, _D, C.POINTER(C.c_int64)]),
    "pplbm_batch_barrier_selftest": (C.c_int, [_P, C.c_uint32]),
    "pplbm_batch_set_isolation": (C.c_int, [_P, C.c_int32]),
    "pplbm_batch_instance_status": (C.c_int, [_P, C.POINTER(C.c_int32)]),
    "pplbm_batch_guard": (C.c_int, [_P, C.POINTER(C.c_double)]),
    "pplbm_adjoint_set_slots": (C.c_int, [_P, C.c_uint32]),
    "pplbm_adjoint_set_param": (C.c_int, [_P, C.c_int32, C.c_double]),
    "pplbm_adjoint_param_gradient": (C.c_int, [_P, _P, _D]),
    "pplbm_fd_set_two_phase_viscosity": (C.c_int, [_P, C.c_double, C.c_double]),
    "pplbm_fd_set_surface_tension": (C.c_int, [_P, C.c_double]),
    "pplbm_forward_stored": (C.c_int, [_P, C.c_int64, _P]),
    "pplbm_backward_stored": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P, _P, C.c_size_t]),
    "pplbm_init": (C.c_int, [C.POINTER(_P), C.POINTER(pplbm_lattice), C.POINTER(pplbm_eos_params),
                             C.POINTER(pplbm_relax), C.c_double, _P, _P, _P, _P, C.c_size_t, _P]),
    "pplbm_batch_init": (C.c_int, [C.POINTER(_P), C.c_int32, C.POINTER(pplbm_lattice), C.POINTER(pplbm_eos_params),
                                   C.POINTER(pplbm_relax), C.c_double, C.POINTER(_P), C.POINTER(_P), C.POINTER(_P),
                                   _P, C.c_size_t, _P]),
    "pplbm_adjoint_segment": (C.c_int, [_P, _P, C.c_int64, _P, _P, _P, _P, _P, C.c_size_t]),
    "pplbm_batch_run_host": (C.c_int, [_P, C.POINTER(C.c_void_p), C.c_int64, C.POINTER(C.c_void_p)]),
    "pplbm_batch_last_error": (C.c_char_p, [_P]),
    "pplbm_batch_destroy": (None, [_P]),
    "pplbm_adjoint_workspace_bytes": (C.c_size_t, [C.POINTER(pplbm_lattice)]),
    "pplbm_adjoint_step": (C.c_int, [_P, _P, _P, _P, _P, _P, C.c_size_t]),
    "pplbm_forward_checkpointed": (C.c_int, [_P, C.c_int64, C.c_int64, _P]),
    "pplbm_backward_checkpointed": (C.c_int, [_P, C.c_int64, C.c_int64, _P, _P, _P, _P, _P, _P, C.c_size_t]),
    "pplbm_adjoint_initial_density": (C.c_int, [_P, _P, _P]),
    "pplbm_eos_grad_constants": (C.c_int, [C.POINTER(pplbm_eos_derived), _D]),
    "pplbm_eos_constant_sensitivity": (C.c_int, [C.POINTER(pplbm_eos_params), C.c_double, C.POINTER(pplbm_relax),
                                                 C.c_int32, C.c_double, _D]),
    "pplbm_fd_workspace_bytes": (C.c_size_t, [C.POINTER(pplbm_lattice)]),
    "pplbm_fd_create": (C.c_int, [C.POINTER(_P), C.POINTER(pplbm_lattice), C.POINTER(pplbm_eos_params), C.c_double,
                                  C.c_double, C.c_double, C.c_double, _P, C.c_size_t, _P]),
    "pplbm_fd_set_state": (C.c_int, [_P, _P, _P, _P]),
    "pplbm_fd_get_state": (C.c_int, [_P, _P, _P, _P]),
    "pplbm_fd_step": (C.c_int, [_P, C.c_int64, C.c_double]),
    "pplbm_fd_sync": (C.c_int, [_P]),
    "pplbm_fd_destroy": (None, [_P]),
    "pplbm_last_error": (C.c_char_p, [_P]),
    "pplbm_status_string": (C.c_char_p, [C.c_int]),
    "pplbm_destroy": (None, [_P]),
}

_lib = None


def declared_symbols():
    """Names of the functions include/pplbm.h declares (parsed from the header)."""
    import re
    hdr = open(os.path.join(os.path.dirname(HERE), "include", "pplbm.h")).read()
    return sorted(set(re.findall(r"\b(pplbm_[a-z_0-9]+)\s*\(", hdr)))


def lib():
    """The loaded library (built in-tree by paper_2107_06355_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_2107_06355_gb300.build` "
                              "(the CUDA library is required; there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class PPLBMError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        s = lib().pplbm_status_string(status).decode()
        super().__init__(f"pplbm status {status} ({s}){': ' + msg if msg else ''}")


def check(status, ctx=None, batch=None):
    if status != PPLBM_OK:
        if batch:
            msg = lib().pplbm_batch_last_error(batch).decode()
        else:
            msg = lib().pplbm_last_error(ctx).decode() if ctx else ""
        raise PPLBMError(status, msg)
