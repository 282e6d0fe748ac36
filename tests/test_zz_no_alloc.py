"""pplbm_step_noalloc: the step for callers that cannot allocate device memory
(a host framework owning all device memory, or a stream that must not be
synchronised by cudaMalloc/cudaFree). Its psi and moment planes live in a static
device array, so it must give the same distributions as the context-based step
(pplbm_create / pplbm_step), call after call, for every EOS and relaxation kind
(and the oracle's). This file is collected last so that
a run stopping at the first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

import lbm_inputs as I
from gpu_helpers import BC_WALLS, make_pair, normwise
from oracle import eos as E

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(L, sim, f_in, f_out):
    msg = C.c_char_p()
    eos = L.pplbm_eos_derived()
    L.check(L.lib().pplbm_get_derived(sim.ctx, C.byref(eos)))
    relax = sim._relax_c
    st = L.lib().pplbm_step_noalloc(C.byref(sim.lattice), C.byref(eos), C.byref(relax),
                                    C.c_void_p(f_in.data_ptr()), C.c_void_p(f_out.data_ptr()),
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(msg))
    return st, (msg.value or b"").decode()


CASES = {
    "unit": ((E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834), {}, True),
    "two_phase": ((E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834), {"kind": 1, "tau_l": 0.6, "visc_ratio": 3.0}, True),
    "full_mrt": ((E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834), {"tau_e": 0.8, "tau_zeta": 1.1, "tau_q": 1.2, "tau_nu": 0.7},
                 True),
    # the two EOS built for Guo forcing (Sec. IV.C, Eqs. PengEOS, PengTheta)
    "peng06": ((E.MODE_PENG, 0.6, 0.387, 0.387, 0.0, 0.45), {}, False),
    "modsmooth06": ((E.MODE_SMOOTH_MOD, 0.6, 0.387, 2.0, 0.446), {}, False),
}


@pytest.mark.parametrize("case", list(CASES), ids=list(CASES))
def test_noalloc_step_matches_context_step_twice(case):
    from paper_2107_06355_gb300 import _lib as L

    eos_case, relax, li = CASES[case]
    olat, sim = make_pair(70, 27, BC_WALLS, eos_case, relax, forcing_li=li)
    e = olat.eos
    rho, ux, uy = I.impact(70, 27, 5, 5, e.rho_v, e.rho_l, 0.01 if not li else 0.03, W=8.0 if not li else 5.0)
    sim.init_equilibrium(rho, ux, uy)
    f0 = sim.get_f()
    a = torch.empty_like(f0)
    b = torch.empty_like(f0)
    st, msg = _noalloc(L, sim, f0, a)          # first call
    assert st == 0, msg
    assert msg == ""
    st, msg = _noalloc(L, sim, a, b)           # second call, same static scratch
    assert st == 0, msg
    sim.step(2)
    ref = sim.get_f()
    torch.cuda.synchronize()
    assert normwise(b.cpu().numpy(), ref.cpu().numpy()) < 1e-12
    # and the oracle's two steps from the same state
    f_or = olat.step(olat.init_equilibrium(rho, ux, uy), 2)
    assert normwise(b.cpu().numpy(), f_or) < 3e-12
    # one step from f0 also matches
    sim.set_f(f0)
    sim.step(1)
    assert normwise(a.cpu().numpy(), sim.get_f().cpu().numpy()) < 1e-12
    sim.close()


def test_noalloc_rejects_lattices_beyond_the_static_limit():
    from paper_2107_06355_gb300 import _lib as L
    import paper_2107_06355_gb300 as P

    eos = L.pplbm_eos_derived()
    p = P.EOSParams().c()
    L.check(L.lib().pplbm_eos_setup(C.byref(p), -1.0, C.byref(eos)))
    lat = L.pplbm_lattice(257, 256, L.BC_PERIODIC, 0)   # 65,792 > 65,536 nodes
    relax = P.Relax().c()
    f = torch.zeros(9 * 257 * 256, dtype=torch.float64, device="cuda")
    g = torch.zeros_like(f)
    msg = C.c_char_p()
    st = L.lib().pplbm_step_noalloc(C.byref(lat), C.byref(eos), C.byref(relax), C.c_void_p(f.data_ptr()),
                                    C.c_void_p(g.data_ptr()), None, C.byref(msg))
    assert st == L.PPLBM_ERR_ARG
    assert b"65536" in msg.value
    # the largest accepted lattice works
    lat = L.pplbm_lattice(256, 256, L.BC_PERIODIC, 0)
    d = P.eos_setup(P.EOSParams())
    rho0 = I.droplet(256, 256, 48, d["rho_v"], d["rho_l"], W=8.0)
    sim = P.Simulation(256, 256, P.BC_PERIODIC, P.EOSParams(), P.Relax())
    sim.init_equilibrium(rho0)
    f0 = sim.get_f()
    out = torch.empty_like(f0)
    st = L.lib().pplbm_step_noalloc(C.byref(lat), C.byref(eos), C.byref(relax), C.c_void_p(f0.data_ptr()),
                                    C.c_void_p(out.data_ptr()), None, C.byref(msg))
    assert st == 0
    sim.step(1)
    assert normwise(out.cpu().numpy(), sim.get_f().cpu().numpy()) < 1e-12
    sim.close()
