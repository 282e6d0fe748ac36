"""CPU tests of the C-ABI library: it loads, exports every symbol include/pplbm.h
declares, and its host-only entry points (EOS set-up, workspace sizing, argument
checks) agree with the oracle. No CUDA call is made here."""
import ctypes as C
import subprocess

import pytest

from oracle import eos as E

P = pytest.importorskip("paper_2107_06355_gb300")
from paper_2107_06355_gb300 import _lib as L  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    from paper_2107_06355_gb300 import build
    build.build()
    return L.lib()


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    declared = L.declared_symbols()
    assert len(declared) >= 16
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    for s in declared:
        assert hasattr(lib, s)


CASES = [(E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834), (E.MODE_SMOOTH, 0.5, 0.363, 2.0, 0.775),
         (E.MODE_SMOOTH, 0.35, 0.363, 2.0, 0.775), (E.MODE_SMOOTH, 0.8, 0.5, 0.5, 0.342),
         (E.MODE_SMOOTH, 0.95, 0.363, 2.0, 0.775), (E.MODE_CS, 0.6, 0.387, 0.387, 0.0),
         (E.MODE_CS, 0.5, 0.363, 0.363, 0.0), (E.MODE_CS, 0.8, 0.5, 0.5, 0.0),
         # instance 61 of the 64-lattice sweep: p_max close to p_sat, the ellipse radicand near 0
         (E.MODE_SMOOTH, 0.35 + 0.6 * 61 / 63, 0.363, 2.0, 0.775)]


def test_peng_and_modified_smooth_setup_match_oracle(lib):
    for mode, Tr, al, av, alpha, rt in [(E.MODE_PENG, 0.6, 0.387, 0.387, 0.0, 0.45),
                                        (E.MODE_PENG, 0.5, 0.363, 0.363, 0.0, 0.44),
                                        (E.MODE_PENG, 0.7, 0.5, 0.5, 0.0, 0.122),
                                        (E.MODE_SMOOTH_MOD, 0.6, 0.387, 2.0, 0.446, 0.0)]:
        d = P.eos_setup(P.EOSParams(mode, Tr, al, av, alpha if alpha > 0 else 0.5, r_theta=rt))
        o = E.make_eos(mode, Tr, al, av, alpha, r_theta=rt)
        if mode == E.MODE_PENG:
            assert d["rho_m"] == pytest.approx(o.rho_m, rel=1e-11)
            assert d["theta"] == pytest.approx(o.theta, rel=1e-11)
        else:
            for k in ("p_max", "a1sq", "b1", "p_min", "a3sq", "b3"):
                assert d[k] == pytest.approx(getattr(o, k), rel=1e-11), k
        assert d["eps"] == 0.0
        assert d["psi_l"] == pytest.approx(float(o.psi(o.rho_l)), rel=1e-12)


@pytest.mark.parametrize("case", CASES, ids=lambda c: "m%d_Tr%.2f_al%.3f_av%.3f_al%.3f" % c)
def test_eos_setup_matches_oracle(lib, case):
    mode, Tr, al, av, alpha = case
    d = P.eos_setup(P.EOSParams(mode, Tr, al, av, alpha if alpha > 0 else 0.5))
    o = E.make_eos(mode, Tr, al, av, alpha)
    o.solve_eps()
    keys = ["Tc_l", "Tc_v", "T_l", "T_v", "rho_v", "rho_l", "p_sat", "p_sat_cs", "rho_max", "rho_min", "p_min_cs"]
    if mode == E.MODE_SMOOTH:
        keys += ["p_max", "p_min", "dP", "dpdrho_v", "dpdrho_l", "a1sq", "b1", "a3sq", "b3"]
    for k in keys:
        want = getattr(o, k)
        assert d[k] == pytest.approx(want, rel=2e-12, abs=1e-300), k
    # the oracle's Simpson estimate of eps carries ~1e-11 rounding (large cancelling terms)
    assert d["eps"] == pytest.approx(o.eps, rel=5e-11)
    assert d["psi_l"] == pytest.approx(float(o.psi(o.rho_l)), rel=1e-12)
    assert d["psi_v"] == pytest.approx(float(o.psi(o.rho_v)), rel=1e-12)


def test_eos_setup_rejects_bad_arguments(lib):
    out = L.pplbm_eos_derived()
    for p, G in [(L.pplbm_eos_params(1, 0, 1.2, 0.5, 0.5, 4, 1, 0.3), -1.0),   # Tr >= 1
                 (L.pplbm_eos_params(1, 0, 0.6, 0.5, 0.5, 4, 1, 0.3), 1.0),    # G > 0
                 (L.pplbm_eos_params(7, 0, 0.6, 0.5, 0.5, 4, 1, 0.3), -1.0),   # mode
                 (L.pplbm_eos_params(1, 0, 0.6, -0.5, 0.5, 4, 1, 0.3), -1.0)]:  # a < 0
        assert lib.pplbm_eos_setup(C.byref(p), G, C.byref(out)) == L.PPLBM_ERR_ARG
    assert lib.pplbm_eos_setup(None, -1.0, C.byref(out)) == L.PPLBM_ERR_ARG


def test_eos_setup_reports_unshapeable_loop(lib):
    # alpha so large that the liquid-side ellipse has no real a_3 (Sec. III.D condition)
    out = L.pplbm_eos_derived()
    p = L.pplbm_eos_params(1, 0, 0.6, 0.387, 2.0, 4, 1, 40.0)
    assert lib.pplbm_eos_setup(C.byref(p), -1.0, C.byref(out)) == L.PPLBM_ERR_EOS_SETUP


def test_workspace_bytes_and_lattice_validation(lib):
    relax = P.Relax().c()
    two = P.Relax(kind=L.RELAX_TWO_PHASE, tau_l=0.6, visc_ratio=2.0).c()
    full = P.Relax(tau_e=0.8).c()
    lat = L.pplbm_lattice(256, 4, L.BC_PERIODIC, 0)
    n = 256 * 4
    assert lib.pplbm_workspace_bytes(C.byref(lat), C.byref(relax)) == 8 * n * (20 + 3)
    assert lib.pplbm_workspace_bytes(C.byref(lat), C.byref(two)) == 8 * n * (20 + 5)
    assert lib.pplbm_workspace_bytes(C.byref(lat), C.byref(full)) == 8 * n * (20 + 9)
    for bad in [L.pplbm_lattice(0, 4, L.BC_PERIODIC, 0), L.pplbm_lattice(4, 0, L.BC_PERIODIC, 0),
                L.pplbm_lattice(4, 4, L.BC_PERIODIC_Y, 0),                       # x not periodic
                L.pplbm_lattice(4, 4, L.BC_PERIODIC_X | L.BC_WALL_BOTTOM, 0),    # one wall only
                L.pplbm_lattice(4, 4, L.BC_PERIODIC | L.BC_WALL_TOP, 0),         # periodic and wall
                L.pplbm_lattice(20000, 20000, L.BC_PERIODIC, 0),                 # 9 n >= 2^31
                L.pplbm_lattice(4, 4, L.BC_PERIODIC, 1)]:                        # reserved
        assert lib.pplbm_workspace_bytes(C.byref(bad), C.byref(relax)) == 0
    bad_tau = P.Relax(tau_nu=0.5).c()
    assert lib.pplbm_workspace_bytes(C.byref(lat), C.byref(bad_tau)) == 0


def test_create_rejects_without_touching_the_gpu(lib):
    ctx = C.c_void_p()
    lat = L.pplbm_lattice(8, 8, L.BC_PERIODIC, 0)
    eos = P.EOSParams().c()
    relax = P.Relax().c()
    # workspace too small, or NULL: rejected before any CUDA call
    assert lib.pplbm_create(C.byref(ctx), C.byref(lat), C.byref(eos), C.byref(relax), -1.0,
                            C.c_void_p(16), 8, None) == L.PPLBM_ERR_ARG
    assert lib.pplbm_create(C.byref(ctx), C.byref(lat), C.byref(eos), C.byref(relax), -1.0,
                            None, 1 << 20, None) == L.PPLBM_ERR_ARG
    assert ctx.value is None
    assert lib.pplbm_status_string(L.PPLBM_ERR_DIVERGED) == b"simulation diverged"


def test_one_call_setups_reject_missing_fields_without_touching_the_gpu(lib):
    lat = L.pplbm_lattice(8, 8, L.BC_PERIODIC, 0)
    eos = P.EOSParams().c()
    relax = P.Relax().c()
    ctx = C.c_void_p(1)
    assert lib.pplbm_init(C.byref(ctx), C.byref(lat), C.byref(eos), C.byref(relax), -1.0, None, None, None,
                          C.c_void_p(256), 1 << 20, None) == L.PPLBM_ERR_ARG
    assert ctx.value is None
    b = C.c_void_p(1)
    lats = (L.pplbm_lattice * 1)(lat)
    eoss = (L.pplbm_eos_params * 1)(eos)
    rels = (L.pplbm_relax * 1)(relax)
    rho = (C.c_void_p * 1)(None)
    assert lib.pplbm_batch_init(C.byref(b), 1, lats, eoss, rels, -1.0, rho, None, None, C.c_void_p(256), 1 << 20,
                                None) == L.PPLBM_ERR_ARG
    assert b.value is None
    assert lib.pplbm_adjoint_segment(None, None, 0, None, None, None, None, None, 0) == L.PPLBM_ERR_ARG


def test_constant_sensitivity_of_the_bulk_branches_has_closed_forms(lib):
    """k2 = -(2/G) a and k1 = (2/G) R T with T = T_r T_c(a), T_c proportional to a
    (Eq. CS, Sec. III.D): dk2/da = -2/G, dk1/da = k1/a on the branch the parameter
    owns and 0 on the other; alpha moves no bulk constant; kappa only its own slot."""
    G = -1.0
    eos = P.EOSParams(P.EOS_SMOOTH, 0.5, 0.363, 2.0, 0.775)
    relax = P.Relax().c()
    p = eos.c()
    d = L.pplbm_eos_derived()
    assert lib.pplbm_eos_setup(C.byref(p), G, C.byref(d)) == L.PPLBM_OK
    c = (C.c_double * L.NGRAD)()
    assert lib.pplbm_eos_grad_constants(C.byref(d), c) == L.PPLBM_OK
    idx = {n: k for k, n in enumerate(L.GRAD_NAMES)}
    sens = {}
    for name, which in L.SENS_PARAMS.items():
        dc = (C.c_double * L.NGRAD)()
        assert lib.pplbm_eos_constant_sensitivity(C.byref(p), G, C.byref(relax), which, 1e-4, dc) == L.PPLBM_OK
        sens[name] = list(dc)
    assert sens["a_vap"][idx["k2_v"]] == pytest.approx(-2.0 / G, rel=1e-9)
    assert sens["a_vap"][idx["k1_v"]] == pytest.approx(c[idx["k1_v"]] / eos.a_vap, rel=1e-9)
    assert sens["a_liq"][idx["k2_l"]] == pytest.approx(-2.0 / G, rel=1e-9)
    assert sens["a_liq"][idx["k1_l"]] == pytest.approx(c[idx["k1_l"]] / eos.a_liq, rel=1e-9)
    for k in ("k1_l", "k2_l"):
        assert abs(sens["a_vap"][idx[k]]) < 1e-9
    for k in ("k1_v", "k2_v"):
        assert abs(sens["a_liq"][idx[k]]) < 1e-9
    for k in ("k1_v", "k2_v", "k1_l", "k2_l", "k4_l"):
        assert abs(sens["alpha"][idx[k]]) < 1e-9
    # Delta P = p_sat(a_v) - p_sat(a_l): both parameters move the liquid shift
    assert abs(sens["a_vap"][idx["k4_l"]]) > 0 and abs(sens["a_liq"][idx["k4_l"]]) > 0
    # kappa (the surface-tension control) is its own slot: the unit vector, and no EOS constant moves
    assert sens["kappa"] == [1.0 if k == idx["kappa"] else 0.0 for k in range(L.NGRAD)]
    for name in ("alpha", "a_vap", "a_liq"):
        assert sens[name][idx["kappa"]] == 0.0
    dc = (C.c_double * L.NGRAD)()
    assert lib.pplbm_eos_constant_sensitivity(C.byref(p), G, C.byref(relax), 4, 1e-4, dc) == L.PPLBM_ERR_ARG


def _declarations():
    """{name: parameter count} of every function include/pplbm.h declares."""
    import os
    import re

    hdr = open(os.path.join(os.path.dirname(L.HERE), "include", "pplbm.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(pplbm_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", hdr):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_bindings_match_the_header_parameter_counts(lib):
    """Every declared entry point has a ctypes signature with the header's number
    of parameters, so no call passes its arguments shifted."""
    decl = _declarations()
    assert len(decl) >= 60
    missing = sorted(set(decl) - set(L._SIGS))
    assert not missing, missing
    wrong = {n: (k, len(L._SIGS[n][1])) for n, k in decl.items() if len(L._SIGS[n][1]) != k}
    assert not wrong, wrong


def test_tall_lattices_are_rejected_where_the_grids_are_two_dimensional(lib):
    """A single lattice and the FD solver launch 2-D grids with 8-row tiles on the y
    axis (at most 65,535): ny <= 524,280 there; the batch's 1-D grids take any ny."""
    relax = P.Relax().c()
    ok = L.pplbm_lattice(4, 524280, L.BC_PERIODIC, 0)
    tall = L.pplbm_lattice(4, 524288, L.BC_PERIODIC, 0)
    assert lib.pplbm_workspace_bytes(C.byref(ok), C.byref(relax)) > 0
    assert lib.pplbm_workspace_bytes(C.byref(tall), C.byref(relax)) == 0
    assert lib.pplbm_fd_workspace_bytes(C.byref(ok)) > 0
    assert lib.pplbm_fd_workspace_bytes(C.byref(tall)) == 0
    rel = (L.pplbm_relax * 1)(relax)
    assert lib.pplbm_batch_workspace_bytes(1, (L.pplbm_lattice * 1)(tall), rel) > 0


def test_surface_tension_kappa_is_validated_at_set_up(lib):
    """kappa (the surface-tension control) must be finite and below 1, where the
    surface tension (1 - kappa) gamma would vanish or change sign; the check runs in
    the single-lattice and batched set-ups before any CUDA call. The relax struct's
    layout in the binding matches the header (kappa after the reserved word)."""
    lat = L.pplbm_lattice(16, 16, L.BC_PERIODIC, 0)
    for kind in ({}, {"kind": L.RELAX_TWO_PHASE, "tau_l": 0.7, "visc_ratio": 5.0}, {"tau_e": 0.8}):
        for kappa, ok in ((0.0, True), (0.5, True), (-2.0, True), (0.999, True), (1.0, False), (3.0, False),
                          (float("nan"), False), (float("inf"), False)):
            r = P.Relax(kappa=kappa, **kind).c()
            assert (lib.pplbm_workspace_bytes(C.byref(lat), C.byref(r)) > 0) == ok, (kind, kappa)
            arr = (L.pplbm_relax * 1)(r)
            assert (lib.pplbm_batch_workspace_bytes(1, (L.pplbm_lattice * 1)(lat), arr) > 0) == ok, (kind, kappa)
    # two-phase relaxation needs finite tau_l > 1/2 and visc_ratio > 0
    for tau_l, vr, ok in ((0.7, 5.0, True), (0.5, 5.0, False), (float("inf"), 5.0, False), (0.7, 0.0, False),
                          (0.7, float("inf"), False)):
        r = P.Relax(kind=L.RELAX_TWO_PHASE, tau_l=tau_l, visc_ratio=vr).c()
        assert (lib.pplbm_workspace_bytes(C.byref(lat), C.byref(r)) > 0) == ok, (tau_l, vr)
    assert C.sizeof(L.pplbm_relax) == 8 + 8 * 9 + 8 + 8
    assert L.pplbm_relax.kappa.offset == C.sizeof(L.pplbm_relax) - 8


def test_noalloc_step_rejects_overlapping_buffers_before_any_cuda_call(lib):
    """pplbm_step_noalloc checks its arguments on the host first: overlapping f_in /
    f_out ranges (an offset view into one buffer) are refused with their own message,
    before the device is touched (no GPU here; the pointers are never dereferenced)."""
    eos = L.pplbm_eos_derived()
    p = P.EOSParams().c()
    assert lib.pplbm_eos_setup(C.byref(p), -1.0, C.byref(eos)) == L.PPLBM_OK
    lat = L.pplbm_lattice(16, 8, L.BC_PERIODIC, 0)
    relax = P.Relax().c()
    n = 16 * 8
    base = 1 << 40
    msg = C.c_char_p()
    for off in (8, 8 * n, 8 * (9 * n - 1)):   # partial overlaps, in bytes
        st = lib.pplbm_step_noalloc(C.byref(lat), C.byref(eos), C.byref(relax), C.c_void_p(base),
                                    C.c_void_p(base + off), None, C.byref(msg))
        assert st == L.PPLBM_ERR_ARG
        assert b"overlap" in msg.value
        st = lib.pplbm_step_noalloc(C.byref(lat), C.byref(eos), C.byref(relax), C.c_void_p(base + off),
                                    C.c_void_p(base), None, C.byref(msg))
        assert st == L.PPLBM_ERR_ARG and b"overlap" in msg.value
    st = lib.pplbm_step_noalloc(C.byref(lat), C.byref(eos), C.byref(relax), C.c_void_p(base), C.c_void_p(base),
                                None, C.byref(msg))
    assert st == L.PPLBM_ERR_ARG and b"overlap" in msg.value
    # too large a lattice is refused by its own message, also before any CUDA call
    big = L.pplbm_lattice(257, 256, L.BC_PERIODIC, 0)
    st = lib.pplbm_step_noalloc(C.byref(big), C.byref(eos), C.byref(relax), C.c_void_p(base),
                                C.c_void_p(base + 8 * 9 * 257 * 256), None, C.byref(msg))
    assert st == L.PPLBM_ERR_ARG and b"65536" in msg.value


def _oracle_dc_in_library_slots(d, wrt, h, G=-1.0):
    """The oracle's d(constants)/d(theta) (oracle.adjoint.constants_derivative, central
    differences with Richardson extrapolation of its own set-up) mapped onto the
    library's slots: 1/a^2 of the ellipses, the cubic's a2 = 2 (p_max - p_min) and
    b2 = 3 (p_min - p_max), z = sigma G^2/432, k1 = (2/G) R T, k2 = -(2/G) a,
    k4 = (2/G) Delta P (Sec. III.D, Eqs. CS, InteractionPotential, LiFS)."""
    from oracle import adjoint as A

    o = A.constants_derivative(E.MODE_SMOOTH, 0.5, 0.363, 2.0, 0.775, h=h, wrt=wrt)
    s = 2.0 / G
    R = 1.0
    return {"p_max": o["p_max"], "b1": o["b1"], "inv_a1sq": -o["a1sq"] / d["a1sq"] ** 2,
            "a2": 2.0 * (o["p_max"] - o["p_min"]), "b2": 3.0 * (o["p_min"] - o["p_max"]), "p_min": o["p_min"],
            "b3": o["b3"], "inv_a3sq": -o["a3sq"] / d["a3sq"] ** 2, "zz_scale": o["sigma"] * G * G / 432.0,
            "k1_v": s * R * o["T_v"], "k2_v": -s * o["a_v"], "k1_l": s * R * o["T_l"], "k2_l": -s * o["a_l"],
            "k4_l": s * o["dP"], "kappa": 0.0}


@pytest.mark.parametrize("which,wrt", [(0, "alpha"), (1, "a_v"), (2, "a_l")])
def test_constant_sensitivity_matches_the_oracle_and_its_error_bound(lib, which, wrt):
    """pplbm_eos_constant_sensitivity (the product's set-up: Maxwell by the chemical
    potential, Gauss-Legendre, Ridders) against the oracle's derivative of its own
    set-up (brentq, adaptive quadrature, Simpson for eps) on the adjoint configuration
    (T_r = 0.5, a_l = 0.363, a_v = 2, alpha = 0.775).

    The header's bound for the library: O(h^4) + 3 delta/h, delta the set-up's error
    in a constant c (~1e-15 |c|). Its estimates at h = 1e-4 and h/2 (bound 6 delta/h)
    therefore differ by at most ~1e-10 |c|; the test allows 1e-9 |c| (+ 1e-8 of the
    derivative for the O(h^4) term). The oracle's (h = 1e-3, its quadratures good to
    ~1e-14 |c|, its eps to ~1e-11) may be off by 3e-11 |c|, 3e-8 for sigma: the test
    allows 1e-7 |c| + 1e-6 of the derivative."""
    G = -1.0
    p = P.EOSParams(P.EOS_SMOOTH, 0.5, 0.363, 2.0, 0.775).c()
    relax = P.Relax().c()
    d = P.eos_setup(P.EOSParams(P.EOS_SMOOTH, 0.5, 0.363, 2.0, 0.775))
    dd = L.pplbm_eos_derived()
    assert lib.pplbm_eos_setup(C.byref(p), G, C.byref(dd)) == L.PPLBM_OK
    cv = (C.c_double * L.NGRAD)()
    assert lib.pplbm_eos_grad_constants(C.byref(dd), cv) == L.PPLBM_OK
    cval = dict(zip(L.GRAD_NAMES, list(cv)))
    cval["zz_scale"] = (-d["eps"] / (16.0 * G)) * G * G / 432.0   # sigma = -eps/(16 G), Sec. III.A
    dc = {}
    for h in (1e-4, 5e-5):
        out = (C.c_double * L.NGRAD)()
        assert lib.pplbm_eos_constant_sensitivity(C.byref(p), G, C.byref(relax), which, h, out) == L.PPLBM_OK
        dc[h] = dict(zip(L.GRAD_NAMES, list(out)))
    want = _oracle_dc_in_library_slots(d, wrt, 1e-3, G)
    for k in L.GRAD_NAMES:
        a, b = dc[1e-4][k], dc[5e-5][k]
        assert abs(a - b) <= 1e-9 * abs(cval[k]) + 1e-8 * abs(a), (k, a, b)
        assert abs(a - want[k]) <= 1e-7 * abs(cval[k]) + 1e-6 * abs(want[k]), (k, a, want[k])
    # the slots each parameter moves are not all zero
    assert sum(abs(v) for v in dc[1e-4].values()) > 0
