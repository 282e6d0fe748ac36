"""Paper-level pins for the oracle (CPU only).

Reproduces Table DropImpactParameters (Sec. IV): planar interface on a
(Nx, Ny) = (2, 200) periodic lattice, initial tanh profile of width W = 10
between the Maxwell densities (Eq. PlanarIntDensity), all relaxation times 1,
Li forcing with sigma from Eq. VaporLiqEq, run until the convergence criterion
of Sec. III.A drops below 1e-6. Checks the vapour-density error
(Eq. DensityError), the interface width and the surface tension
(Eq. SurfaceTension) against the printed values. The seven planar runs are
independent and run once, side by side in spawned processes; each test checks
its own run.
"""
import json
import multiprocessing
import os
from concurrent.futures import ProcessPoolExecutor

import pytest

import lbm_inputs as I
from oracle import eos as E
from oracle import lbm as L

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
CASES = GOLD["table_drop_impact_parameters"]["cases"]
PM = GOLD["peng_and_modified_smooth"]["cases"]
TPP = GOLD["peng_table_param_peng"]


def _eos(case):
    """The oracle EOS of a golden case (Table DropImpactParameters, the Peng and
    Modified Smooth cases, or Table ParamPeng's row)."""
    if case["mode"] == "TPP":
        return E.make_eos(E.MODE_PENG, TPP["Tr"], TPP["a"], TPP["a"], 0.0, r_theta=case["r_theta"])
    mode = {"SMOOTH": E.MODE_SMOOTH, "CS": E.MODE_CS, "PENG": E.MODE_PENG, "SMOOTH_MOD": E.MODE_SMOOTH_MOD}
    return E.make_eos(mode[case["mode"]], case["Tr"], case["a_l"], case["a_v"], case["alpha"],
                      r_theta=case.get("r_theta", 0.0))


def _planar_run(case):
    """Converged density profile of the (2, 200) planar interface (Sec. III.A), or
    None without convergence; Table ParamPeng's row runs a fixed 40,000 steps from
    its wider start."""
    eos = _eos(case)
    li = case["mode"] in ("SMOOTH", "CS")
    lat = L.Lattice(2, 200, L.BC_PERIODIC_X | L.BC_PERIODIC_Y, eos, L.Relax(sigma=eos.sigma() if li else 0.0))
    if case["mode"] == "TPP":
        f = lat.init_equilibrium(I.planar(2, 200, eos.rho_v, eos.rho_l, W=case["W_start"]))
        return lat.step(f, 40000).sum(axis=0)
    f = lat.init_equilibrium(I.planar(2, 200, eos.rho_v, eos.rho_l, W=10.0))
    prev = f.sum(axis=0)
    for _ in range(2000):
        f = lat.step(f, 100)
        rho = f.sum(axis=0)
        r = L.convergence_residual(rho, prev)
        prev = rho
        if r < 1e-6:
            return rho
    return None


@pytest.fixture(scope="module")
def runs():
    cases = {c["name"]: c for c in CASES + PM}
    cases["TPP_w7"] = dict(TPP["cases"][0], mode="TPP")
    ctx = multiprocessing.get_context("spawn")
    with ProcessPoolExecutor(max_workers=min(len(cases), os.cpu_count() or 1), mp_context=ctx) as ex:
        futures = {name: ex.submit(_planar_run, c) for name, c in cases.items()}
        return {name: fu.result() for name, fu in futures.items()}


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_planar_interface_reproduces_table(case, runs):
    eos = _eos(case)
    rho = runs[case["name"]]
    if rho is None:
        pytest.fail("no convergence")
    rho_v, rho_l = rho[0, 0], rho[100, 0]
    err = L.vapor_density_error(rho_v, eos.rho_v)
    assert err == pytest.approx(case["E_percent"], rel=0.01)
    assert L.interface_width(rho[:, 0], rho_v, rho_l) == case["w"]
    gamma = L.surface_tension_planar(eos.psi(rho[:, 0]), eos.G)
    assert gamma * 1e3 == pytest.approx(case["gamma_e3"], rel=0.06)
    ratio = GOLD["density_ratio_Tr05"].get(case["name"])
    if ratio is not None:   # Sec. IV.B's simulated density ratios at T_r = 0.5
        assert rho_l / rho_v == pytest.approx(ratio["ratio"], rel=ratio["rel"])


@pytest.mark.parametrize("case", PM, ids=[c["name"] for c in PM])
def test_planar_interface_peng_and_modified_smooth(case, runs):
    eos = _eos(case)
    assert eos.sigma() == 0.0   # both are used with the Guo scheme
    rho = runs[case["name"]]
    if rho is None:
        pytest.fail("no convergence")
    rho_v, rho_l = rho[0, 0], rho[100, 0]
    if case["E_percent"] is not None:
        # the paper's 0.0046 % is one part in 2e4 of rho_v: compare absolutely
        assert abs(L.vapor_density_error(rho_v, eos.rho_v) - case["E_percent"]) < 0.002
    assert L.interface_width(rho[:, 0], rho_v, rho_l) == case["w"]
    gamma = L.surface_tension_planar(eos.psi(rho[:, 0]), eos.G)
    assert gamma * 1e3 == pytest.approx(case["gamma_e3"], rel=0.03)


def test_peng_table_param_peng_w7_row(runs):
    """Table ParamPeng, r_theta = 0.290 at T_r = 0.5 (a = 0.5, Guo forcing): w = 7 and a
    vapour-density error close to 0.12 %. Started from a tanh of width 18 (from
    W = 10 this loop diverges in the start-up transient); 40,000 steps, after which
    the residual of Sec. III.A is about 2e-5 and w, E are settled to the digits
    checked."""
    case = dict(TPP["cases"][0], mode="TPP")
    eos = _eos(case)
    rho = runs["TPP_w7"]
    rho_v, rho_l = rho[0, 0], rho[100, 0]
    assert L.interface_width(rho[:, 0], rho_v, rho_l) == case["w"]
    assert abs(L.vapor_density_error(rho_v, eos.rho_v) - case["E_percent_about"]) < case["E_tol"]
