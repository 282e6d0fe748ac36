"""Paper-level pins for the oracle (CPU only, ~90 s).

Reproduces Table DropImpactParameters (Sec. IV): planar interface on a
(Nx, Ny) = (2, 200) periodic lattice, initial tanh profile of width W = 10
between the Maxwell densities (Eq. PlanarIntDensity), all relaxation times 1,
Li forcing with sigma from Eq. VaporLiqEq, run until the convergence criterion
of Sec. III.A drops below 1e-6. Checks the vapour-density error
(Eq. DensityError), the interface width and the surface tension
(Eq. SurfaceTension) against the printed values.
"""
import json
import os

import pytest

import lbm_inputs as I
from oracle import eos as E
from oracle import lbm as L

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
CASES = GOLD["table_drop_impact_parameters"]["cases"]


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_planar_interface_reproduces_table(case):
    mode = E.MODE_SMOOTH if case["mode"] == "SMOOTH" else E.MODE_CS
    eos = E.make_eos(mode, case["Tr"], case["a_l"], case["a_v"], case["alpha"])
    lat = L.Lattice(2, 200, L.BC_PERIODIC_X | L.BC_PERIODIC_Y, eos, L.Relax(sigma=eos.sigma()))
    f = lat.init_equilibrium(I.planar(2, 200, eos.rho_v, eos.rho_l, W=10.0))
    prev = f.sum(axis=0)
    for _ in range(2000):
        f = lat.step(f, 100)
        rho = f.sum(axis=0)
        r = L.convergence_residual(rho, prev)
        prev = rho
        if r < 1e-6:
            break
    else:
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


PM = GOLD["peng_and_modified_smooth"]["cases"]


@pytest.mark.parametrize("case", PM, ids=[c["name"] for c in PM])
def test_planar_interface_peng_and_modified_smooth(case):
    mode = E.MODE_PENG if case["mode"] == "PENG" else E.MODE_SMOOTH_MOD
    eos = E.make_eos(mode, case["Tr"], case["a_l"], case["a_v"], case["alpha"], r_theta=case["r_theta"])
    assert eos.sigma() == 0.0   # both are used with the Guo scheme
    lat = L.Lattice(2, 200, L.BC_PERIODIC_X | L.BC_PERIODIC_Y, eos, L.Relax(sigma=0.0))
    f = lat.init_equilibrium(I.planar(2, 200, eos.rho_v, eos.rho_l, W=10.0))
    prev = f.sum(axis=0)
    for _ in range(2000):
        f = lat.step(f, 100)
        rho = f.sum(axis=0)
        r = L.convergence_residual(rho, prev)
        prev = rho
        if r < 1e-6:
            break
    else:
        pytest.fail("no convergence")
    rho_v, rho_l = rho[0, 0], rho[100, 0]
    if case["E_percent"] is not None:
        # the paper's 0.0046 % is one part in 2e4 of rho_v: compare absolutely
        assert abs(L.vapor_density_error(rho_v, eos.rho_v) - case["E_percent"]) < 0.002
    assert L.interface_width(rho[:, 0], rho_v, rho_l) == case["w"]
    gamma = L.surface_tension_planar(eos.psi(rho[:, 0]), eos.G)
    assert gamma * 1e3 == pytest.approx(case["gamma_e3"], rel=0.03)


TPP = GOLD["peng_table_param_peng"]


def test_peng_table_param_peng_w7_row():
    """Table ParamPeng, r_theta = 0.290 at T_r = 0.5 (a = 0.5, Guo forcing): w = 7 and a
    vapour-density error close to 0.12 %. Started from a tanh of width 18 (from
    W = 10 this loop diverges in the start-up transient); 40,000 steps, after which
    the residual of Sec. III.A is about 2e-5 and w, E are settled to the digits
    checked."""
    case = TPP["cases"][0]
    eos = E.make_eos(E.MODE_PENG, TPP["Tr"], TPP["a"], TPP["a"], 0.0, r_theta=case["r_theta"])
    lat = L.Lattice(2, 200, L.BC_PERIODIC_X | L.BC_PERIODIC_Y, eos, L.Relax(sigma=0.0))
    f = lat.init_equilibrium(I.planar(2, 200, eos.rho_v, eos.rho_l, W=case["W_start"]))
    f = lat.step(f, 40000)
    rho = f.sum(axis=0)
    rho_v, rho_l = rho[0, 0], rho[100, 0]
    assert L.interface_width(rho[:, 0], rho_v, rho_l) == case["w"]
    assert abs(L.vapor_density_error(rho_v, eos.rho_v) - case["E_percent_about"]) < case["E_tol"]
