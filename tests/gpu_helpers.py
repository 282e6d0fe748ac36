"""Shared set-up for the GPU parity tests: one configuration is built twice, once
as an oracle lattice and once as a CUDA simulation, from the same seeded inputs."""
from __future__ import annotations

import numpy as np

from oracle import eos as E
from oracle import lbm as L

BC_PER = L.BC_PERIODIC_X | L.BC_PERIODIC_Y
BC_WALLS = L.BC_PERIODIC_X | L.BC_WALL_BOTTOM | L.BC_WALL_TOP

_EOS_CACHE = {}


SMOOTH_MODES = (E.MODE_SMOOTH, E.MODE_SMOOTH_MOD)


def oracle_eos(mode, Tr, a_l, a_v, alpha, r_theta=0.0):
    key = (mode, Tr, a_l, a_v, alpha, r_theta)
    if key not in _EOS_CACHE:
        e = E.make_eos(mode, Tr, a_l, a_v if mode in SMOOTH_MODES else a_l, alpha, r_theta=r_theta)
        if mode in (E.MODE_CS, E.MODE_SMOOTH):
            e.solve_eps()
        _EOS_CACHE[key] = e
    return _EOS_CACHE[key]


def make_pair(nx, ny, bc, eos_case, relax_kw, forcing_li=True):
    """(oracle Lattice, gpu Simulation) for the same parameters.

    eos_case = (mode, Tr, a_l, a_v, alpha); relax_kw: keyword arguments of the
    library's Relax (kind, tau_*, tau_l, visc_ratio, kappa)."""
    import paper_2107_06355_gb300 as P

    mode, Tr, a_l, a_v, alpha = eos_case[:5]
    r_theta = eos_case[5] if len(eos_case) > 5 else 0.0
    oe = oracle_eos(*eos_case)
    sigma = oe.sigma() if forcing_li else 0.0
    kind = relax_kw.get("kind", P.RELAX_MRT)
    orelax = L.Relax(kind=kind, tau_rho=relax_kw.get("tau_rho", 1.0), tau_e=relax_kw.get("tau_e", 1.0),
                     tau_zeta=relax_kw.get("tau_zeta", 1.0), tau_j=relax_kw.get("tau_j", 1.0),
                     tau_q=relax_kw.get("tau_q", 1.0), tau_nu=relax_kw.get("tau_nu", 1.0),
                     tau_l=relax_kw.get("tau_l", 1.0), visc_ratio=relax_kw.get("visc_ratio", 1.0), sigma=sigma,
                     kappa=relax_kw.get("kappa", 0.0))
    olat = L.Lattice(nx, ny, bc, oe, orelax)
    gp = P.EOSParams(mode=mode, Tr=Tr, a_liq=a_l, a_vap=a_v if mode in SMOOTH_MODES else a_l,
                     alpha=alpha if alpha > 0 else 0.5, r_theta=r_theta)
    grelax = P.Relax(forcing=P.FORCING_LI if forcing_li else P.FORCING_GUO, sigma_auto=True, **relax_kw)
    sim = P.Simulation(nx, ny, bc, gp, grelax)
    return olat, sim


def normwise(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
