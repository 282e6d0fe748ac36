"""Parameter sweeps of planar-interface equilibria on the batched engine (Sec. III).

`planar_coexistence` advances many (Nx, Ny) = (2, 200) periodic planar interfaces
(one per (EOS, relaxation) case) in one batch until the convergence criterion of
Sec. III.A holds for each, then reports the paper's observables: the vapour
density error of Eq. DensityError, the interface width (nodes with
0.01 < (rho - rho_v)/(rho_l - rho_v) < 0.99, with the simulated densities) and
the surface tension of Eq. SurfaceTension (fourth-order central differences,
Simpson's rule). Instances are isolated: one that diverges is reported as such
and the others continue. Stepping and the per-check guard (residual, bad nodes)
run in the library's kernels; the host evaluates the observables on the
returned fields at the end.

`laplace_law` fits the 2-D Laplace law on static droplets; with
`kappa_for_surface_tension` it sets the surface-tension control that the
paper's Sec. V proposes for keeping the Weber number when alpha changes.
"""
from __future__ import annotations

import numpy as np

from . import _lib as L
from .batch import Batch


def _inputs():
    """The seeded initial-field generators (module lbm_inputs beside this package),
    the one definition of the planar, droplet and impact profiles."""
    import importlib
    import os
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    return importlib.import_module("lbm_inputs")


def planar_profile(ny, rho_v, rho_l, W):
    """Eq. PlanarIntDensity along y: interfaces at 1/4 and 3/4 of the length."""
    return _inputs().planar(1, ny, rho_v, rho_l, W=W)[:, 0].copy()


def density_error(rho_v_sim, rho_v_maxwell):
    """Eq. DensityError, in percent."""
    return 100.0 * (rho_v_sim - rho_v_maxwell) / rho_v_maxwell


def interface_width(profile, rho_v, rho_l):
    """Nodes of the first interface with 0.01 < phi < 0.99 (Sec. III.B definition)."""
    phi = (np.asarray(profile) - rho_v) / (rho_l - rho_v)
    first = phi[: len(phi) // 2]
    return int(np.count_nonzero((first > 0.01) & (first < 0.99)))


def interface_width_interp(profile, rho_v, rho_l):
    """Continuous width of the first interface: the distance between the points where
    phi = (rho - rho_v)/(rho_l - rho_v) crosses 0.01 and 0.99, each located by linear
    interpolation between the neighbouring nodes. Used to tune a shaping parameter
    to a target width; the node count of `interface_width` is the paper's measure."""
    phi = (np.asarray(profile, dtype=np.float64) - rho_v) / (rho_l - rho_v)
    seg = phi[: len(phi) // 2 + 1]

    def crossing(level):
        k = int(np.argmax(seg >= level))
        if k == 0 or seg[k] < level:
            return float("nan")
        return k - 1 + (level - seg[k - 1]) / (seg[k] - seg[k - 1])

    return crossing(0.99) - crossing(0.01)


def surface_tension(psi_profile, G=-1.0):
    """Eq. SurfaceTension on a periodic profile with two interfaces (half the period integral)."""
    p = np.asarray(psi_profile, dtype=np.float64)
    n = len(p)
    d = (p[(np.arange(n) - 2) % n] - 8 * p[(np.arange(n) - 1) % n] + 8 * p[(np.arange(n) + 1) % n]
         - p[(np.arange(n) + 2) % n]) / 12.0
    g = np.append(d * d, d[0] * d[0])
    w = np.ones(n + 1)
    w[1:-1:2] = 4.0
    w[2:-1:2] = 2.0
    return -G / 6.0 * float(np.dot(w, g) / 3.0) / 2.0


def planar_coexistence(cases, nx=2, ny=200, W=10.0, tol=1e-6, check_every=100, max_steps=300000, G=-1.0):
    """cases: list of (EOSParams, Relax) or (EOSParams, Relax, W) (W: that case's
    initial width; otherwise `W`). Returns one dict per case with keys
    converged, diverged, steps and, unless the case diverged, rho_v, rho_l,
    E_percent, width, width_interp, gamma and the density profile along y.
    The Sec. III.A residual and the divergence test run in the library's guard.
    gamma is Eq. IntegralSurfaceTension of the case's pressure tensor: with the
    surface-tension control (Relax.kappa) the planar profile does not change and
    gamma is (1 - kappa) times Eq. SurfaceTension."""
    import torch

    n = len(cases)
    b = Batch([(nx, ny, L.BC_PERIODIC)] * n, [c[0] for c in cases], [c[1] for c in cases], G=G)
    b.set_isolation(True)
    maxwell = []
    for i in range(n):
        d = b.derived(i)
        maxwell.append((d["rho_v"], d["rho_l"]))
        prof = planar_profile(ny, d["rho_v"], d["rho_l"], cases[i][2] if len(cases[i]) > 2 else W)
        b.init_equilibrium(i, np.repeat(prof[:, None], nx, axis=1))
    b.set_plan(L.PLAN_GRAPH, 0)
    b.guard()   # first snapshot
    done = [False] * n
    out = [dict(converged=False, diverged=False, steps=0) for _ in range(n)]
    steps = 0
    while steps < max_steps and not all(done):
        b.step(check_every)
        steps += check_every
        g = b.guard()
        status = b.instance_status()
        for i in range(n):
            if done[i]:
                continue
            if status[i] != 0 or g[i, 2] > 0 or not np.isfinite(g[i, 3]):
                done[i] = True
                out[i].update(diverged=True, steps=steps)
            elif g[i, 3] < tol:
                done[i] = True
                out[i].update(converged=True, steps=steps)
    for i in range(n):
        if out[i]["diverged"]:
            continue
        if not done[i]:
            out[i]["steps"] = steps
        rho, _, _, psi = [t.cpu().numpy() for t in b.fields(i)]
        col_r, col_p = rho[:, 0], psi[:, 0]
        rv, rl = float(col_r[0]), float(col_r[ny // 2])
        out[i].update(rho_v=rv, rho_l=rl, E_percent=density_error(rv, maxwell[i][0]),
                      width=interface_width(col_r, rv, rl), width_interp=interface_width_interp(col_r, rv, rl),
                      gamma=(1.0 - cases[i][1].kappa) * surface_tension(col_p, G), profile=col_r.copy())
    b.close()
    torch.cuda.synchronize()
    return out


def planar_coexistence_started(cases, widths=(10.0, 18.0, 22.0, 25.0), **kw):
    """planar_coexistence, retrying every case that diverges from the next, wider
    initial profile in `widths`. From the W = 10 tanh between the Maxwell densities,
    the Peng loop at T_r <= 0.55 drives the vapour-side node negative within a few
    hundred steps although wider starts converge (Table ParamPeng's interfaces).
    Each result records the initial width W it converged from."""
    out = [None] * len(cases)
    todo = list(range(len(cases)))
    for W in widths:
        if not todo:
            break
        res = planar_coexistence([(cases[i][0], cases[i][1], W) for i in todo], **kw)
        left = []
        for i, r in zip(todo, res):
            r["W"] = W
            out[i] = r
            if r["diverged"]:
                left.append(i)
        todo = left
    return out


def _settable(eos, G=-1.0):
    """True if the library's EOS set-up accepts these parameters (host only)."""
    from .lattice import eos_setup

    try:
        eos_setup(eos, G)
        return True
    except L.PPLBMError:
        return False


def tune_to_width(families, grid=8, rounds=3, **planar_kw):
    """Shaping parameter giving a target interface width (Sec. IV.D, stability study:
    every EOS is set to the interface width the C-S EOS has at the same T_r).

    families: list of dicts with `make` (p -> (EOSParams, Relax)), the search interval
    `lo` < `hi` (p > 0) and the `target` continuous width (`interface_width_interp`).
    The width is taken to be monotone in p. Each round evaluates `grid` geometrically
    spaced values of every family in one batch, keeps the adjacent pair whose widths
    straddle the target and refines inside it; the answer is the linear interpolation
    of the last pair, verified by one more batched run. Each run starts from
    W = 10 and, if it diverges, from wider profiles (`planar_coexistence_started`).
    Candidates the EOS set-up rejects, and runs that diverge from every start,
    count as having no width.

    Returns one dict per family: ok, param, and the verification run's result
    (width, width_interp, E_percent, rho_v, rho_l, gamma) when ok."""
    nf = len(families)
    lo = [float(f["lo"]) for f in families]
    hi = [float(f["hi"]) for f in families]
    alive = [True] * nf
    brackets = [None] * nf   # (p0, w0, p1, w1) of the last round, per family
    for _ in range(rounds):
        cases, owner, params = [], [], []
        for k, f in enumerate(families):
            if not alive[k]:
                continue
            for p in np.geomspace(lo[k], hi[k], grid):
                eos, relax = f["make"](float(p))
                if _settable(eos):
                    cases.append((eos, relax))
                    owner.append(k)
                    params.append(float(p))
        res = planar_coexistence_started(cases, **planar_kw) if cases else []
        for k, f in enumerate(families):
            if not alive[k]:
                continue
            pts = [(p, r.get("width_interp", float("nan")) if r["converged"] else float("nan"))
                   for o, p, r in zip(owner, params, res) if o == k]
            bracket = None
            for (p0, w0), (p1, w1) in zip(pts, pts[1:]):
                if np.isfinite(w0) and np.isfinite(w1) and (w0 - f["target"]) * (w1 - f["target"]) <= 0:
                    bracket = (p0, w0, p1, w1)
                    break
            if bracket is None:
                alive[k] = False
                continue
            lo[k], hi[k] = bracket[0], bracket[2]
            brackets[k] = bracket
    out, cases, owner = [], [], []
    for k, f in enumerate(families):
        if not alive[k]:
            out.append(dict(ok=False))
            continue
        p0, w0, p1, w1 = brackets[k]
        p = p0 if w1 == w0 else p0 + (f["target"] - w0) * (p1 - p0) / (w1 - w0)
        out.append(dict(ok=True, param=float(p)))
        cases.append(f["make"](float(p)))
        owner.append(k)
    for k, r in zip(owner, planar_coexistence_started(cases, **planar_kw) if cases else []):
        r = dict(r)
        r.pop("profile", None)
        out[k].update(r)
        out[k]["ok"] = bool(r["converged"])
    return out


def stability_map(cases, Trs, vrs, steps=4000, check_every=500, u_limit=float("inf"), nx=600, ny=250, R=50,
                  film=25, V_d=0.1, tau_l=0.6, G=-1.0):
    """Droplet impact on a liquid film over reduced temperature x viscosity ratio
    (Sec. IV.D, stability map): (Lx, Ly) = (600, 250), periodic in x, bounce-back
    walls, film height 25, R = 50, V_d = 0.1 and tau_l = 0.6 (Re = 300), tau(rho)
    of Eq. RelaxationTime with tau_v = 0.5 + v_r (tau_l - 0.5), every other
    relaxation time 1.

    cases: dict name -> {T_r: (EOSParams, forcing, W)} (W: initial interface width,
    the planar width at that T_r); a (name, T_r) that is missing is reported as
    not run. Every (name, T_r, v_r) runs as one instance of one batch, initialised
    with the tanh profiles of the planar test between the Maxwell densities and the
    drop moving down with V_d. A run is stable when, at every check, its guard
    reports no non-finite or non-positive density (and, if u_limit is finite,
    max |u| < u_limit; the paper states no velocity criterion).

    Returns {(name, T_r, v_r): dict(run, stable, fail_step, reason, umax,
    mass_drift)}: reason is "diverged" (non-finite or non-positive density) or
    "velocity" (max |u| reached u_limit), fail_step the check at which it was seen,
    umax the largest max |u| over the checks passed."""
    import torch

    from . import _lib as LL
    from .lattice import Relax

    keys, lats, eoss, relaxes, inits = [], [], [], [], []
    for name, per_t in cases.items():
        for Tr in Trs:
            if Tr not in per_t or per_t[Tr] is None:
                continue
            eos, forcing, W = per_t[Tr]
            for vr in vrs:
                keys.append((name, Tr, vr))
                lats.append((nx, ny, LL.BC_WALLS_Y))
                eoss.append(eos)
                relaxes.append(Relax(kind=LL.RELAX_TWO_PHASE, forcing=forcing, tau_l=tau_l, visc_ratio=float(vr)))
                inits.append(W)
    out = {}
    for name, per_t in cases.items():
        for Tr in Trs:
            if Tr not in per_t or per_t[Tr] is None:
                for vr in vrs:
                    out[(name, Tr, vr)] = dict(run=False, stable=False)
    if not keys:
        return out
    b = Batch(lats, eoss, relaxes, G=G)
    b.set_isolation(True)
    for i, W in enumerate(inits):
        d = b.derived(i)
        rho, ux, uy = _inputs().impact(nx, ny, R, film, d["rho_v"], d["rho_l"], V_d, W=W)
        b.init_equilibrium(i, rho, ux, uy)
    b.set_plan(L.PLAN_GRAPH, 0)
    g0 = b.guard()
    g = g0
    alive = np.ones(len(keys), dtype=bool)
    reason = [None] * len(keys)
    fail_step = [None] * len(keys)
    umax = np.zeros(len(keys))
    done = 0
    while done < steps and alive.any():
        k = min(check_every, steps - done)
        b.step(k)
        done += k
        g = b.guard()
        status = np.asarray(b.instance_status())
        diverged = (status != 0) | (g[:, 2] > 0)
        fast = ~diverged & ~(g[:, 1] < u_limit)
        for i in np.nonzero(alive & (diverged | fast))[0]:
            reason[i] = "diverged" if diverged[i] else "velocity"
            fail_step[i] = done
        umax = np.where(alive & ~diverged, np.maximum(umax, g[:, 1]), umax)
        alive &= ~(diverged | fast)
    for i, key in enumerate(keys):
        out[key] = dict(run=True, stable=bool(alive[i]), fail_step=fail_step[i], reason=reason[i],
                        umax=float(umax[i]),
                        mass_drift=float(abs(g[i, 0] - g0[i, 0]) / g0[i, 0]) if alive[i] else float("nan"))
    b.close()
    torch.cuda.synchronize()
    return out


def kappa_for_surface_tension(gamma_target, gamma_at_kappa0):
    """kappa of the surface-tension control that turns a surface tension gamma_0
    (kappa = 0) into gamma_target, from gamma = (1 - kappa) gamma_0: the use the
    paper's Sec. V proposes, keeping the Weber number (and so the impact velocity)
    when a smaller alpha lowers the surface tension."""
    if not (gamma_target > 0 and gamma_at_kappa0 > 0):
        raise ValueError("surface tensions must be positive")
    return 1.0 - gamma_target / gamma_at_kappa0


def laplace_law(cases, radii, n=256, steps=40000, W=8.0, G=-1.0):
    """Static droplets: for each (EOSParams, Relax) case and radius R a centred
    droplet on a periodic n x n lattice, all advanced together in one batch for
    `steps` steps. Per droplet: dp = p_EOS(centre) - p_EOS(corner), with p_EOS =
    rho/3 + G psi^2/2 from the library's psi (Eq. InteractionPotential), and the
    equimolar radius; per case the 2-D Laplace law dp R = gamma + b/R fitted over the
    radii. Returns one dict per case: dpR (list), radius (list), gamma, b, diverged."""
    import torch

    m = len(cases) * len(radii)
    b = Batch([(n, n, L.BC_PERIODIC)] * m, [c[0] for c in cases for _ in radii],
              [c[1] for c in cases for _ in radii], G=G)
    b.set_isolation(True)
    for k in range(m):
        d = b.derived(k)
        b.init_equilibrium(k, _inputs().droplet(n, n, radii[k % len(radii)], d["rho_v"], d["rho_l"], W=W))
    b.autotune(trial_steps=4)
    b.step(steps)
    b.sync()
    status = b.instance_status()
    out = []
    for c in range(len(cases)):
        dpR, req, bad = [], [], False
        for j in range(len(radii)):
            k = c * len(radii) + j
            rho, _, _, psi = [t.cpu().numpy() for t in b.fields(k)]
            if status[k] != 0 or not np.all(np.isfinite(rho)):
                bad = True
                break
            p = rho / 3.0 + G * psi * psi / 2.0
            rin, rout = rho[n // 2, n // 2], rho[0, 0]
            Re = float(np.sqrt(((rho - rout) / (rin - rout)).sum() / np.pi))
            dpR.append(float(p[n // 2, n // 2] - p[0, 0]) * Re)
            req.append(Re)
        if bad:
            out.append(dict(diverged=True))
            continue
        slope, gamma = np.polyfit(1.0 / np.array(req), np.array(dpR), 1)
        out.append(dict(diverged=False, dpR=dpR, radius=req, gamma=float(gamma), b=float(slope)))
    b.close()
    torch.cuda.synchronize()
    return out


def stability_study(Trs, vrs, steps=4000, a_cs=0.363, a_v=2.0, check_every=500):
    """The stability study of Sec. IV.D end to end, on the batched engine:

    1. planar C-S interfaces with a = a_cs at every T_r (Li forcing): simulated
       densities and the continuous width w(T_r);
    2. the Smooth C-S EOS (a_l = a_cs, a_v) tuned in alpha, and the Peng C-S EOS
       (a = a_cs, Guo forcing) tuned in r_theta, to the same width at each T_r
       (`tune_to_width`); a T_r at which no parameter in the search interval gives
       a converged interface of that width is not run for that EOS;
    3. the droplet impact at Re = 300 for every (EOS, T_r, v_r) in one batch
       (`stability_map`), each started with the planar width of its T_r.

    Returns dict(planar={name: {T_r: result}}, tuned={name: {T_r: param}},
    map={(name, T_r, v_r): result})."""
    from .lattice import EOSParams, Relax

    cs_cases = [(EOSParams(L.EOS_CS, Tr, a_cs, a_cs, 0.5), Relax()) for Tr in Trs]
    cs = planar_coexistence_started(cs_cases)
    fams, owners = [], []
    for Tr, r in zip(Trs, cs):
        if not r["converged"]:
            continue
        fams.append(dict(target=r["width_interp"], lo=0.02, hi=2.0,
                         make=lambda p, Tr=Tr: (EOSParams(L.EOS_SMOOTH, Tr, a_cs, a_v, p), Relax())))
        owners.append(("Smooth C-S", Tr))
        fams.append(dict(target=r["width_interp"], lo=0.005, hi=2.0,
                         make=lambda p, Tr=Tr: (EOSParams(L.EOS_PENG, Tr, a_cs, a_cs, 0.5, r_theta=p),
                                                Relax(forcing=L.FORCING_GUO))))
        owners.append(("Peng C-S", Tr))
    tuned = tune_to_width(fams)
    planar = {"C-S": {}, "Smooth C-S": {}, "Peng C-S": {}}
    params = {"Smooth C-S": {}, "Peng C-S": {}}
    cases = {"C-S": {}, "Smooth C-S": {}, "Peng C-S": {}}
    for Tr, r, (eos, relax) in zip(Trs, cs, cs_cases):
        r = {k: v for k, v in r.items() if k != "profile"}
        planar["C-S"][Tr] = r
        if r["converged"]:
            cases["C-S"][Tr] = (eos, relax.forcing, max(4.0, float(r["width"])))
    for (name, Tr), f, t in zip(owners, fams, tuned):
        planar[name][Tr] = t
        if t.get("ok"):
            params[name][Tr] = t["param"]
            eos, relax = f["make"](t["param"])
            cases[name][Tr] = (eos, relax.forcing, max(4.0, float(t["width"])))
    m = stability_map(cases, Trs, vrs, steps=steps, check_every=check_every)
    return dict(planar=planar, tuned=params, map=m)


def weber_matching(Trs, a_cs=0.363, a_v=2.0, verify=True, radii=(24.0, 32.0, 48.0), n=192, steps=60000):
    """Sec. V's proposal across T_r: the Smooth C-S EOS is set to the C-S interface
    width (alpha tuned as in the stability study, `tune_to_width`), which changes
    its surface tension; the surface-tension control with
    kappa = 1 - gamma_CS / gamma_alpha (planar Eq. SurfaceTension values) gives it
    the C-S surface tension back, so impacts keep their Weber number at an unchanged
    impact velocity. With `verify`, static droplets of both (C-S, and Smooth C-S
    with that kappa) at every T_r run in one batch and their Laplace fits
    (`laplace_law`) are returned beside the planar values.

    Returns {T_r: dict(alpha, width, gamma_cs, gamma_alpha, kappa[, laplace_cs,
    laplace_matched])}; a T_r whose C-S interface or width tuning fails is absent."""
    from .lattice import EOSParams, Relax

    cs_cases = [(EOSParams(L.EOS_CS, Tr, a_cs, a_cs, 0.5), Relax()) for Tr in Trs]
    cs = planar_coexistence_started(cs_cases)
    fams, keep = [], []
    for Tr, r in zip(Trs, cs):
        if r["converged"]:
            fams.append(dict(target=r["width_interp"], lo=0.02, hi=2.0,
                             make=lambda p, Tr=Tr: (EOSParams(L.EOS_SMOOTH, Tr, a_cs, a_v, p), Relax())))
            keep.append((Tr, r))
    tuned = tune_to_width(fams) if fams else []
    out = {}
    for (Tr, r), t in zip(keep, tuned):
        if not t.get("ok") or not t.get("converged", True):
            continue
        k = kappa_for_surface_tension(r["gamma"], t["gamma"])
        out[Tr] = dict(alpha=t["param"], width=r["width_interp"], gamma_cs=r["gamma"], gamma_alpha=t["gamma"],
                       kappa=k)
    if verify and out:
        cases = []
        for Tr, v in out.items():
            cases.append((EOSParams(L.EOS_CS, Tr, a_cs, a_cs, 0.5), Relax()))
            cases.append((EOSParams(L.EOS_SMOOTH, Tr, a_cs, a_v, v["alpha"]), Relax(kappa=v["kappa"])))
        lap = laplace_law(cases, radii, n=n, steps=steps)
        for j, Tr in enumerate(out):
            c, m = lap[2 * j], lap[2 * j + 1]
            out[Tr]["laplace_cs"] = None if c["diverged"] else c["gamma"]
            out[Tr]["laplace_matched"] = None if m["diverged"] else m["gamma"]
    return out


def _main(argv=None):
    """Command line: the stability study over T_r in [0.35, 0.75] (step 0.05) and
    v_r in 2..24 (step 2), printed as a map and as JSON; or, with --weber, the
    surface-tension control that keeps the C-S surface tension at each T_r."""
    import argparse
    import json
    import time

    ap = argparse.ArgumentParser(description=_main.__doc__)
    ap.add_argument("--steps", type=int, default=4000, help="impact steps per run (t* = steps V_d / D)")
    ap.add_argument("--json", default=None, help="write the full result to this file")
    ap.add_argument("--weber", action="store_true",
                    help="instead: the surface-tension control that keeps the C-S surface tension for the "
                         "width-matched Smooth C-S at each T_r, with Laplace-law checks (Sec. V)")
    args = ap.parse_args(argv)
    if args.weber:
        Trs = [round(0.35 + 0.05 * k, 2) for k in range(9)]
        t0 = time.perf_counter()
        res = weber_matching(Trs)
        print("  T_r   alpha   gamma_CS   gamma_alpha   kappa    Laplace C-S   Laplace Smooth+kappa")
        for Tr, v in res.items():
            print("  %.2f  %.4f  %.4e  %.4e  %+.4f  %s  %s" % (
                Tr, v["alpha"], v["gamma_cs"], v["gamma_alpha"], v["kappa"],
                "%.4e" % v["laplace_cs"] if v.get("laplace_cs") else "diverged",
                "%.4e" % v["laplace_matched"] if v.get("laplace_matched") else "diverged"))
        print("wall %.1f s" % (time.perf_counter() - t0))
        if args.json:
            with open(args.json, "w") as fh:
                json.dump({str(k): v for k, v in res.items()}, fh, indent=1, default=float)
        return
    Trs = [round(0.35 + 0.05 * k, 2) for k in range(9)]
    vrs = list(range(2, 25, 2))
    t0 = time.perf_counter()
    res = stability_study(Trs, vrs, steps=args.steps)
    wall = time.perf_counter() - t0
    for name in ("C-S", "Smooth C-S", "Peng C-S"):
        print(name)
        for Tr in Trs:
            cells = []
            for vr in vrs:
                r = res["map"][(name, Tr, vr)]
                cells.append("S" if r["stable"] else ("-" if not r["run"] else "x"))
            p = res["planar"][name].get(Tr, {})
            ratio = p["rho_l"] / p["rho_v"] if "rho_v" in p and p.get("converged") else float("nan")
            print("  T_r %.2f  %s  rho_l/rho_v %.4g" % (Tr, " ".join(cells), ratio))
    print("v_r: " + " ".join(str(v) for v in vrs))
    print("wall %.1f s" % wall)
    if args.json:
        out = dict(planar={n: {str(k): v for k, v in d.items()} for n, d in res["planar"].items()},
                   tuned={n: {str(k): v for k, v in d.items()} for n, d in res["tuned"].items()},
                   map=[dict(eos=k[0], Tr=k[1], vr=k[2], **v) for k, v in res["map"].items()], wall_s=wall)
        with open(args.json, "w") as fh:
            json.dump(out, fh, indent=1, default=float)


if __name__ == "__main__":
    _main()
