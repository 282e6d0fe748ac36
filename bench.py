"""Benchmark of the pseudopotential D2Q9 LBM step on GB300.

Default workload (one bench step = one LBM time step of all four lattices):
four 512 x 512 periodic static droplets, radii 32, 48, 64, 96, reduced
temperature 0.6, Smooth C-S EOS (a_l = 0.387, a_v = 2, alpha = 0.834),
all relaxation times 1, Li forcing with sigma from the mechanical-stability
condition; initial tanh profiles of width 8. The four lattices' buffers
(f in/out, psi, moments: ~180 MB per step) exceed the 126 MB L2, so the state
streams from HBM every step (no explicit flush).

Prints one JSON line: MLUPS (million lattice-node updates per second) over all
ranks, the roofline of the dominant kernel, an end-to-end figure through the
host-buffer C-ABI call, clocks sampled during the timed region and the oracle
timed on the host cores (rank 0 only).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

RADII = (32, 48, 64, 96)
NX = NY = 512
TR, A_L, A_V, ALPHA = 0.6, 0.387, 2.0, 0.834
METRIC = "D2Q9 pseudopotential MLUPS (4 x 512^2 static droplets, T_r=0.6, Smooth C-S, FP64)"
WORKLOAD = "static droplets 512x512 periodic, R in {32,48,64,96}, T_r=0.6, Smooth C-S (a_l=0.387, a_v=2, alpha=0.834), tau=1, Li forcing"
E2E_INNER = 100  # LBM steps per end-to-end call

# FP64 instructions of one node update per kernel (unit relaxation times, Li forcing,
# bulk nodes), counted from the kernels' arithmetic; ncu's FP64-pipe cycles agree.
FP64_OPS_PER_NODE = {"rho_psi": 33, "collide": 51}
BYTES_PER_NODE = {"rho_psi": 72 + 32, "collide": 24 + 8 + 72}
# FP64 instructions of one MacCormack step per grid point: predictor 113, corrector
# 119, two EOS passes of 27 (the kernels' arithmetic; ncu's sm__inst_executed_pipe_fp64
# on the 2048 x 1024 grid, profiles/k_fd_update_k_fd_eos_2048x1024.md)
FD_FP64_PER_POINT = 113 + 119 + 2 * 27
# FP64 instructions per node of the two-phase (tau(rho), walls) batched passes of the
# impact sweep (ncu sm__inst_executed_pipe_fp64, profiles/k_batch_shear_tau_impact_sweep.md)
IMPACT_FP64_PER_NODE = 42.0 + 67.5

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of each
# batched pass on this workload, averaged over three launches of an ncu capture of
# `bench.py --profile-batch` (profiles/k_batch_collide_k_batch_rho_psi_droplets512.md).
# They hold for the kernel sources whose digest is recorded with them; once those
# sources change, traffic is reported as null until the capture is repeated.
TRAFFIC = {"sources": "31b781817864a4b6", "rho_psi": 75548160 + 2560768, "collide": 33602987 + 13737131}
KERNEL_SOURCES = ("batch.cu", "step_device.cuh", "eos_dev.cuh", "eos.cuh", "fp64.cuh", "internal.h")


def kernel_sources_digest():
    """sha256 (first 16 hex digits) over the sources the batched step kernels are
    compiled from, in a fixed order, each preceded by its file name."""
    import hashlib

    d = os.path.join(ROOT, "paper_2107_06355_gb300", "csrc")
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        h.update(name.encode())
        with open(os.path.join(d, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def step_traffic():
    if TRAFFIC["sources"] is None or TRAFFIC["sources"] != kernel_sources_digest():
        return None
    return TRAFFIC["rho_psi"] + TRAFFIC["collide"]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def build_lib():
    from paper_2107_06355_gb300 import build
    build.build()


def make_droplets(torch, stream):
    import lbm_inputs as I
    import paper_2107_06355_gb300 as P

    eos = P.EOSParams(P.EOS_SMOOTH, TR, A_L, A_V, ALPHA)
    relax = P.Relax()
    sims, rho0s = [], []
    for R in RADII:
        s = P.Simulation(NX, NY, P.BC_PERIODIC, eos, relax, stream=stream)
        d = s.derived()
        rho0 = I.droplet(NX, NY, R, d["rho_v"], d["rho_l"], W=8.0)
        s.init_equilibrium(rho0)
        sims.append(s)
        rho0s.append(rho0)
    return sims, rho0s


def time_oracle_sample(max_seconds=20.0):
    """The oracle (numpy, as it stands) on one 512^2 droplet lattice of the workload."""
    import lbm_inputs as I
    from oracle import eos as E
    from oracle import lbm as L

    e = E.make_eos(E.MODE_SMOOTH, TR, A_L, A_V, ALPHA)
    lat = L.Lattice(NX, NY, L.BC_PERIODIC_X | L.BC_PERIODIC_Y, e, L.Relax(sigma=e.sigma()))
    f = lat.init_equilibrium(I.droplet(NX, NY, RADII[1], e.rho_v, e.rho_l, W=8.0))
    f = lat.step(f, 1)
    n, t0 = 0, time.perf_counter()
    while True:
        f = lat.step(f, 1)
        n += 1
        dt = time.perf_counter() - t0
        if dt > max_seconds or n >= 200:
            break
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    threads = _numpy_threads()
    return {"value": NX * NY * n / dt / 1e6, "unit": "MLUPS", "cores": threads, "host_cores": cores,
            "kind": "oracle",
            "sample": f"{n} LBM steps of one 512x512 droplet lattice (R=48) of the workload, {dt:.1f} s"}


def _numpy_threads():
    try:
        from threadpoolctl import threadpool_info
        return max((i.get("num_threads", 1) for i in threadpool_info()), default=1)
    except Exception:
        return 1


def profile_case():
    """One 2048 x 1024 periodic droplet lattice (R = 100) of the workload's EOS, 3 steps:
    369 MB of workspace (larger than L2), 3 launches of each step kernel."""
    import torch
    import lbm_inputs as I
    import paper_2107_06355_gb300 as P

    build_lib()
    s = P.Simulation(2048, 1024, P.BC_PERIODIC, P.EOSParams(P.EOS_SMOOTH, TR, A_L, A_V, ALPHA), P.Relax())
    d = s.derived()
    s.init_equilibrium(I.droplet(2048, 1024, 100, d["rho_v"], d["rho_l"], W=8.0))
    s.step(3)
    s.sync()
    torch.cuda.synchronize()
    print("profile case done")


def profile_batch(kappa=0.0):
    """The benchmark's four 512 x 512 droplets in one batch, launches plan, 3 steps:
    3 launches of each batched pass over 1,048,576 nodes (184 MB of state, > L2);
    kappa != 0 runs them with the surface-tension control."""
    import torch
    import lbm_inputs as I
    import paper_2107_06355_gb300 as P

    build_lib()
    specs = [dict(kind="droplet", nx=NX, ny=NY, R=R, Tr=TR) for R in RADII]
    b, _, _, _ = make_batch(P, I, specs, torch.cuda.current_stream(), kappa=kappa)
    b.set_plan(P.PLAN_LAUNCHES, 0)
    b.step(3)
    b.sync()
    torch.cuda.synchronize()
    print("profile batch done")


def profile_fd():
    """The finite-difference solver on the 2048 x 1024 droplet grid of fd_throughput,
    3 steps: 3 launches of each of its two kernels per half-step pair."""
    import torch
    import lbm_inputs as I
    import paper_2107_06355_gb300 as P

    build_lib()
    eos = P.EOSParams(P.EOS_SMOOTH, TR, A_L, A_V, ALPHA)
    d = P.eos_setup(eos)
    fd = P.FDSolver(2048, 1024, eos, dx=1.0)
    rho = I.droplet(2048, 1024, 100, d["rho_v"], d["rho_l"], W=8.0)
    fd.set_state(rho, np.zeros_like(rho), np.zeros_like(rho))
    fd.step(3, 0.4)
    torch.cuda.synchronize()
    print("profile fd done")


def profile_adjoint():
    """Checkpointed forward and reverse pass on a 1024 x 1024 droplet (T_r = 0.5,
    tau = 1), 12 steps with interval 4, gradient slots of alpha: 12 launches of each
    adjoint kernel on 75 MB states (> L2 with the adjoint planes)."""
    import ctypes as C
    import torch
    import lbm_inputs as I
    import paper_2107_06355_gb300 as P
    from paper_2107_06355_gb300 import _lib as L

    build_lib()
    nx = ny = 1024
    steps, interval = 12, 4
    sim = P.Simulation(nx, ny, P.BC_PERIODIC, P.EOSParams(P.EOS_SMOOTH, 0.5, 0.363, 2.0, 0.775), P.Relax())
    d = sim.derived()
    sim.init_equilibrium(I.droplet(nx, ny, 192.0, d["rho_v"], d["rho_l"], W=7.0))
    dev = sim.device
    ckpt = torch.empty((steps // interval, 9, ny, nx), dtype=torch.float64, device=dev)
    seg = torch.empty((interval, 9, ny, nx), dtype=torch.float64, device=dev)
    lam = torch.ones((9, ny, nx), dtype=torch.float64, device=dev)
    lam0 = torch.empty_like(lam)
    grad = torch.zeros(L.NGRAD, dtype=torch.float64, device=dev)
    nb = L.lib().pplbm_adjoint_workspace_bytes(C.byref(sim.lattice))
    ws = torch.empty(nb // 8 + 1, dtype=torch.float64, device=dev)
    p = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    L.check(L.lib().pplbm_adjoint_set_slots(sim.ctx, (1 << 9) - 1), sim.ctx)  # alpha's slots, as in adjoint_cost
    L.check(L.lib().pplbm_forward_checkpointed(sim.ctx, steps, interval, p(ckpt)), sim.ctx)
    L.check(L.lib().pplbm_backward_checkpointed(sim.ctx, steps, interval, p(ckpt), p(seg), p(lam), p(lam0), p(grad),
                                                p(ws), nb), sim.ctx)
    torch.cuda.synchronize()
    sim.close()
    print("profile adjoint done")


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    timed = []
    for k in range(args.warmup + args.steps):
        r = time_oracle_sample(max_seconds=max(2.0, 60.0 / max(1, args.steps + args.warmup)))
        if k >= args.warmup:
            timed.append(r)
    last = timed[-1]
    val = sum(r["value"] for r in timed) / len(timed)   # mean rate over the timed samples
    nodes = NX * NY * len(RADII)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": nodes / (val * 1e6) * 1e3,   # one step of the whole 4-lattice workload at this rate
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": last["cores"], "kind": "oracle",
                             "sample": last["sample"]},
            "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def serial_sims(torch, stream):
    sims, rho0s = make_droplets(torch, stream)
    return sims, rho0s


def make_batch(P, I, specs, stream, kappa=0.0):
    """A Batch over `specs` (dicts with nx, ny, Tr, kind, R) with tanh initial fields;
    kappa: the surface-tension control of every instance (0 = off)."""
    eos = [P.EOSParams(P.EOS_SMOOTH, s["Tr"], s.get("a_l", A_L), s.get("a_v", A_V), s.get("alpha", ALPHA))
           for s in specs]
    relax = [P.Relax(kappa=kappa) for _ in specs]
    b = P.Batch([(s["nx"], s["ny"], P.BC_PERIODIC) for s in specs], eos, relax, stream=stream)
    inits = []
    for k, s in enumerate(specs):
        d = b.derived(k)
        if s["kind"] == "planar":
            rho = I.planar(s["nx"], s["ny"], d["rho_v"], d["rho_l"], W=8.0)
        else:
            rho = I.droplet(s["nx"], s["ny"], s["R"], d["rho_v"], d["rho_l"], W=8.0)
        b.init_equilibrium(k, rho)
        inits.append(rho)
    return b, eos, relax, inits


def time_device(torch, stream, fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def sweep_comparison(torch, stream, steps):
    """64-lattice sweep (seed 210706355): batched engine vs one context per lattice,
    the latter as per-instance CUDA graphs (the baseline) and as plain launches."""
    import lbm_inputs as I
    import paper_2107_06355_gb300 as P

    specs = I.batch_specs()
    for s in specs:
        s["a_l"], s["a_v"], s["alpha"] = 0.363, 2.0, 0.775
    nodes = sum(s["nx"] * s["ny"] for s in specs)
    b, eos, relax, inits = make_batch(P, I, specs, stream)
    plan = b.autotune(trial_steps=4)
    b.step(2)
    ms_b = time_device(torch, stream, lambda: b.step(steps))
    b.sync()
    b.close()
    del b
    torch.cuda.empty_cache()
    sims = []
    for k, s in enumerate(specs):
        sim = P.Simulation(s["nx"], s["ny"], P.BC_PERIODIC, eos[k], relax[k], stream=stream)
        sim.init_equilibrium(inits[k])
        sims.append(sim)

    def serial():
        for _ in range(steps):
            for sim in sims:
                sim.step(1)

    for sim in sims:
        sim.step(2)
    ms_s = time_device(torch, stream, serial)

    # the baseline the batch is measured against: per-instance CUDA graphs of two
    # steps (pplbm_step only enqueues kernels), replayed one instance after another
    import ctypes as C
    from paper_2107_06355_gb300 import _lib as L

    for sim in sims:
        sim.sync()
    cs = torch.cuda.Stream()
    graphs = []
    for sim in sims:
        L.check(L.lib().pplbm_set_stream(sim.ctx, C.c_void_p(cs.cuda_stream)), sim.ctx)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cs):
            sim.step(2)
        graphs.append(g)

    def serial_graphs():
        for _ in range(steps // 2):
            for g in graphs:
                g.replay()

    cur = torch.cuda.current_stream()
    for g in graphs:
        g.replay()
    ms_g = time_device(torch, cur, serial_graphs) * steps / (2 * (steps // 2))
    torch.cuda.synchronize()
    del graphs
    for sim in sims:
        sim.sync()
        sim.close()
    mode = {0: "launches", 1: "graph", 2: "persistent"}[plan["mode"]]
    return {"instances": len(specs), "nodes": nodes, "steps": steps, "plan": mode,
            "tile_width": plan["tile_width"] or "per-instance",
            "batched_instance_steps_per_s": len(specs) * steps / (ms_b / 1e3),
            "serial_instance_steps_per_s": len(specs) * steps / (ms_g / 1e3),
            "batched_mlups": nodes * steps / (ms_b / 1e3) / 1e6,
            "serial_mlups": nodes * steps / (ms_g / 1e3) / 1e6,
            "serial_baseline": "64 per-instance CUDA graphs of 2 steps, replayed serially",
            "speedup": ms_g / ms_b,
            "serial_plain_launches_mlups": nodes * steps / (ms_s / 1e3) / 1e6}


def adjoint_cost(torch, steps=2000, interval=45):
    """Adjoint configuration (256 x 256 droplet, R = 48, T_r = 0.5, tau = 1): time of a
    checkpointed forward rollout vs its reverse pass (recomputation + adjoint kernels)."""
    import ctypes as C
    import lbm_inputs as I
    import paper_2107_06355_gb300 as P
    from paper_2107_06355_gb300 import _lib as L

    nx = ny = 256
    eos = P.EOSParams(P.EOS_SMOOTH, 0.5, 0.363, 2.0, 0.775)
    sim = P.Simulation(nx, ny, P.BC_PERIODIC, eos, P.Relax())
    d = sim.derived()
    rho0 = I.droplet(nx, ny, 48.0, d["rho_v"], d["rho_l"], W=7.0)
    nseg = -(-steps // interval)
    dev = sim.device
    ckpt = torch.empty((nseg, 9, ny, nx), dtype=torch.float64, device=dev)
    seg = torch.empty((interval, 9, ny, nx), dtype=torch.float64, device=dev)
    lam = torch.ones((9, ny, nx), dtype=torch.float64, device=dev)
    lam0 = torch.empty_like(lam)
    grad = torch.zeros(L.NGRAD, dtype=torch.float64, device=dev)
    nb = L.lib().pplbm_adjoint_workspace_bytes(C.byref(sim.lattice))
    ws = torch.empty(nb // 8 + 1, dtype=torch.float64, device=dev)
    p = lambda t: C.c_void_p(t.data_ptr())
    lib = L.lib()
    alpha_slots = (1 << 9) - 1   # the shaped-branch constants and the Li-term scale: all alpha moves
    out = {}
    # every EOS constant and the Li-term scale (the kappa slot would run the surface-tension kernels)
    eos_slots = (1 << L.GRAD_NAMES.index("kappa")) - 1
    for label, mask in (("alpha", alpha_slots), ("all_slots", eos_slots)):
        L.check(lib.pplbm_adjoint_set_slots(sim.ctx, mask), sim.ctx)
        res = []
        for _ in range(2):  # second round is timed
            sim.init_equilibrium(rho0)
            t_f = time_device(torch, torch.cuda.current_stream(),
                              lambda: L.check(lib.pplbm_forward_checkpointed(sim.ctx, steps, interval, p(ckpt)),
                                              sim.ctx))
            t_b = time_device(torch, torch.cuda.current_stream(),
                              lambda: L.check(lib.pplbm_backward_checkpointed(sim.ctx, steps, interval, p(ckpt),
                                                                              p(seg), p(lam), p(lam0), p(grad), p(ws),
                                                                              nb), sim.ctx))
            res = (t_f, t_b)
        out[label] = res
    # the same rollout with every step's psi and moments kept (4 planes x 2,000 steps =
    # 4.2 GB): no recomputation in the reverse pass
    L.check(lib.pplbm_adjoint_set_slots(sim.ctx, alpha_slots), sim.ctx)
    fields = torch.empty((steps, 4, ny, nx), dtype=torch.float64, device=dev)
    res = []
    for _ in range(2):
        sim.init_equilibrium(rho0)
        t_f = time_device(torch, torch.cuda.current_stream(),
                          lambda: L.check(lib.pplbm_forward_stored(sim.ctx, steps, p(fields)), sim.ctx))
        t_b = time_device(torch, torch.cuda.current_stream(),
                          lambda: L.check(lib.pplbm_backward_stored(sim.ctx, steps, p(fields), p(lam), p(lam0),
                                                                    p(grad), p(ws), nb), sim.ctx))
        res = (t_f, t_b)
    out["stored"] = res
    del fields
    sim.close()
    f_ms, b_ms = out["alpha"]
    return {"config": f"256x256 droplet R=48, T_r=0.5, {steps} steps, checkpoint interval {interval}, "
                      "gradients w.r.t. rho0 and alpha",
            "forward_ms": f_ms, "backward_ms": b_ms, "adjoint_over_forward": b_ms / f_ms,
            "forward_mlups": nx * ny * steps / (f_ms / 1e3) / 1e6,
            "adjoint_over_forward_all_slots": out["all_slots"][1] / out["all_slots"][0],
            "stored_fields": {"forward_ms": out["stored"][0], "backward_ms": out["stored"][1],
                              "adjoint_over_forward": out["stored"][1] / out["stored"][0],
                              "bytes": 32 * nx * ny * steps}}


def eos_variant_throughput(torch, steps=1000):
    """The bench workload (4 x 512^2 droplets, tau = 1) with each EOS the kernels
    support (T_r = 0.6; the two Guo-forced EOS at 0.7), and the Smooth C-S with the
    surface-tension control, batched graph plan: MLUPS per variant."""
    import lbm_inputs as I
    import paper_2107_06355_gb300 as P

    variants = {
        "cs_a0.387_li": (P.EOSParams(P.EOS_CS, 0.6, 0.387, 0.387, 0.5), P.Relax()),
        "smooth_alpha0.834_li": (P.EOSParams(P.EOS_SMOOTH, 0.6, 0.387, 2.0, 0.834), P.Relax()),
        # the same with the surface-tension control (Sec. V's technique): its cost per step
        "smooth_alpha0.834_li_kappa0.5": (P.EOSParams(P.EOS_SMOOTH, 0.6, 0.387, 2.0, 0.834), P.Relax(kappa=0.5)),
        # Peng + Guo droplets diverge below T_r ~ 0.65 (the paper's minimum for that method)
        "peng_r0.45_Tr0.7_guo": (P.EOSParams(P.EOS_PENG, 0.7, 0.387, 0.387, 0.5, r_theta=0.45),
                                 P.Relax(forcing=P.FORCING_GUO)),
        # Modified Smooth + Guo droplets also diverge at T_r = 0.6 (the oracle agrees); 0.7 is stable
        "modsmooth_alpha0.446_Tr0.7_guo": (P.EOSParams(P.EOS_SMOOTH_MOD, 0.7, 0.387, 2.0, 0.446),
                                           P.Relax(forcing=P.FORCING_GUO)),
    }
    out = {}
    for name, (eos, relax) in variants.items():
        b = P.Batch([(NX, NY, P.BC_PERIODIC)] * 4, [eos] * 4, [relax] * 4)
        d = b.derived(0)
        for k, R in enumerate(RADII):
            b.init_equilibrium(k, I.droplet(NX, NY, R, d["rho_v"], d["rho_l"], W=8.0))
        b.set_plan(P.PLAN_GRAPH, 0)
        b.step(20)
        ms = time_device(torch, torch.cuda.current_stream(), lambda: b.step(steps))
        try:
            b.sync()
            out[name] = 4 * NX * NY * steps / (ms / 1e3) / 1e6
        except P.PPLBMError as e:
            out[name] = f"diverged ({e})"
        b.close()
    return out


def impact_sweep_throughput(torch, steps=2000):
    """A slice of the stability study (Sec. IV.D) on the batched engine: droplet
    impact at Re = 300 on (600, 250) lattices with walls, C-S a = 0.363, Li forcing,
    two-phase tau(rho), T_r in {0.45, ..., 0.75} x v_r in {2, ..., 10}: 35 instances,
    5.25 M nodes, graph plan with divergence isolation. Every run is stable here, so
    all nodes count."""
    b, n_inst = impact_sweep_batch()
    b.step(20)
    ms = time_device(torch, torch.cuda.current_stream(), lambda: b.step(steps))
    g = b.guard()
    stable = int(((np.asarray(b.instance_status()) == 0) & (g[:, 2] == 0)).sum())
    b.close()
    nodes = 600 * 250 * n_inst
    mlups = nodes * steps / (ms / 1e3) / 1e6 if stable == n_inst else None
    out = {"instances": n_inst, "stable": stable, "nodes": nodes, "steps": steps, "mlups": mlups}
    if mlups is not None and IMPACT_FP64_PER_NODE is not None:
        _, sm_max, _ = load_peaks()
        peak = 2 * 152 * sm_max * 1e6
        achieved = IMPACT_FP64_PER_NODE * mlups * 1e6
        out["roofline"] = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                           "frac": achieved / peak, "fp64_per_node": IMPACT_FP64_PER_NODE}
    return out


def impact_sweep_batch():
    """The impact-sweep batch, initialised, on the graph plan: (Batch, instances)."""
    import paper_2107_06355_gb300 as P
    from paper_2107_06355_gb300 import sweeps as SW

    # initial interface widths: the planar C-S (a = 0.363) widths at each T_r
    width = {0.45: 6.0, 0.50: 7.0, 0.55: 7.0, 0.60: 9.0, 0.65: 9.0, 0.70: 10.0, 0.75: 11.0}
    Trs = sorted(width)
    vrs = [2, 4, 6, 8, 10]
    lats, eoss, relaxes, Ws = [], [], [], []
    for Tr in Trs:
        for vr in vrs:
            lats.append((600, 250, P.BC_WALLS_Y))
            eoss.append(P.EOSParams(P.EOS_CS, Tr, 0.363, 0.363, 0.5))
            relaxes.append(P.Relax(kind=P.RELAX_TWO_PHASE, tau_l=0.6, visc_ratio=float(vr)))
            Ws.append(width[Tr])
    b = P.Batch(lats, eoss, relaxes)
    b.set_isolation(True)
    for i in range(len(lats)):
        d = b.derived(i)
        b.init_equilibrium(i, *SW._impact_profile(600, 250, 50, 25, d["rho_v"], d["rho_l"], 0.1, Ws[i]))
    b.set_plan(P.PLAN_GRAPH, 0)
    return b, len(lats)


def profile_impact():
    """The impact-sweep batch (35 lattices 600 x 250, two-phase tau, walls), launches
    plan, 3 steps: 3 launches of each two-phase batched pass over 5.25 M nodes."""
    import torch
    import paper_2107_06355_gb300 as P

    build_lib()
    b, _ = impact_sweep_batch()
    b.set_plan(P.PLAN_LAUNCHES, 0)
    b.step(3)
    b.sync()
    torch.cuda.synchronize()
    b.close()
    print("profile impact done")


def fd_throughput(torch, steps=200):
    """The finite-difference solver (App. A) on a 2048 x 1024 periodic droplet grid
    (dx = 1, Smooth C-S at T_r = 0.6): grid-point updates per second. dt = 0.4: with
    the paper's 0.8 dx^2 the static droplet diverges in this scheme (CPU oracle too)."""
    import lbm_inputs as I
    import paper_2107_06355_gb300 as P

    nx, ny = 2048, 1024
    eos = P.EOSParams(P.EOS_SMOOTH, TR, A_L, A_V, ALPHA)
    d = P.eos_setup(eos)
    fd = P.FDSolver(nx, ny, eos, dx=1.0)
    rho = I.droplet(nx, ny, 100, d["rho_v"], d["rho_l"], W=8.0)
    z = torch.zeros((ny, nx), dtype=torch.float64)
    fd.set_state(rho, z, z)
    fd.step(5, 0.4)
    ms = time_device(torch, torch.cuda.current_stream(), lambda: fd.step(steps, 0.4))
    fd.sync()
    r = fd.get_state()[0]
    ok = bool(torch.isfinite(r).all())
    fd.close()
    _, sm_max, _ = load_peaks()
    peak = 2 * 152 * sm_max * 1e6
    achieved = FD_FP64_PER_POINT * nx * ny * steps / (ms / 1e3)
    return {"grid": f"{nx}x{ny}, dx=1, dt=0.4", "mlups": nx * ny * steps / (ms / 1e3) / 1e6,
            "ms_per_step": ms / steps, "finite": ok, "launches_per_step": 4,
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                         "frac": achieved / peak, "fp64_per_point_step": FD_FP64_PER_POINT,
                         "peak_source": f"2 FP64 instr/clk/SM x 152 SMs x {sm_max:.0f} MHz"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=12000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--plan", default="auto", choices=["auto", "launches", "graph", "persistent"],
                    help="batched-engine plan for the timed run (auto: autotuned)")
    ap.add_argument("--profile-case", action="store_true",
                    help="run one 2048x1024 droplet lattice for 3 steps (a small case for ncu captures) and exit")
    ap.add_argument("--profile-adjoint", action="store_true", help="checkpointed adjoint on 1024 x 1024 (for ncu)")
    ap.add_argument("--profile-impact", action="store_true", help="3 steps of the impact-sweep batch (for ncu)")
    ap.add_argument("--profile-fd", action="store_true", help="3 steps of the FD solver on 2048 x 1024 (for ncu)")
    ap.add_argument("--profile-batch", action="store_true",
                    help="run the four 512x512 droplets through the batched engine (launches plan) for 3 steps and exit")
    ap.add_argument("--profile-kappa", type=float, default=None,
                    help="as --profile-batch, with the surface-tension control at this kappa")
    args = ap.parse_args()
    if args.profile_case:
        return profile_case()
    if args.profile_batch:
        return profile_batch()
    if args.profile_kappa is not None:
        return profile_batch(args.profile_kappa)
    if args.profile_fd:
        return profile_fd()
    if args.profile_impact:
        return profile_impact()
    if args.profile_adjoint:
        return profile_adjoint()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import lbm_inputs as I
    import paper_2107_06355_gb300 as P

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or ws == 1:
        build_lib()
    if ws > 1:
        torch.distributed.barrier()
        build_lib()  # no-op after rank 0 (up to date)

    stream = torch.cuda.current_stream()
    specs = [dict(kind="droplet", nx=NX, ny=NY, R=R, Tr=TR) for R in RADII]
    batch, _, _, rho0s = make_batch(P, I, specs, stream)
    nodes = NX * NY * len(specs)
    if args.plan == "auto":
        plan = batch.autotune(trial_steps=20)
    else:
        batch.set_plan({"launches": P.PLAN_LAUNCHES, "graph": P.PLAN_GRAPH, "persistent": P.PLAN_PERSISTENT}[args.plan], 0)
        plan = batch.plan()
    batch.step(args.warmup)
    torch.cuda.synchronize()
    batch.enable_timing(4)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    batch.step(args.steps)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    call_ms, call_steps = batch.times()
    batch.enable_timing(0)
    from paper_2107_06355_gb300.replicas import max_over_ranks

    ms = max_over_ranks(ms, device="cuda")  # each rank runs its own replica; slowest rank sets the time
    batch.sync()

    # the same four lattices stepped one context at a time (two launches per lattice per step)
    sims, _ = serial_sims(torch, stream)
    for s in sims:
        s.step(args.warmup)
    serial_steps = min(args.steps, 2000)
    for s in sims:
        s.enable_kernel_timing(serial_steps)

    def serial():
        for _ in range(serial_steps):
            for s in sims:
                s.step(1)

    ms_serial = time_device(torch, stream, serial)
    k_ms, k_n = [0.0, 0.0], [0, 0]
    for s in sims:
        t, n = s.kernel_times()
        s.enable_kernel_timing(0)
        for i in range(2):
            k_ms[i] += t[i]
            k_n[i] += n[i]

    # end to end through the batch's host-to-host call: the four host densities in
    # (pinned), f = f_eq, E2E_INNER steps with the tuned plan, the four densities out
    pin_in = [torch.from_numpy(np.ascontiguousarray(r)).pin_memory() for r in rho0s]
    pin_out = [torch.empty((NY, NX), dtype=torch.float64).pin_memory() for _ in specs]

    def e2e_call():
        batch.run_host(pin_in, E2E_INNER, pin_out)

    e2e_call()
    e2e_steps = 5
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_call()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_mlups = nodes * E2E_INNER / e2e_s / 1e6 * ws
    if not all(bool(torch.isfinite(po).all()) for po in pin_out):
        raise RuntimeError("end-to-end densities are not finite")
    for s in sims:
        m, umax, bad = s.guard()
        if bad:
            raise RuntimeError("benchmark state diverged")
        s.close()

    hbm_gbs, sm_max, peak_src = load_peaks()
    ms_per_step = ms / args.steps
    mlups = nodes * args.steps / (ms / 1e3) / 1e6 * ws
    fp64_peak = 2 * 152 * sm_max * 1e6  # FP64 instructions/s: 2 per SM per clock
    ops_per_node = FP64_OPS_PER_NODE["rho_psi"] + FP64_OPS_PER_NODE["collide"]
    bytes_per_node = BYTES_PER_NODE["rho_psi"] + BYTES_PER_NODE["collide"]
    step_s = call_ms / max(1, call_steps) / 1e3
    achieved = ops_per_node * nodes / step_s
    mode = {0: "launches", 1: "graph", 2: "persistent"}[plan["mode"]]
    launches_per_step = 0 if plan["mode"] == 2 else 2
    line = {
        "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattices": len(specs), "nx": NX, "ny": NY, "nodes_per_step": nodes,
                   "engine": f"batched ({mode}, tiles {plan['tile_width'] or 'per-instance'})",
                   "parallelism": f"replicas{ws}", "l2": "state > L2 (about 180 MB per step), no flush"},
        "roofline": {"bound": "alu", "kernel": f"batched step: density/psi + collision passes ({mode})",
                     "achieved": achieved / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
                     "frac": achieved / fp64_peak, "traffic": step_traffic(),
                     "traffic_unit": "DRAM bytes per step (both passes; ncu, same kernel sources)",
                     "flop_convention": "1 per FP64 add/mul/fma instruction; 84 per node update",
                     "peak_source": f"2 FP64 instr/clk/SM x 152 SMs x {sm_max:.0f} MHz",
                     "launch_ms": step_s * 1e3},
        "roofline_hbm": {"achieved": bytes_per_node * nodes / step_s / 1e9, "peak": hbm_gbs, "unit": "GB/s",
                         "frac": bytes_per_node * nodes / step_s / 1e9 / hbm_gbs,
                         "bytes_per_node": bytes_per_node, "peak_source": peak_src},
        "autotune_ms_per_step": {"launches": plan["ms_launches"], "graph": plan["ms_graph"],
                                 "persistent": plan["ms_persistent"]},
        "serial_contexts": {"mlups": nodes * serial_steps / (ms_serial / 1e3) / 1e6, "steps": serial_steps,
                            "kernel_ms": {"rho_psi": k_ms[0] / max(1, k_n[0]),
                                          "collide": k_ms[1] / max(1, k_n[1])}},
        "e2e": {"value": e2e_mlups, "unit": "MLUPS",
                "h2d_bytes_per_step": 8 * NX * NY * len(specs) // E2E_INNER,
                "d2h_bytes_per_step": 8 * NX * NY * len(specs) // E2E_INNER,
                "steps_per_call": E2E_INNER, "h2d_bytes_per_call": 8 * NX * NY * len(specs),
                "d2h_bytes_per_call": 8 * NX * NY * len(specs),
                "call": f"pplbm_batch_run_host: H2D of the four rho0 (pinned), f=f_eq, {E2E_INNER} steps "
                        "(tuned plan), D2H of the four rho"},
        "gpu_launches": launches_per_step * args.steps + (1 if plan["mode"] == 2 else 0),
        "clocks": clk,
    }
    if rank == 0 and ws == 1 and not args.no_sweep:
        line["batch_sweep"] = sweep_comparison(torch, stream, 100)
        line["adjoint"] = adjoint_cost(torch)
        line["eos_variants_mlups"] = eos_variant_throughput(torch)
        line["fd_solver"] = fd_throughput(torch)
        line["impact_sweep"] = impact_sweep_throughput(torch)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = time_oracle_sample()
    if rank == 0:
        print(json.dumps(line), flush=True)
    batch.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
