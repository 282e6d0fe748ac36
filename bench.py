"""Benchmark of the pseudopotential D2Q9 LBM step on GB300.

Headline workload (one bench step = one LBM time step of every lattice): the
batched sweep of 64 independent lattices, seed 210706355 -- even k a planar
interface 4 x L, odd k a static droplet L x L with R = L/4, L uniform in
64..1024, reduced temperature 0.35 + 0.6 k/63 -- Smooth C-S EOS (a_l = 0.363,
a_v = 2, alpha = 0.775), all relaxation times 1, Li forcing with sigma from the
mechanical-stability condition, periodic, tanh initial profiles of width 8:
12,946,797 node updates per step. The state (two f buffers, psi, moments:
about 2.4 GB) is far larger than the 126 MB L2, so every step streams it from
HBM; there is no explicit flush.

Timing: W untimed warm-up steps, then blocks of exactly K steps, each bracketed
by a barrier and a device synchronisation and timed with CUDA events on the
batch's stream, repeated until at least 1.5 s and 5 blocks have run (nvidia-smi
samples the clocks meanwhile); `value` is from the median block, the max over
ranks. Each pass's launches are bracketed by their own CUDA events inside the
same blocks, which gives the dominant kernel's live launch duration for the
roofline. Its peak is the FP64 issue rate measured here by pplbm_fp64_peak.

Also reported: the 2048 x 1024 droplet impact (walls, two-phase tau, T_r = 0.35,
Re = 300) as a single lattice; per-plan times of the 64-lattice batch over 1,000
steps; batched against serial per-instance launches; the adjoint's cost; EOS
variants; the FD solver; an end-to-end figure through the host-buffer C-ABI
call; and the CPU oracle on one core and on all host cores (rank 0 only).

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

# the 64-lattice sweep's EOS (every instance; T_r from the spec)
SWEEP_EOS = dict(a_l=0.363, a_v=2.0, alpha=0.775)
METRIC = "D2Q9 pseudopotential MLUPS (64-lattice batched sweep, FP64)"
WORKLOAD = ("batched sweep: 64 independent D2Q9 lattices, seed 210706355: even k planar 4 x L, odd k droplet "
            "L x L (R = L/4), L ~ U{64..1024}, T_r = 0.35 + 0.6 k/63; Smooth C-S (a_l=0.363, a_v=2, alpha=0.775), "
            "tau=1, Li forcing, periodic, tanh profiles W=8")
E2E_INNER = 100  # LBM steps per end-to-end call
MIN_TIMED_S = 1.5
MIN_BLOCKS = 5

# FP64 instructions of one node update per kernel, from the kernels' arithmetic on
# bulk nodes (unit relaxation times, Li forcing), counting what runs on the FP64 pipe:
# the density pass 15 (the C-S branch 9 with v = 1/(1 - eta), sqrt 5; its moments are
# integer sums in one fixed-point frame), the collision pass 19 (products, the
# reciprocal and the Li term; its force stencil, the sums j + h, j + 2h, j + 3h and
# the nine output populations are exact integer combinations in fixed-point frames).
# These are the fallback; the roofline uses the counts ncu measured on the workload
# (COUNTS).
FP64_PER_NODE = {"rho_psi": 15, "collide": 19}
# integer-pipe (ALU) instructions per node of the same passes (ncu; fallback figures)
ALU_PER_NODE = {"rho_psi": 223, "collide": 1020}
# ALU pipe issue rate: 64 thread instructions per SM per clock (ncu's
# sm__pipe_alu_cycles_active scale: 82.7 % active at 16.6e12 instructions/s)
ALU_PER_SM_CLK = 64
# the two-phase relaxation (rows 7, 8 relax with 1/tau(rho)), walls: pass 1 adds the
# two stress moments to its fixed-point frame, pass 2 tau(rho), its reciprocal and the
# rows 7, 8 corrections (two more terms of its output frame)
FP64_PER_NODE_SHEAR = {"rho_psi": 14.4, "collide": 32}  # ncu on the impact lattice: 14.42, 32.00
# algorithmic bytes per node of each pass as built (moments handed from pass 1 to
# pass 2): pass 1 reads 9 f and writes psi + 3 moments (5 with tau(rho)); pass 2
# reads the moments and the psi tile and writes 9 f
BYTES_PER_NODE = {"rho_psi": 72 + 32, "collide": 24 + 8 + 72}
BYTES_PER_NODE_SHEAR = {"rho_psi": 72 + 48, "collide": 40 + 8 + 72}
# the scope table's algorithmic count for the pull design: 72 + 8 (pass 1) and
# 72 + 8 + 72 (pass 2) bytes per node
BYTES_PER_NODE_SCOPE = 232
# FP64-pipe and integer-pipe (ALU) instructions of one MacCormack step per grid point
# (ncu, sm__inst_executed_pipe_fp64 / _alu x 32 per point, one kernel per capture, the
# 2048 x 1024 grid of fd_throughput): predictor 54.0 / 1,947, corrector 60.0 / 1,963,
# two EOS passes of 24.9 / 11; the update kernels' stencil differences are integer
# combinations in fixed-point frames (at 3 blocks per SM: ALU 89 % / 86 %, FP64 79 % /
# 84 % active)
FD_FP64_PER_POINT = 54.0 + 60.0 + 2 * 24.9
FD_ALU_PER_POINT = 1947 + 1963 + 2 * 11

# Per launch of each batched pass on the headline workload (all 64 lattices), from
# one ncu capture per kernel (--metrics dram__bytes_read.sum, dram__bytes_write.sum,
# the thread-level DFMA/DADD/DMUL counts and sm__inst_executed_pipe_alu.sum;
# bench.py --profile-sweep 64): DRAM bytes per launch, FP64 and ALU instructions per
# node. They hold for the device code whose digest is recorded with them; once it
# changes, traffic is null and the source counts above are used until the capture is
# repeated.
COUNTS = {"sources": "d5b0fa9fdc3eb98c",
          "rho_psi": {"dram_bytes": 1316718336, "fp64_per_node": 14.542, "alu_per_node": 222.7},
          "collide": {"dram_bytes": 1302610432, "fp64_per_node": 19.000, "alu_per_node": 1020.1},
          # the pipelined plan's mixed kernel: one launch runs the density pass of one
          # group and the collision pass of the other (half the nodes each); a step is
          # two launches
          "mixed": {"dram_bytes": 1399193600}}
KERNEL_SOURCES = ("batch_kernels.cuh", "step_device.cuh", "eos_dev.cuh", "eos.cuh", "fp64.cuh", "fixsum.cuh",
                  "internal.h")


def kernel_sources_digest():
    """sha256 (first 16 hex digits) over the device code the batched step kernels are
    compiled from, in a fixed order, each preceded by its file name."""
    import hashlib

    d = os.path.join(ROOT, "paper_2107_06355_gb300", "csrc")
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        h.update(name.encode())
        with open(os.path.join(d, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def counts_valid():
    return COUNTS["sources"] is not None and COUNTS["sources"] == kernel_sources_digest()


def pass_traffic(name):
    return COUNTS[name]["dram_bytes"] if counts_valid() else None


def pass_fp64(name):
    """(FP64 instructions per node, where the figure comes from)."""
    if counts_valid():
        return COUNTS[name]["fp64_per_node"], "ncu on this workload (thread-level DFMA + DADD + DMUL per node)"
    return FP64_PER_NODE[name], "the kernel's arithmetic on bulk nodes"


def pass_alu(name):
    return COUNTS[name]["alu_per_node"] if counts_valid() else ALU_PER_NODE[name]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, tag="main"):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}_{tag}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "samples": 0, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
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
                "power_w_median": float(np.median(power)) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def build_lib():
    from paper_2107_06355_gb300 import build
    build.build()


def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


# ---- workloads -------------------------------------------------------------------

def sweep_specs(n=64):
    import lbm_inputs as I

    specs = I.batch_specs(n)
    for s in specs:
        s.update(SWEEP_EOS)
    return specs


def initial_density(I, s, rho_v, rho_l):
    if s["kind"] == "planar":
        return I.planar(s["nx"], s["ny"], rho_v, rho_l, W=8.0)
    return I.droplet(s["nx"], s["ny"], s["R"], rho_v, rho_l, W=8.0)


def make_batch(P, I, specs, stream, kappa=0.0):
    """A Batch over `specs` (dicts with nx, ny, Tr, kind, R, a_l, a_v, alpha) with
    tanh initial fields; kappa: the surface-tension control of every instance."""
    eos = [P.EOSParams(P.EOS_SMOOTH, s["Tr"], s["a_l"], s["a_v"], s["alpha"]) for s in specs]
    relax = [P.Relax(kappa=kappa) for _ in specs]
    b = P.Batch([(s["nx"], s["ny"], P.BC_PERIODIC) for s in specs], eos, relax, stream=stream)
    inits = []
    for k, s in enumerate(specs):
        d = b.derived(k)
        rho = initial_density(I, s, d["rho_v"], d["rho_l"])
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


def timed_blocks(torch, stream, fn, barrier, min_seconds=MIN_TIMED_S, min_blocks=MIN_BLOCKS, max_blocks=2000,
                 after=None):
    """Runs fn() in blocks, each bracketed by barrier() and timed with CUDA events on
    `stream`, until min_seconds of device time and min_blocks blocks; block times in ms.
    after(), if given, runs after each block's closing barrier (outside the timing)."""
    times = []
    while len(times) < max_blocks and (len(times) < min_blocks or sum(times) < 1e3 * min_seconds):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        fn()
        e1.record(stream)
        barrier()
        times.append(e0.elapsed_time(e1))
        if after is not None:
            after()
    return times


# ---- FP64 issue-rate peak ---------------------------------------------------------

def measure_fp64_peak(torch, local, seconds=0.6, repeats=3):
    """pplbm_fp64_peak: 8 independent FMA chains per thread, 8 blocks of 256 per SM,
    sized to run `seconds`; best of `repeats`, with the clocks sampled meanwhile."""
    import ctypes as C
    from paper_2107_06355_gb300 import _lib as L

    lib = L.lib()
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = (C.c_double * 3)()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    L.check(lib.pplbm_fp64_peak(8, 8, 0, 4000, C.c_void_p(sink.data_ptr()), out, stream))  # warm-up, calibration
    iters = max(1000, int(4000 * seconds / max(out[1] * 1e-3, 1e-6)))
    clocks = ClockSampler(local, "fp64")
    clocks.start()
    rates, ms = [], []
    for _ in range(repeats):
        L.check(lib.pplbm_fp64_peak(8, 8, 0, iters, C.c_void_p(sink.data_ptr()), out, stream))
        rates.append(out[0])
        ms.append(out[1])
    clk = clocks.stop()
    best = max(rates)
    return {"value": best / 1e12, "unit": "TFLOP/s (1 per FP64 FMA instruction per thread)",
            "median": float(np.median(rates)) / 1e12,
            "launch_ms": ms, "blocks": int(out[2]), "iters": iters, "clocks": clk,
            "how": "pplbm_fp64_peak: 8 independent FP64 FMA chains per thread, 256 threads x 8 blocks per SM, "
                   "CUDA events, best of 3"}


def fp64_probe_sweep(torch, local):
    """pplbm_fp64_peak over chain counts, occupancies and operations (each launch
    ~0.1-0.2 s at the running clock, sampled by nvidia-smi): whether any issue pattern
    beats the rate the bench uses as its peak. One JSON line."""
    import ctypes as C
    from paper_2107_06355_gb300 import _lib as L

    lib = L.lib()
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = (C.c_double * 3)()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    variants = [(8, 8, 0), (4, 8, 0), (2, 8, 0), (1, 8, 0), (8, 1, 0), (8, 2, 0), (8, 4, 0), (8, 16, 0),
                (4, 32, 0), (8, 8, 1), (8, 8, 2), (8, 8, 3), (8, 8, 4), (8, 4, 3), (8, 4, 4), (8, 8, 5),
                (8, 8, 6), (4, 4, 5)]
    L.check(lib.pplbm_fp64_peak(8, 8, 0, 4000, C.c_void_p(sink.data_ptr()), out, stream))
    clocks = ClockSampler(local, "sweep")
    clocks.start()
    rows = []
    for bpsm, ch, op in variants:
        iters = max(1000, int(160000 * 8 / (bpsm * ch)))
        L.check(lib.pplbm_fp64_peak(bpsm, ch, op, iters, C.c_void_p(sink.data_ptr()), out, stream))
        rows.append({"blocks_per_sm": bpsm, "chains": ch,
                     "op": ("fma", "add", "mul", "integer-pipe add", "fma + integer-pipe add",
                                "int64 -> f64 conversion", "f64 -> int64 conversion")[op],
                     "rate": out[0] / 1e12, "ms": out[1]})
    clk = clocks.stop()
    mhz = clk["sm_mhz"] or 2070.0
    for r in rows:
        r["per_sm_clk"] = r["rate"] * 1e12 / (152 * mhz * 1e6)
    print(json.dumps({"fp64_probe_sweep": rows, "clocks": clk, "unit": "T FP64 instr/s"}), flush=True)


# ---- the 2048 x 1024 droplet impact (single lattice) ---------------------------------

def impact_2048(torch, stream, barrier, steps=1000):
    """Droplet impact on a liquid film: 2048 x 1024, periodic x, walls in y, Smooth C-S
    at T_r = 0.35 (a_l = 0.363, a_v = 2, alpha = 0.838), two-phase tau(rho) with
    tau_l = 0.6 and v_r = 1, R = 100, film 102, V_d = 0.05 (Re = V_d 2R / nu_l = 300),
    tanh width 6. One context (two launches per step, per-kernel CUDA events)."""
    import lbm_inputs as I
    import paper_2107_06355_gb300 as P

    nx, ny = 2048, 1024
    eos = P.EOSParams(P.EOS_SMOOTH, 0.35, 0.363, 2.0, 0.838)
    sim = P.Simulation(nx, ny, P.BC_WALLS_Y, eos, P.Relax(kind=P.RELAX_TWO_PHASE, tau_l=0.6, visc_ratio=1.0),
                       stream=stream)
    d = sim.derived()
    sim.init_equilibrium(*I.impact(nx, ny, 100, 102, d["rho_v"], d["rho_l"], 0.05, W=6.0))
    m0 = sim.guard()[0]
    sim.step(20)
    sim.sync()
    sim.enable_kernel_timing(3 * steps)
    times = timed_blocks(torch, stream, lambda: sim.step(steps), barrier, min_seconds=1.0, min_blocks=3,
                         max_blocks=3)
    (k_ms, k_n) = sim.kernel_times()
    sim.enable_kernel_timing(0)
    m1, umax, bad, _ = sim.guard()
    sim.close()
    if bad or not abs(m1 - m0) < 1e-10 * m0:
        raise RuntimeError("impact lattice diverged or lost mass")
    med = float(np.median(times))
    nodes = nx * ny
    _, sm_max, _ = load_peaks()
    per = {k: k_ms[i] / max(1, k_n[i]) for i, k in enumerate(("rho_psi", "collide"))}
    out = {"config": "2048x1024 droplet impact on a film, walls in y, Smooth C-S T_r=0.35 (a_l=0.363, a_v=2, "
                     "alpha=0.838), tau(rho) tau_l=0.6 v_r=1, R=100, film 102, V_d=0.05 (Re=300)",
           "steps_per_block": steps, "blocks_ms": times, "ms_per_step": med / steps,
           "mlups": nodes * steps / (med / 1e3) / 1e6, "kernel_ms": per, "max_u": umax,
           "mass_drift": abs(m1 - m0) / m0}
    hbm_gbs, _, peak_src = load_peaks()
    step_s = med / steps / 1e3
    out["roofline_hbm"] = {
        "scope_bytes_per_node": BYTES_PER_NODE_SCOPE,
        "achieved_scope": BYTES_PER_NODE_SCOPE * nodes / step_s / 1e9,
        "frac_scope": BYTES_PER_NODE_SCOPE * nodes / step_s / 1e9 / hbm_gbs,
        "built_bytes_per_node": sum(BYTES_PER_NODE_SHEAR.values()),
        "frac_built": sum(BYTES_PER_NODE_SHEAR.values()) * nodes / step_s / 1e9 / hbm_gbs,
        "peak": hbm_gbs, "unit": "GB/s", "peak_source": peak_src}
    out["fp64_per_node"] = FP64_PER_NODE_SHEAR
    return out


# ---- batch plans and batched vs serial ----------------------------------------------

def plan_times(torch, stream, batch, P, steps=1000):
    """Per-plan ms per step of the batch over `steps` steps each (state restored)."""
    out = {}
    saved = [batch.get_f(k).clone() for k in range(batch.n)]
    for name, mode in (("launches", P.PLAN_LAUNCHES), ("graph", P.PLAN_GRAPH), ("persistent", P.PLAN_PERSISTENT),
                       ("pipelined", P.PLAN_PIPELINED)):
        batch.set_plan(mode, 0)
        batch.step(4)
        ms = time_device(torch, stream, lambda: batch.step(steps))
        out[name] = ms / steps
    for k in range(batch.n):
        batch.set_f(k, saved[k])
    return out


def serial_comparison(torch, stream, specs, batch_ms_per_step, steps=200):
    """The same lattices as one context each: per-instance CUDA graphs of two steps
    replayed one instance after another (the baseline), and plain launches."""
    import ctypes as C
    import lbm_inputs as I
    import paper_2107_06355_gb300 as P
    from paper_2107_06355_gb300 import _lib as L

    nodes = sum(s["nx"] * s["ny"] for s in specs)
    sims = []
    for s in specs:
        sim = P.Simulation(s["nx"], s["ny"], P.BC_PERIODIC,
                           P.EOSParams(P.EOS_SMOOTH, s["Tr"], s["a_l"], s["a_v"], s["alpha"]), P.Relax(),
                           stream=stream)
        d = sim.derived()
        sim.init_equilibrium(initial_density(I, s, d["rho_v"], d["rho_l"]))
        sims.append(sim)

    def serial():
        for _ in range(steps):
            for sim in sims:
                sim.step(1)

    for sim in sims:
        sim.step(2)
    ms_s = time_device(torch, stream, serial)
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
    serial_ms = ms_g / steps
    return {"instances": len(specs), "nodes": nodes, "steps": steps,
            "serial_baseline": "per-instance CUDA graphs of 2 steps, replayed serially",
            "batched_ms_per_step": batch_ms_per_step, "serial_ms_per_step": serial_ms,
            "batched_instance_steps_per_s": len(specs) / (batch_ms_per_step / 1e3),
            "serial_instance_steps_per_s": len(specs) / (serial_ms / 1e3),
            "batched_mlups": nodes / (batch_ms_per_step / 1e3) / 1e6,
            "serial_mlups": nodes / (serial_ms / 1e3) / 1e6,
            "speedup": serial_ms / batch_ms_per_step,
            "serial_plain_launches_mlups": nodes * steps / (ms_s / 1e3) / 1e6}


# ---- figures of the batched engine, the adjoint, the EOS variants, FD and the sweeps ----

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
    p = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    lib = L.lib()
    alpha_slots = (1 << 9) - 1   # the shaped-branch constants and the Li-term scale: all alpha moves
    out = {}
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
    """Four 512 x 512 periodic static droplets (R = 32, 48, 64, 96; tau = 1) with each
    EOS the kernels support (T_r = 0.6; the two Guo-forced EOS at 0.7), and the Smooth
    C-S with the surface-tension control, batched graph plan: MLUPS per variant."""
    import lbm_inputs as I
    import paper_2107_06355_gb300 as P

    variants = {
        "cs_a0.387_li": (P.EOSParams(P.EOS_CS, 0.6, 0.387, 0.387, 0.5), P.Relax()),
        "smooth_alpha0.834_li": (P.EOSParams(P.EOS_SMOOTH, 0.6, 0.387, 2.0, 0.834), P.Relax()),
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
        b = P.Batch([(512, 512, P.BC_PERIODIC)] * 4, [eos] * 4, [relax] * 4)
        d = b.derived(0)
        for k, R in enumerate((32, 48, 64, 96)):
            b.init_equilibrium(k, I.droplet(512, 512, R, d["rho_v"], d["rho_l"], W=8.0))
        b.autotune(trial_steps=20)
        b.step(20)
        ms = time_device(torch, torch.cuda.current_stream(), lambda: b.step(steps))
        try:
            b.sync()
            out[name] = 4 * 512 * 512 * steps / (ms / 1e3) / 1e6
        except P.PPLBMError as e:
            out[name] = f"diverged ({e})"
        b.close()
    return out


def impact_sweep_throughput(torch, fp64_peak, steps=2000):
    """A slice of the stability study (Sec. IV.D) on the batched engine: droplet
    impact at Re = 300 on (600, 250) lattices with walls, C-S a = 0.363, Li forcing,
    two-phase tau(rho), T_r in {0.45, ..., 0.75} x v_r in {2, ..., 10}: 35 instances,
    5.25 M nodes, autotuned plan with divergence isolation."""
    b, n_inst = impact_sweep_batch()
    plan = {0: "launches", 1: "graph", 2: "persistent", 3: "pipelined"}[b.plan()["mode"]]
    b.step(20)
    ms = time_device(torch, torch.cuda.current_stream(), lambda: b.step(steps))
    g = b.guard()
    stable = int(((np.asarray(b.instance_status()) == 0) & (g[:, 2] == 0)).sum())
    b.close()
    nodes = 600 * 250 * n_inst
    mlups = nodes * steps / (ms / 1e3) / 1e6 if stable == n_inst else None
    out = {"instances": n_inst, "stable": stable, "nodes": nodes, "steps": steps, "mlups": mlups, "plan": plan}
    if mlups is not None:
        per = sum(FP64_PER_NODE_SHEAR.values())
        achieved = per * mlups * 1e6
        out["roofline"] = {"bound": "alu", "achieved": achieved / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                           "frac": achieved / 1e12 / fp64_peak, "fp64_per_node": per}
    return out


def impact_sweep_batch():
    """The impact-sweep batch, initialised, on the autotuned plan: (Batch, instances)."""
    import lbm_inputs as I
    import paper_2107_06355_gb300 as P

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
        b.init_equilibrium(i, *I.impact(600, 250, 50, 25, d["rho_v"], d["rho_l"], 0.1, W=Ws[i]))
    b.autotune(trial_steps=20)
    return b, len(lats)


def fd_throughput(torch, fp64_peak, sm_mhz, steps=200):
    """The finite-difference solver (App. A) on a 2048 x 1024 periodic droplet grid
    (dx = 1, Smooth C-S at T_r = 0.6): grid-point updates per second. dt = 0.4: with
    the paper's 0.8 dx^2 the static droplet diverges in this scheme (CPU oracle too)."""
    import lbm_inputs as I
    import paper_2107_06355_gb300 as P

    nx, ny = 2048, 1024
    eos = P.EOSParams(P.EOS_SMOOTH, 0.6, 0.387, 2.0, 0.834)
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
    pts = nx * ny * steps / (ms / 1e3)
    achieved = FD_FP64_PER_POINT * pts
    alu = FD_ALU_PER_POINT * pts
    alu_peak = ALU_PER_SM_CLK * 152 * sm_mhz * 1e6
    return {"grid": f"{nx}x{ny}, dx=1, dt=0.4", "mlups": pts / 1e6,
            "ms_per_step": ms / steps, "finite": ok, "launches_per_step": 4,
            "roofline": {"bound": "alu", "pipe": "integer (the update kernels' stencil sums)",
                         "achieved": alu / 1e12, "peak": alu_peak / 1e12, "unit": "T integer instr/s",
                         "frac": alu / alu_peak, "alu_per_point_step": FD_ALU_PER_POINT},
            "fp64_pipe": {"achieved": achieved / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                          "frac": achieved / 1e12 / fp64_peak, "fp64_per_point_step": FD_FP64_PER_POINT}}


# ---- the oracle on the host cores ---------------------------------------------------

def _oracle_worker(conn, specs, threads_env):
    """Spawned process: builds the oracle lattices of `specs` (untimed), then on each
    'step' message advances every one of them by one step and replies with the seconds
    it took."""
    os.environ.update(threads_env)
    sys.path.insert(0, ROOT)
    import lbm_inputs as I
    from oracle import eos as E
    from oracle import lbm as L
    import warnings

    warnings.simplefilter("ignore")
    lats, fs = [], []
    for s in specs:
        e = E.make_eos(E.MODE_SMOOTH, s["Tr"], s["a_l"], s["a_v"], s["alpha"])
        lat = L.Lattice(s["nx"], s["ny"], L.BC_PERIODIC_X | L.BC_PERIODIC_Y, e, L.Relax(sigma=e.sigma()))
        lats.append(lat)
        fs.append(lat.init_equilibrium(initial_density(I, s, e.rho_v, e.rho_l)))
    conn.send("ready")
    while True:
        msg = conn.recv()
        if msg == "stop":
            break
        t0 = time.perf_counter()
        for k, lat in enumerate(lats):
            fs[k] = lat.step(fs[k], 1)
        conn.send(time.perf_counter() - t0)
    conn.close()


class OraclePool:
    """The oracle (plain numpy, as it stands) advancing the instances of `specs` in
    `workers` spawned processes, one numpy thread each, instances assigned largest
    first to the least-loaded process. step() advances every instance by one LBM step
    and returns the wall time of the slowest process."""

    def __init__(self, specs, workers):
        import multiprocessing as mp

        from paper_2107_06355_gb300.replicas import shard_instances

        ctx = mp.get_context("spawn")
        sizes = [s["nx"] * s["ny"] for s in specs]
        shards = [sh for sh in shard_instances(sizes, max(1, min(workers, len(specs)))) if sh]
        env = {k: "1" for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        self.nodes = sum(sizes)
        self.conns, self.procs = [], []
        for sh in shards:
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(b, [specs[i] for i in sh], env), daemon=True)
            p.start()
            self.conns.append(a)
            self.procs.append(p)
        for c in self.conns:
            assert c.recv() == "ready"

    @property
    def workers(self):
        return len(self.procs)

    def step(self):
        for c in self.conns:
            c.send("step")
        return max(c.recv() for c in self.conns)

    def close(self):
        for c in self.conns:
            c.send("stop")
        for p in self.procs:
            p.join(timeout=30)


def cpu_baseline(specs, max_seconds=20.0):
    """The oracle on the host cores: (1) one process on a bounded sample of the
    workload (the instances every 8th, from index 1), (2) every instance across all
    host cores, a few steps. MLUPS each."""
    cores = host_cores()
    sample = [specs[k] for k in range(1, len(specs), 8)]
    one = OraclePool(sample, 1)
    t, n = 0.0, 0
    while t < 0.5 * max_seconds and n < 50:
        t += one.step()
        n += 1
    one.close()
    single = one.nodes * n / t / 1e6
    pool = OraclePool(specs, cores)
    t2, n2 = 0.0, 0
    while t2 < 0.25 * max_seconds and n2 < 20:
        t2 += pool.step()
        n2 += 1
    pool.close()
    all_cores = pool.nodes * n2 / t2 / 1e6
    return {"value": all_cores, "unit": "MLUPS", "cores": pool.workers, "kind": "oracle",
            "sample": f"all {len(specs)} instances of the workload ({pool.nodes} nodes), {n2} steps, "
                      f"{pool.workers} processes x 1 thread, {t2:.1f} s",
            "single_core": {"value": single, "unit": "MLUPS", "cores": 1,
                            "sample": f"{len(sample)} instances (every 8th; {one.nodes} nodes), {n} steps, "
                                      f"{t:.1f} s"},
            "host_cores": cores}


def run_reference(args):
    """The oracle as the reference arm: each bench step is one LBM step of the whole
    64-lattice workload, spread over the host cores."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    specs = sweep_specs()
    pool = OraclePool(specs, host_cores())
    for _ in range(args.warmup):
        pool.step()
    t = sum(pool.step() for _ in range(args.steps))
    pool.close()
    val = pool.nodes * args.steps / t / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "nodes_per_step": pool.nodes},
            "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": pool.workers, "kind": "oracle",
                             "sample": f"{args.steps} steps of all 64 instances, {pool.workers} processes"},
            "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- small cases for ncu captures -----------------------------------------------------

def profile_sweep(n=16, plan="launches"):
    """The first `n` lattices of the 64-lattice sweep (the bench's EOS and tiles),
    3 steps: under the launches plan 3 launches of each batched pass, under the
    pipelined plan 7 launches of the mixed kernel (prologue, 5 mixed, epilogue)."""
    import torch
    import lbm_inputs as I
    import paper_2107_06355_gb300 as P

    build_lib()
    specs = sweep_specs()[:n]
    b, _, _, _ = make_batch(P, I, specs, torch.cuda.current_stream())
    b.set_plan(P.PLAN_PIPELINED if plan == "pipelined" else P.PLAN_LAUNCHES, 0)
    b.step(3)
    b.sync()
    torch.cuda.synchronize()
    print(f"profile sweep done: {len(specs)} lattices, {sum(s['nx'] * s['ny'] for s in specs)} nodes")


def profile_impact_single():
    """The 2048 x 1024 impact lattice of impact_2048, 3 steps."""
    import torch
    import lbm_inputs as I
    import paper_2107_06355_gb300 as P

    build_lib()
    sim = P.Simulation(2048, 1024, P.BC_WALLS_Y, P.EOSParams(P.EOS_SMOOTH, 0.35, 0.363, 2.0, 0.838),
                       P.Relax(kind=P.RELAX_TWO_PHASE, tau_l=0.6, visc_ratio=1.0))
    d = sim.derived()
    sim.init_equilibrium(*I.impact(2048, 1024, 100, 102, d["rho_v"], d["rho_l"], 0.05, W=6.0))
    sim.step(3)
    sim.sync()
    torch.cuda.synchronize()
    sim.close()
    print("profile impact done")


def profile_fd():
    """The finite-difference solver on the 2048 x 1024 droplet grid, 3 steps."""
    import torch
    import lbm_inputs as I
    import paper_2107_06355_gb300 as P

    build_lib()
    eos = P.EOSParams(P.EOS_SMOOTH, 0.6, 0.387, 2.0, 0.834)
    d = P.eos_setup(eos)
    fd = P.FDSolver(2048, 1024, eos, dx=1.0)
    rho = I.droplet(2048, 1024, 100, d["rho_v"], d["rho_l"], W=8.0)
    fd.set_state(rho, np.zeros_like(rho), np.zeros_like(rho))
    fd.step(3, 0.4)
    torch.cuda.synchronize()
    print("profile fd done")


def profile_adjoint():
    """Checkpointed forward and reverse pass on a 1024 x 1024 droplet (T_r = 0.5,
    tau = 1), 12 steps with interval 4, gradient slots of alpha."""
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
    L.check(L.lib().pplbm_adjoint_set_slots(sim.ctx, (1 << 9) - 1), sim.ctx)
    L.check(L.lib().pplbm_forward_checkpointed(sim.ctx, steps, interval, p(ckpt)), sim.ctx)
    L.check(L.lib().pplbm_backward_checkpointed(sim.ctx, steps, interval, p(ckpt), p(seg), p(lam), p(lam0), p(grad),
                                                p(ws), nb), sim.ctx)
    torch.cuda.synchronize()
    sim.close()
    print("profile adjoint done")


# ---- main ---------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="headline line only (no extra keys)")
    ap.add_argument("--plan", default="auto", choices=["auto", "launches", "graph", "persistent", "pipelined"],
                    help="batched-engine plan for the timed run (auto: autotuned)")
    ap.add_argument("--profile-sweep", type=int, default=None, metavar="N",
                    help="3 steps of the first N lattices of the sweep (a small case for ncu) and exit")
    ap.add_argument("--profile-impact", action="store_true", help="3 steps of the 2048x1024 impact (for ncu)")
    ap.add_argument("--profile-adjoint", action="store_true", help="checkpointed adjoint on 1024 x 1024 (for ncu)")
    ap.add_argument("--profile-fd", action="store_true", help="3 steps of the FD solver on 2048 x 1024 (for ncu)")
    ap.add_argument("--fp64-probe-sweep", action="store_true",
                    help="the FP64 issue-rate probe over chains, occupancy and operation, then exit")
    args = ap.parse_args()
    if args.fp64_probe_sweep:
        import torch
        build_lib()
        return fp64_probe_sweep(torch, dist_env()[2])
    if args.profile_sweep is not None:
        return profile_sweep(args.profile_sweep, "pipelined" if args.plan == "pipelined" else "launches")
    if args.profile_impact:
        return profile_impact_single()
    if args.profile_fd:
        return profile_fd()
    if args.profile_adjoint:
        return profile_adjoint()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import lbm_inputs as I
    import paper_2107_06355_gb300 as P
    from paper_2107_06355_gb300.replicas import max_over_ranks

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

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    fp64 = measure_fp64_peak(torch, local)
    specs = sweep_specs()
    nodes = sum(s["nx"] * s["ny"] for s in specs)
    batch, _, _, rho0s = make_batch(P, I, specs, stream)
    if args.plan == "auto":
        plan = batch.autotune(trial_steps=100)
    else:
        batch.set_plan({"launches": P.PLAN_LAUNCHES, "graph": P.PLAN_GRAPH,
                        "persistent": P.PLAN_PERSISTENT, "pipelined": P.PLAN_PIPELINED}[args.plan], 0)
        plan = batch.plan()
    mode = {0: "launches", 1: "graph", 2: "persistent", 3: "pipelined"}[plan["mode"]]
    # per-pass kernel durations exist where each launch runs one pass
    per_pass = plan["mode"] in (P.PLAN_LAUNCHES, P.PLAN_GRAPH)
    batch.step(args.warmup)
    torch.cuda.synchronize()
    batch.enable_timing(1)
    acc = {"pass_ms": [0.0, 0.0], "pass_n": [0, 0], "call_ms": 0.0, "call_steps": 0}
    state = {"timed": False}

    def collect():
        """After each block: the per-call (and per-pass) CUDA-event sums; then switch the
        per-pass events on or off for the next block (outside the block's timing)."""
        ms_, n_ = batch.times()
        acc["call_ms"] += ms_
        acc["call_steps"] += n_
        if state["timed"]:
            (a0, a1), (n0, n1) = batch.pass_times()
            acc["pass_ms"][0] += a0
            acc["pass_ms"][1] += a1
            acc["pass_n"][0] += n0
            acc["pass_n"][1] += n1
        if per_pass:
            state["timed"] = not state["timed"]
            batch.enable_pass_timing(args.steps if state["timed"] else 0)
        kinds.append(state["timed"])

    # Blocks alternate: plain (the plan as tuned: `value`) and instrumented (event
    # records around each pass: the kernels' launch durations for the roofline).
    kinds = [False]
    clocks = ClockSampler(local)
    clocks.start()
    blocks = timed_blocks(torch, stream, lambda: batch.step(args.steps), barrier, min_blocks=2 * MIN_BLOCKS,
                          after=collect)
    clk = clocks.stop()
    batch.enable_timing(0)
    if per_pass:
        batch.enable_pass_timing(0)
    # the probe again, right after the timed blocks (the clock the step ran at): the
    # issue rate scales with the SM clock, and the first probe may have run while the
    # clock was still rising; the higher of the two is the peak
    fp64_after = measure_fp64_peak(torch, local)
    fp64_first = fp64
    fp64 = max(fp64_first, fp64_after, key=lambda r: r["value"])
    fp64["probes"] = [{"value": r["value"], "sm_mhz": r["clocks"].get("sm_mhz"), "when": w}
                      for r, w in ((fp64_first, "before the autotuner"), (fp64_after, "after the timed blocks"))]
    kinds = kinds[:len(blocks)]
    plain = [t for t, k in zip(blocks, kinds) if not k]
    instrumented = [t for t, k in zip(blocks, kinds) if k]
    call_ms, call_steps = acc["call_ms"], acc["call_steps"]
    pass_ms, pass_n = acc["pass_ms"], acc["pass_n"]
    med_ms = max_over_ranks(float(np.median(plain)), device="cuda")  # each rank runs its own replica
    batch.sync()
    g = batch.guard()
    if (g[:, 2] > 0).any():
        raise RuntimeError("benchmark state diverged")

    hbm_gbs, sm_max, peak_src = load_peaks()
    ms_per_step = med_ms / args.steps
    step_s = ms_per_step / 1e3
    mlups = nodes * args.steps / (med_ms / 1e3) / 1e6 * ws
    fp64_peak = fp64["value"]  # T FP64 instructions/s, measured above
    fp64_node = {k: pass_fp64(k)[0] for k in ("rho_psi", "collide")}
    fp64_src = pass_fp64("collide")[1]
    if per_pass:
        kern = {"rho_psi": pass_ms[0] / max(1, pass_n[0]), "collide": pass_ms[1] / max(1, pass_n[1])}
        dom = max(kern, key=kern.get)
        dom_s = kern[dom] / 1e3
        dom_name = {"rho_psi": "k_batch_rho_psi", "collide": "k_batch_collide"}[dom]
        dom_flops = fp64_node[dom] * nodes
        dom_bytes = BYTES_PER_NODE[dom] * nodes
        share = kern[dom] / (kern["rho_psi"] + kern["collide"])
    else:
        # the plan's launches run both passes: the step's time against both passes'
        # instruction counts
        kern = {mode: call_ms / max(1, call_steps)}
        dom, share = mode, 1.0
        dom_name = {"persistent": "k_batch_persistent", "pipelined": "k_batch_mixed"}[mode]
        dom_s = call_ms / max(1, call_steps) / 1e3
        dom_flops = sum(fp64_node.values()) * nodes
        dom_bytes = sum(BYTES_PER_NODE.values()) * nodes
    achieved = dom_flops / dom_s / 1e12
    # kernel launches per timed block: two per step; one cooperative launch per call
    # (persistent); 2 steps + 1 (pipelined: prologue, two mixed launches per step less
    # one, epilogue)
    launches_per_block = {"launches": 2 * args.steps, "graph": 2 * args.steps, "persistent": 1,
                          "pipelined": 2 * args.steps + 1}[mode]
    # the dominant kernel against both arithmetic pipes: FP64 instructions against the
    # measured FP64 issue rate, integer instructions against the ALU pipe's 64 per SM per
    # clock at the sampled clock; `roofline` is the pipe closer to its limit (the bound)
    mhz = clk.get("sm_mhz") or sm_max
    alu_peak = ALU_PER_SM_CLK * 152 * mhz * 1e6 / 1e12
    fp64_pipe = {"pipe": "fp64", "kernel": dom_name, "achieved": achieved, "peak": fp64_peak,
                 "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                 "flop_convention": "1 per FP64 add/mul/fma instruction (per thread); "
                                    f"{fp64_node.get(dom, sum(fp64_node.values()))} per node ({fp64_src})",
                 "peak_source": "measured: pplbm_fp64_peak in this run (fp64_peak_measured)"}
    alu_node = pass_alu(dom) if per_pass else sum(pass_alu(k) for k in ("rho_psi", "collide"))
    int_pipe = {"pipe": "integer", "kernel": dom_name, "alu_per_node": alu_node,
                "achieved": alu_node * nodes / dom_s / 1e12,
                "peak": alu_peak, "unit": "T integer instr/s",
                "frac": alu_node * nodes / dom_s / 1e12 / alu_peak,
                "peak_source": f"derived: 64 integer lanes per SM x 152 SMs x {mhz:.0f} MHz (sampled)",
                "note": "the pass's sums run on the integer pipe (fixed-point frames and software IEEE adds)"}
    if int_pipe["frac"] > fp64_pipe["frac"]:
        roof, other = dict(int_pipe), fp64_pipe
    else:
        roof, other = dict(fp64_pipe), int_pipe
    if per_pass:
        traffic, traffic_unit = pass_traffic(dom), "DRAM bytes per launch (ncu capture, same kernel sources)"
    elif mode == "pipelined" and counts_valid():
        traffic = 2 * COUNTS["mixed"]["dram_bytes"]
        traffic_unit = "DRAM bytes per step: two mixed launches (ncu capture of one, same kernel sources)"
    else:
        traffic, traffic_unit = None, "DRAM bytes per step"
    roof = {"bound": "alu", **roof, "traffic": traffic, "traffic_unit": traffic_unit,
            "launch_ms": dom_s * 1e3, "share_of_step": share}
    line = {
        "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattices": len(specs), "nodes_per_step": nodes,
                   "engine": f"batched ({mode}, tiles {plan['tile_width'] or 'per-instance'})",
                   "parallelism": f"replicas{ws}",
                   "timing": (f"{len(blocks)} blocks of {args.steps} steps ({sum(blocks) / 1e3:.2f} s), alternating "
                              f"plain blocks (value: median of {len(plain)}) and blocks with per-pass CUDA events "
                              f"(kernel durations: {len(instrumented)})") if per_pass else
                             (f"{len(blocks)} blocks of {args.steps} steps ({sum(blocks) / 1e3:.2f} s), value: median "
                              f"of the {len(plain)} blocks; the {mode} plan's launches run both passes, so the kernel "
                              "duration is the call's CUDA-event time per step"),
                   "l2": "state about 2.4 GB >> 126 MB L2, no flush"},
        "blocks_ms": plain,
        "blocks_ms_instrumented": instrumented,
        "roofline": roof,
        "kernel_ms": kern,
        "other_pipe": other,
        "fp64_peak_measured": fp64,
        "roofline_hbm": {
            "dominant_kernel": {"achieved": dom_bytes / dom_s / 1e9, "frac": dom_bytes / dom_s / 1e9 / hbm_gbs,
                                "bytes_per_node": BYTES_PER_NODE.get(dom, sum(BYTES_PER_NODE.values()))},
            "step_scope": {"bytes_per_node": BYTES_PER_NODE_SCOPE,
                           "achieved": BYTES_PER_NODE_SCOPE * nodes / step_s / 1e9,
                           "frac": BYTES_PER_NODE_SCOPE * nodes / step_s / 1e9 / hbm_gbs},
            "step_built": {"bytes_per_node": sum(BYTES_PER_NODE.values()),
                           "achieved": sum(BYTES_PER_NODE.values()) * nodes / step_s / 1e9,
                           "frac": sum(BYTES_PER_NODE.values()) * nodes / step_s / 1e9 / hbm_gbs},
            "peak": hbm_gbs, "unit": "GB/s", "peak_source": peak_src},
        "fp64_roofline_step": {"fp64_per_node": sum(fp64_node.values()),
                               "achieved": sum(fp64_node.values()) * nodes / step_s / 1e12,
                               "frac": sum(fp64_node.values()) * nodes / step_s / 1e12 / fp64_peak},
        "autotune_ms_per_step": {"launches": plan["ms_launches"], "graph": plan["ms_graph"],
                                 "persistent": plan["ms_persistent"], "pipelined": plan["ms_pipelined"]},
        "gpu_launches": launches_per_block * len(blocks),
        "clocks": clk,
    }

    # end to end through the batch's host-to-host call: the 64 host densities in
    # (pinned), f = f_eq, E2E_INNER steps with the tuned plan, the 64 densities out
    pin_in = [torch.from_numpy(np.ascontiguousarray(r)).pin_memory() for r in rho0s]
    pin_out = [torch.empty(r.shape, dtype=torch.float64).pin_memory() for r in rho0s]
    batch.run_host(pin_in, E2E_INNER, pin_out)
    e2e_calls = 3
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_calls):
        batch.run_host(pin_in, E2E_INNER, pin_out)
    barrier()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_calls)
    if not all(bool(torch.isfinite(po).all()) for po in pin_out):
        raise RuntimeError("end-to-end densities are not finite")
    line["e2e"] = {"value": nodes * E2E_INNER / e2e_s / 1e6 * ws, "unit": "MLUPS",
                   "h2d_bytes_per_step": 8 * nodes // E2E_INNER, "d2h_bytes_per_step": 8 * nodes // E2E_INNER,
                   "steps_per_call": E2E_INNER, "h2d_bytes_per_call": 8 * nodes, "d2h_bytes_per_call": 8 * nodes,
                   "call": f"pplbm_batch_run_host: H2D of the 64 rho0 (pinned), f=f_eq, {E2E_INNER} steps "
                           "(tuned plan), D2H of the 64 rho"}

    if rank == 0 and ws == 1 and not args.no_extras:
        line["plans_ms_per_step"] = plan_times(torch, stream, batch, P, steps=1000)
        line["batched_vs_serial"] = serial_comparison(torch, stream, specs, ms_per_step)
        batch.close()
        torch.cuda.empty_cache()
        line["impact_2048x1024"] = impact_2048(torch, stream, barrier)
        line["adjoint"] = adjoint_cost(torch)
        line["eos_variants_mlups"] = eos_variant_throughput(torch)
        line["fd_solver"] = fd_throughput(torch, fp64_peak, clk.get("sm_mhz") or sm_max)
        line["impact_sweep"] = impact_sweep_throughput(torch, fp64_peak)
    else:
        batch.close()
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline(specs)
        except Exception as e:  # the line still reports the GPU figures
            line["cpu_baseline"] = {"value": None, "unit": "MLUPS", "kind": "oracle", "error": repr(e)[:300]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
