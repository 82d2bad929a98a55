"""Benchmark: particle-steps/s of the PIC-MCC particle loop on GB300.

Workload (N=1): `scale_512` — 2.5 cm gap, 512 cells, U = 300 V, p = 20 Pa,
metastable fraction 5%, 1000 steps per RF cycle, ions subcycled x10,
4e6 e + 4e6 O- + 8e6 O2+ (quasi-neutral load), synthetic seeded inputs,
settled 100 RF cycles before the warm-up (the load drains for ~90 cycles;
afterwards the live counts drift by < 0.5 % per cycle).  One bench step = one
RF cycle (1000 time steps: every step pushes the electrons, every 10th also
the ions and runs the O-/O2+ neutralization; each step ends with the deposit
and the Poisson solve), run as one replay of the library's step graph
(o2pic_batch_* with a single discharge).  Other workloads (their own JSON
line): `stress_2048` (2048 cells, 1.2e8 particles, no subcycling, 2000
steps per cycle), `parity_128` (the small parity case, 400 steps per cycle)
and `batch_sweep_64` (the 64-discharge sweep of the batched stepper).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

Under torchrun each rank runs an independent replica (seed = rank): the
method does not shard (one discharge is one coupled field solve), so N GPUs
run N discharges and `value` sums their particle-steps over the max time.
`--impl reference` times the CPU oracle (test infrastructure) on all host
cores on bounded samples of the same workload.
"""
import argparse
import hashlib
import json
import os
import platform
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np

from paper_0705_0497_gb300 import inputs, xsec

WORKLOAD = "scale_512"
# per workload: RF cycles run before the warm-up (to reach the periodic
# state), and the oracle's bounded sample for the CPU baseline (time steps)
SETTLE = {"scale_512": 100, "stress_2048": 3, "parity_128": 10}
CPU_SAMPLE_STEPS = {"scale_512": 10, "stress_2048": 2, "parity_128": 400}
METRIC = "particle-steps/s (push+MCC+deposit) on 1 GB300, fraction of HBM roofline"
UNIT = "particle-steps/s"
BYTES_PER_PARTICLE_STEP = 40          # read + write of x, vx, vy, vz, id (algorithmic)
IMPL_BYTES_PER_PARTICLE_STEP = 20     # this implementation: read x, vx, tc (12 B), write x, vx (8 B) in place
PROFILE = os.path.join(ROOT, "profiles", "push_e_scale_512.md")


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_hash():
    h = hashlib.sha256()
    for f in ("push.cu", "common.cuh", "internal.h"):
        with open(os.path.join(ROOT, "paper_0705_0497_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_traffic():
    """DRAM bytes per launch of the electron kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    if not os.path.exists(PROFILE):
        return None, None
    vals = {}
    for line in open(PROFILE):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip()
    try:
        if vals.get("kernel_source_sha256_16") != kernel_hash():
            return None, None
        return float(vals["dram_bytes_per_particle"]), vals
    except (KeyError, ValueError):
        return None, None


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    local = env_int("LOCAL_RANK", 0)
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def allreduce(vals, op):
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return vals
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(vals, dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return t.cpu().tolist()


def aggregate(ms, ps, pe, ps_e2e, e2e_wall):
    """Whole-job figures over the replicas: the slowest rank's times, the
    summed particle-steps (each rank runs its own discharge)."""
    t_max, e2e_t = allreduce([float(ms), float(e2e_wall)], "max")
    ps_sum, pe_sum, e2e_ps_sum = allreduce([float(ps), float(pe), float(ps_e2e)], "sum")
    return {"t_max_ms": t_max, "e2e_t_max": e2e_t, "ps_sum": ps_sum, "pe_sum": pe_sum, "e2e_ps_sum": e2e_ps_sum}


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# slots per species per initial particle (the stress discharge at 500 V
# multiplies its electrons and ions)
CAPACITY_FACTOR = {"stress_2048": 3.0}


def capacity(counts, wl=WORKLOAD):
    f = CAPACITY_FACTOR.get(wl, 1.5)
    return tuple(int(n * f) + (1 << 20) for n in counts)


def cpu_model():
    """The host CPU's model (x86: model name; Arm: implementer/part)."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
        for key in ("model name", "Model", "CPU part"):
            for line in info:
                if line.startswith(key):
                    v = line.split(":", 1)[1].strip()
                    if key == "CPU part":
                        impl = [l.split(":", 1)[1].strip() for l in info if l.startswith("CPU implementer")]
                        return f"{platform.machine()} implementer {impl[0] if impl else '?'} part {v}"
                    return v
    except OSError:
        pass
    return platform.processor() or platform.machine()


def set_processes(obj, cfg, majorant):
    """The oxygen process set on a library context or an oracle, with the
    ions' majorant caps (majorant "capped") or nu_max over the whole grid
    ("grid")."""
    if majorant == "capped":
        obj.set_majorant_cap(inputs.majorant_caps(cfg))
    obj.set_processes(xsec.oxygen_set())


def run_cpu_oracle(cfg, counts, T, nsteps, threads, majorant, seed=0):
    """The oracle on `threads` host threads on the first `nsteps` time steps
    of the workload with its full initial load; returns particle-steps/s,
    particle-steps, seconds and the threads used."""
    import oracle
    st = inputs.initial_state(cfg, counts, T, seed=seed)
    o = oracle.Oracle(cfg, 32)
    used = min(threads, o.set_threads(threads))
    o.set_threads(used)
    set_processes(o, cfg, majorant)
    for s, p in enumerate(st):
        o.load(s, p["x"], p["vx"], p["vy"], p["vz"], p["id"])
    del st
    o.field()   # initial deposit + field solve (not timed)
    c0 = o.counters()["particle_steps"]
    t = time.perf_counter()
    o.step(nsteps)
    dt = time.perf_counter() - t
    ps = o.counters()["particle_steps"] - c0
    return ps / dt, ps, dt, used


def bench_reference(args, world, rank):
    """The reference arm: the CPU oracle on all host cores, one time step of
    the workload per bench step (a bounded sample of an RF cycle)."""
    if rank != 0:
        return 0
    wl = args.workload if args.workload != "batch_sweep_64" else WORKLOAD
    cfg, counts, T, _ = inputs.workload(wl)
    spc = cfg["steps_per_cycle"]
    import oracle
    st = inputs.initial_state(cfg, counts, T)
    o = oracle.Oracle(cfg, 32)
    threads = o.set_threads(os.cpu_count() or 1)
    o.set_threads(threads)
    set_processes(o, cfg, args.majorant)
    for s, p in enumerate(st):
        o.load(s, p["x"], p["vx"], p["vy"], p["vz"], p["id"])
    del st
    o.field()
    o.step(args.warmup)
    c0 = o.counters()["particle_steps"]
    t0 = time.perf_counter()
    o.step(args.steps)
    wall = time.perf_counter() - t0
    ps = o.counters()["particle_steps"] - c0
    value = ps / wall
    sample = (f"time steps {args.warmup}..{args.warmup + args.steps - 1} of {wl} with the full "
              f"{sum(counts):.3g}-particle load, {threads} host threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": wl, "step": "one time step (bounded sample of an RF cycle)",
                       "n_cells": cfg["n_cells"], "particles": list(counts), "steps_per_cycle": spc,
                       "ion_subcycle": cfg["ion_subcycle"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                             "nproc": os.cpu_count(), "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def bench_gpu(args, world, rank, local):
    import torch
    from paper_0705_0497_gb300 import api
    torch.cuda.set_device(local)
    wl = args.workload
    cfg, counts, T, cycles = inputs.workload(wl, seed=rank)
    spc = cfg["steps_per_cycle"]
    st = inputs.initial_state(cfg, counts, T, seed=rank)
    # compaction check every 20 steps: a divisor of the RF cycle and of the
    # ion subcycle, so one RF cycle is one replay of the library's step graph
    g = api.Discharge(cfg, capacity(counts, wl), device=local, compact_check=20)
    set_processes(g, cfg, args.majorant)
    g.load_state(st)
    del st
    b = api.Batch([g], steps_per_launch=spc)
    settle = SETTLE.get(wl, 0) if args.settle < 0 else args.settle
    if settle:
        b.step(settle)
    b.step(args.warmup)
    b.synchronize()
    live0 = [g.count(s) for s in range(3)]

    # ---- timed region A: K RF cycles, device-resident: K replays of the
    # one-cycle graph on the batch's stream, timed by CUDA events on it
    s0 = g.stats()
    l0 = g.launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.5)
    barrier()
    torch.cuda.synchronize()
    ms = b.timed_step(args.steps)
    b.synchronize()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    s1 = g.stats()
    launches = g.launch_count() - l0
    ps = s1["particle_steps"] - s0["particle_steps"]
    live1 = [g.count(s) for s in range(3)]
    b.close()

    # ---- timed region B: the same loop with an event pair around every
    # launch (the per-kernel split and the roofline kernel's average launch);
    # the events add a gap after every launch and undo the programmatic
    # overlap, so these per-kernel times sum to more than region A's cycle
    kb = max(1, min(args.steps, 10))
    g.set_timing(True)
    sb0 = g.stats()
    for _ in range(kb):
        g.step(spc)
    g.synchronize()
    tm = g.timing()
    sb1 = g.stats()
    g.set_timing(False)
    pe = sb1["particle_steps_0"] - sb0["particle_steps_0"]

    # ---- end to end through the C ABI with host (pinned) buffers: every step
    # loads the state from the host, runs one RF cycle and reads the state
    # and the cycle-averaged moments back
    e2e_steps = max(1, min(args.steps, 5))
    host = []
    for s in range(3):
        n = int(g.count(s) * 1.2) + 4096
        d = {k: torch.empty(n, dtype=torch.float32).pin_memory().numpy() for k in ("x", "vx", "vy", "vz")}
        d["id"] = torch.empty(n, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
        d["n"] = g.read_into(s, d)
        host.append(d)
    g.moments(reset=True)
    torch.cuda.synchronize()
    ps_e2e = 0
    h2d = d2h = 0
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for s in range(3):
            d = host[s]
            n = d["n"]
            g.load(s, d["x"][:n], d["vx"][:n], d["vy"][:n], d["vz"][:n], d["id"][:n])
            h2d += 20 * n
        c0 = g.stats()["particle_steps"]
        g.step(spc)
        for s in range(3):
            d = host[s]
            need = g.count(s)
            if need > len(d["x"]):
                for k in ("x", "vx", "vy", "vz"):
                    d[k] = torch.empty(int(need * 1.2), dtype=torch.float32).pin_memory().numpy()
                d["id"] = torch.empty(int(need * 1.2), dtype=torch.int32).pin_memory().numpy().view(np.uint32)
            d["n"] = g.read_into(s, d)
            d2h += 20 * d["n"]
        dens, _ = g.moments(reset=True)
        d2h += dens.nbytes
        ps_e2e += g.stats()["particle_steps"] - c0
    e2e_wall = time.perf_counter() - t0
    g.close()

    agg = aggregate(ms, ps, pe, ps_e2e, e2e_wall)
    if rank != 0:
        return 0
    t_max, ps_sum, e2e_ps_sum, e2e_t = agg["t_max_ms"], agg["ps_sum"], agg["e2e_ps_sum"], agg["e2e_t_max"]
    value = ps_sum / (t_max * 1e-3)
    peak, peak_kind = measured_peaks()
    ms_e, n_e = tm["push_e"]
    per_launch = pe / n_e if n_e else None
    launch_s = ms_e / n_e * 1e-3 if n_e else None
    achieved = per_launch * BYTES_PER_PARTICLE_STEP / launch_s / 1e9 if n_e else None
    traffic_pp, prof = profile_traffic()
    roofline = {"bound": "hbm",
                "kernel": "k_push<e> (gather, push, absorb, free flights, deposit, real collisions' kinematics)",
                "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs: copy bandwidth)",
                "traffic": (traffic_pp * per_launch) if (traffic_pp and n_e) else None,
                "algorithmic_bytes_per_particle_step": BYTES_PER_PARTICLE_STEP,
                "note": ("achieved = the algorithmic 40 B per particle-step (read + write of x, vx, vy, vz, id) "
                         "/ average launch time; the kernel moves 20 B per particle (x, vx, tc read, x, vx "
                         "written in place; id, vy, vz for collision candidates only, impl_frac) and the "
                         "electrons' 12 B per particle stay in L2 between ion steps, so this is an effective "
                         "bandwidth, not a DRAM measurement (traffic = ncu DRAM bytes per launch)"),
                "impl_bytes_per_particle_step": IMPL_BYTES_PER_PARTICLE_STEP,
                "impl_frac": (per_launch * IMPL_BYTES_PER_PARTICLE_STEP / launch_s / 1e9 / peak) if n_e else None,
                "electron_particles_per_launch": per_launch,
                "avg_launch_us": ms_e / n_e * 1e3 if n_e else None,
                "whole_loop_frac": value * BYTES_PER_PARTICLE_STEP / 1e9 / peak,
                "per_kernel_ms_per_cycle_instrumented": {k: v[0] / kb for k, v in tm.items() if v[1]},
                "kernel_share_of_instrumented_cycle": ms_e / sum(v[0] for v in tm.values()) if n_e else None}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        nsteps = CPU_SAMPLE_STEPS.get(wl, 10)
        allc = os.cpu_count() or 1
        v, cps, cdt, used = run_cpu_oracle(cfg, counts, T, nsteps, allc, args.majorant)
        v1, cps1, cdt1, _ = run_cpu_oracle(cfg, counts, T, nsteps, 1, args.majorant)
        cpu = {"value": v, "unit": UNIT, "cores": used, "kind": "oracle",
               "sample": f"first {nsteps} time steps of {wl} with the full {sum(counts):.3g}-particle load: "
                         f"{cps} particle-steps in {cdt:.2f} s on {used} threads",
               "nproc": os.cpu_count(), "cpu_model": cpu_model(),
               "single_thread": {"value": v1, "cores": 1, "seconds": cdt1}}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl, "step": f"one RF cycle = {spc} time steps",
                       "L_m": cfg["L"], "n_cells": cfg["n_cells"], "U_V": cfg["U"], "p_Pa": cfg["p"],
                       "C_meta": cfg["C_meta"], "ion_subcycle": cfg["ion_subcycle"],
                       "initial_particles": list(counts), "settle_cycles": settle,
                       "majorant": args.majorant,
                       "majorant_caps_eV": list(inputs.majorant_caps(cfg)) if args.majorant == "capped" else None,
                       "warn_numax_timed": s1["warn_numax"] - s0["warn_numax"],
                       "live_at_timed_start": live0, "live_at_timed_end": live1,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": ("particle arrays (all species, x, vx, vy, vz, id, tc) exceed the 129 MB L2, no flush; "
                              "the electrons' per-step working set (x, vx, tc) stays in L2 between ion steps"
                              if wl != "parity_128" else
                              "L2-resident by design (2.2e4 particles: the latency-bound parity case), no flush")},
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": e2e_ps_sum / e2e_t, "unit": UNIT, "h2d_bytes_per_step": h2d // e2e_steps,
                    "d2h_bytes_per_step": d2h // e2e_steps, "steps": e2e_steps,
                    "what": "load state from pinned host memory, one RF cycle, read state + moments back"},
            "gpu_launches": launches, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def bench_batch(args, world, rank, local):
    """The batched sweep (64 discharges): launch shapes from the library's
    autotuner (on a 100-step graph), then one CUDA graph of 200 time steps of
    every discharge per bench step; whole-job particle-steps/s."""
    import torch
    from paper_0705_0497_gb300 import api
    torch.cuda.set_device(local)
    sweep = inputs.batch_sweep(64, seed=1000 * rank)
    gs = []
    t_setup = time.perf_counter()
    for cfg, counts, T in sweep:
        cap = tuple(3 * n + (1 << 20) for n in counts)
        g = api.Discharge(cfg, cap, device=local, compact_check=20)
        set_processes(g, cfg, args.majorant)
        g.load_state(inputs.initial_state(cfg, counts, T))
        gs.append(g)
    t_setup = time.perf_counter() - t_setup
    bt = api.Batch(gs, steps_per_launch=100)
    tune = bt.autotune()
    bt.synchronize()
    bt.close()
    K = 200
    b = api.Batch(gs, steps_per_launch=K)
    b.step(args.warmup)
    b.synchronize()
    ps0 = sum(g.stats()["particle_steps"] for g in gs)
    live0 = sum(g.count(s) for g in gs for s in range(3))
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.5)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.step(args.steps)
    b.synchronize()
    wall = time.perf_counter() - t0
    barrier()
    clk = clocks.stop()
    ps = sum(g.stats()["particle_steps"] for g in gs) - ps0
    live1 = sum(g.count(s) for g in gs for s in range(3))
    t_max = allreduce([wall], "max")[0]
    ps_sum = allreduce([float(ps)], "sum")[0]
    b.close()
    if rank != 0:
        return 0
    value = ps_sum / t_max
    peak, peak_kind = measured_peaks()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch_sweep_64", "step": f"one graph replay: {K} time steps of all 64 discharges",
                       "discharges": len(sweep), "n_cells": 256, "U_V": "uniform 100-500", "p_Pa": "log-uniform 5-50",
                       "particles_per_discharge": "N e + N O- + 2N O2+, N log-uniform 1e5-2e6",
                       "total_initial_particles": sum(sum(c) for _, c, _ in sweep),
                       "live_at_timed_start": live0, "live_at_timed_end": live1,
                       "timing": "host wall clock around the graph replays, synchronized on both sides",
                       "setup_s": t_setup},
            "autotune": tune,
            "loop_roofline": {"bound": "hbm", "achieved": value * BYTES_PER_PARTICLE_STEP / 1e9, "peak": peak,
                              "unit": "GB/s", "frac": value * BYTES_PER_PARTICLE_STEP / 1e9 / peak,
                              "what": f"whole loop, 40 B per particle-step, peak {peak_kind}"},
            "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def profile_steps(n, majorant="capped", state=None):
    """The workload stepped n single steps through the public API, nothing
    timed: a short, fixed launch sequence for ncu captures (with ion
    subcycling 10, the electron push of step 6 is launch 8 of k_push).  With
    `state` (a file written by save_settled) the discharge starts from that
    saved state at its step instead of the initial load."""
    from paper_0705_0497_gb300 import api, inputs
    cfg, counts, T, _ = inputs.workload(WORKLOAD)
    if state:
        z = np.load(state)
        st = [{k: z[f"{k}{s}"] for k in ("x", "vx", "vy", "vz", "id", "tc")} for s in range(3)]
        step = int(z["step"])
    else:
        st, step = inputs.initial_state(cfg, counts, T), 0
    g = api.Discharge(cfg, capacity(counts))
    set_processes(g, cfg, majorant)
    g.load_state(st)
    if step:
        g.set_step(step)
    g.step(n)
    g.synchronize()
    print(json.dumps({"profile_steps": n, "step": g.stats()["step"], "live": [g.count(s) for s in range(3)]}))
    g.close()
    return 0


def save_settled(path, cycles, majorant="capped"):
    """The workload settled `cycles` RF cycles (the bench's own graph path)
    and its particles, free flights and step saved to `path` (.npz) for
    profile_steps."""
    from paper_0705_0497_gb300 import api, inputs
    cfg, counts, T, _ = inputs.workload(WORKLOAD)
    g = api.Discharge(cfg, capacity(counts), compact_check=20)
    set_processes(g, cfg, majorant)
    g.load_state(inputs.initial_state(cfg, counts, T))
    b = api.Batch([g], steps_per_launch=cfg["steps_per_cycle"])
    b.step(cycles)
    b.synchronize()
    b.close()
    out = {"step": np.array(g.stats()["step"])}
    for s in range(3):
        p = g.particles(s, flight=True)
        for k in ("x", "vx", "vy", "vz", "id", "tc"):
            out[f"{k}{s}"] = p[k]
    np.savez(path, **out)
    print(json.dumps({"saved": path, "step": int(out["step"]), "live": [g.count(s) for s in range(3)]}))
    g.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--majorant", default="capped", choices=["capped", "grid"],
                    help="null-collision nu_max: ions capped at 2|U| + 50 eV (default) or the whole table grid")
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD, "stress_2048", "parity_128", "batch_sweep_64"])
    ap.add_argument("--settle", type=int, default=-1,
                    help="RF cycles run before the warm-up (default: per workload, 100 for scale_512)")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="only step the workload this many single steps (a fixed launch sequence for ncu) and exit")
    ap.add_argument("--profile-state", default=None,
                    help="with --profile-steps: start from this saved state (see --save-settled)")
    ap.add_argument("--save-settled", default=None,
                    help="settle the workload --settle RF cycles (default 100), save its state here (.npz) and exit")
    args = ap.parse_args()
    if args.save_settled:
        return save_settled(args.save_settled, args.settle if args.settle >= 0 else SETTLE[WORKLOAD], args.majorant)
    if args.profile_steps > 0:
        return profile_steps(args.profile_steps, args.majorant, args.profile_state)
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return bench_reference(args, world, rank)
    if args.workload == "batch_sweep_64":
        return bench_batch(args, world, rank, local)
    return bench_gpu(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
