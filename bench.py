#!/usr/bin/env python
"""Benchmark of the fast-electron hybrid-PIC step on one GB300.

Workload: 128^3 cells of 1 um gold, 1e7 macro-electrons injected over
100 fs at 1e21 W/cm^2 (T_hot = 13.7 MeV), dt = 0.5 fs, reflux on all faces;
the 200-step injection runs before timing, then K steps are timed with the
full population resident in HBM.  One step = push/collide/emit/deposit,
E and B update, heating, (injection), and a cell sort folded into every third step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64]
    python bench.py --impl reference ...   # the FP64 CPU oracle, timed alone

With N > 1 (torchrun), every rank runs an independent replica of the
workload (the step has no exchange to shard): value = all ranks'
particle-steps over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fast-electron particle-steps/s at 1e7 e-, FP32 vs FP64, CE(>1MeV) within 1%"
UNIT = "particle-steps/s"
WORKLOAD = ("128^3 cells x 1 um Au (Z=79, n_i=5.9e28 m^-3, T0=1 eV), 1e7 e- injected over "
            "100 fs at 1e21 W/cm^2 in a 5 um disc, 30 deg cone, dt=0.5 fs, reflux on all faces, "
            "timed after the injection window")
# algorithmic bytes per particle-step of the push kernel: the SoA state is
# read once (x,y,z,ux,uy,uz,tau + u32 id) and written once (7 reals)
ALG_BYTES = {"fp32": 7 * 4 + 4 + 7 * 4, "fp64": 7 * 8 + 4 + 7 * 8}
# a step that also sorts (every SORT_INTERVAL steps) reads each slot's sort key
# and rank and writes its id to the sorted slot: 12 B more per particle-step;
# in the single-target step, the step before it (when it injects nothing)
# writes each surviving electron's key and rank: 8 B more
SORT_STEP_EXTRA_BYTES = 4 + 4 + 4
KEY_STEP_EXTRA_BYTES = 4 + 4
# DRAM bytes (read + write) per particle-step of k_push measured by ncu on
# this workload (dram__bytes_read.sum + dram__bytes_write.sum of one launch
# over its particle-steps; launch 204 a plain step, 205 a keying step, 206 a
# sorting step): a plain step streams the state once (absorbed slots are not
# rewritten), a keying step adds the keys and ranks it writes, a sorting step
# reads them and scatters its stores (partial sectors); None where not captured
NCU_DRAM_BYTES_PER_PSTEP = {"fp32": {"plain": 55.1, "key": 62.8, "sort": 76.9}, "fp64": None}
# the same for k_batch_push, captured on the first 16 targets of the scan
# (the full scan holds too much device memory for a multi-pass capture): the traffic is the
# electron state streamed once, so it scales with the particle-steps
NCU_BATCH_DRAM_BYTES_PER_PSTEP = {"fp32": {"plain": 60.9, "sort": 93.7}, "fp64": None}
# the launch shape those counters were taken at (blocks per SM of 256 threads);
# another shape runs the same code but reports no traffic of its own
NCU_BATCH_CAPTURE_BLOCKS = 4
# FP64 FLOP per particle-step of the FP64 k_push (2 per DFMA, 1 per DADD and
# DMUL; ncu thread-level counts on config 1 in FP64, launches at steps 110
# and 111) and the FP64 rate the GB300 is stated to have (TFLOP/s)
NCU_FP64_FLOP_PER_PSTEP = 1210.0
FP64_STATED_TFLOPS = 1.25
# the accuracy window: the injection (200 steps) and 1 ps beyond
ACCURACY_STEPS = 2200
# cell sort every 3 steps, folded into the step and keyed by the cell reached halfway
# through the interval; measured over 600 steps after the injection: intervals 3 / 4 / 5 /
# 6 / 8 give steps of 0.796 / 0.794 / 0.792 / 0.795 / 0.801 ms with k_push at 0.639 /
# 0.646 / 0.650 / 0.657 / 0.668 ms (the step is flat; 3 keeps the push kernel fastest)
SORT_INTERVAL = 3


def n_sort_steps(step0: int, steps: int, interval: int = SORT_INTERVAL) -> int:
    """Steps of [step0, step0 + steps) that also sort."""
    if interval <= 0:
        return 0
    return sum(1 for s in range(step0, step0 + steps) if (s + 1) % interval == 0)


def n_key_steps(step0: int, steps: int, interval: int = SORT_INTERVAL) -> int:
    """Steps of [step0, step0 + steps) whose push keys the next sort (single
    target, past the injection window)."""
    if interval < 2:
        return 0
    return sum(1 for s in range(step0, step0 + steps) if (s + 2) % interval == 0)


def push_bytes(precision: str, k_ps: float, k_launches: int, step0: int, steps: int,
               interval: int = SORT_INTERVAL, keyed: bool = True) -> float:
    """Algorithmic bytes of the push launches of steps [step0, step0 + steps)
    (keyed: the pushes of the steps before a sort compute its keys)."""
    n_sort = n_sort_steps(step0, steps, interval)
    n_key = n_key_steps(step0, steps, interval) if keyed else 0
    per_launch = k_ps / max(k_launches, 1)
    return (ALG_BYTES[precision] * k_ps + SORT_STEP_EXTRA_BYTES * n_sort * per_launch
            + KEY_STEP_EXTRA_BYTES * n_key * per_launch)


def push_traffic(table: dict, precision: str, k_ps: float, k_launches: int, step0: int,
                 steps: int, interval: int = SORT_INTERVAL, keyed: bool = True):
    """ncu DRAM bytes per push launch of those steps, from the per-particle-step
    figures of a plain, a keying (keyed) and a sorting step."""
    tb = table[precision]
    if not tb or k_launches <= 0:
        return None
    n_sort = n_sort_steps(step0, steps, interval)
    n_key = n_key_steps(step0, steps, interval) if keyed else 0
    if (n_sort and tb.get("sort") is None) or (n_key and tb.get("key") is None):
        return None
    per_ps = (tb["plain"] * (k_launches - n_sort - n_key) + tb["sort"] * n_sort
              + (tb["key"] * n_key if n_key else 0.0)) / k_launches
    return per_ps * k_ps / k_launches


def peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "of measured"}
    return {"hbm_gbs": 6800.0, "source": "of fallback"}


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("HPIC_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce(world, vals, op="max"):
    """Max or sum of per-rank values (replica timing and work counts)."""
    if world == 1:
        return vals
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(vals, dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return t.tolist()


def replica_rate(world, ms, particle_steps):
    """Whole-job rate of N independent replicas: all ranks' particle-steps
    over the slowest rank's time."""
    ms_max, = allreduce(world, [ms], "max")
    ps_sum, = allreduce(world, [particle_steps], "sum")
    return ps_sum / (ms_max / 1e3), ms_max, ps_sum


def host_cpu() -> dict:
    """The host's CPU model and core count, read at run time."""
    model = None
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for ln in r.stdout.splitlines():
            k, _, v = ln.partition(":")
            if k.strip() in ("Model name", "Model") and v.strip() and not v.strip().isdigit():
                model = v.strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None and os.path.exists("/proc/cpuinfo"):
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu model")):
                model = ln.split(":", 1)[1].strip()
                break
    return {"cpu_model": model, "host_cores": os.cpu_count()}


def oracle_rate(steps_timed: int, warmup: int, budget_s: float, threads: bool = False) -> dict:
    """The FP64 CPU oracle, as it stands, on a bounded sample of the workload:
    the same 128^3 target and laser, stepped from t = 0 through the start of
    the injection window (5e4 new electrons per step), every step including
    the full 128^3 field and heating update.  threads: the oracle's OpenMP
    build on all host cores (its electrons, field and heating loops in
    parallel); else the serial oracle on one core."""
    from oracle import oracle as O
    from paper_2107_01723_gb300 import workloads as W
    cfg = W.config2()
    o = O.OracleSim(cfg["target"], cfg["laser"], cfg["run"], threads=threads)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)) if threads else 1
    o.step(max(warmup, 1))
    ps0 = o.tallies()["particle_steps"]
    t0 = time.perf_counter()
    done = 0
    while done < steps_timed:
        o.step(1)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    ps = o.tallies()["particle_steps"] - ps0
    return {"value": ps / dt, "unit": UNIT, "cores": cores, "kind": "oracle", **host_cpu(),
            "sample": (f"oracle steps {max(warmup, 1)}..{max(warmup, 1) + done - 1} of the headline "
                       f"workload (injection phase, {int(ps / max(done, 1))} live e- per step on "
                       f"average, full 128^3 field/heat update each step), FP64, "
                       f"{'OpenMP on ' + str(cores) + ' threads' if threads else 'serial'}, {dt:.1f} s"),
            "steps_timed": done, "seconds": dt}


def oracle_threads_ok() -> bool:
    """Whether the oracle's OpenMP build is available on this host."""
    try:
        from oracle import oracle as O
        O.build(threads=True)
        return True
    except Exception:  # noqa: BLE001 - no OpenMP runtime: the serial oracle
        return False


def run_reference(args, world, rank):
    if rank != 0:
        return
    r = oracle_rate(args.steps, args.warmup, budget_s=150.0, threads=oracle_threads_ok())
    line = {"impl": "reference", "metric": METRIC, "value": r["value"], "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * r["seconds"] / max(r["steps_timed"], 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "precision": "fp64 oracle"},
            "cpu_baseline": {k: r[k] for k in ("value", "unit", "cores", "kind", "sample", "cpu_model",
                                               "host_cores")},
            "e2e": {"value": r["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def pinned_state(p: dict, fill: bool = True) -> dict:
    """Page-locked host arrays shaped like the electron state p (float64
    x .. tau, uint32 id), filled with p unless fill is False."""
    import numpy as np
    import torch
    n = len(p["id"])
    out = {}
    for k in ("x", "y", "z", "ux", "uy", "uz", "tau"):
        out[k] = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
        if fill:
            out[k][:] = p[k]
    out["id"] = torch.empty(n, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    if fill:
        out["id"][:] = p["id"]
    return out


def run_gpu(args, world, rank, local):
    import numpy as np
    import torch

    from paper_2107_01723_gb300 import build as B
    from paper_2107_01723_gb300 import hpic
    from paper_2107_01723_gb300 import workloads as W

    torch.cuda.set_device(local)
    if rank == 0 or not os.path.exists(B.LIB):
        B.build()
    barrier(world)
    cfg = W.config2()
    run = dict(cfg["run"], target_index=rank)
    prec = hpic.HPIC_FP32_MIXED if args.precision == "fp32" else hpic.HPIC_FP64
    stream = torch.cuda.Stream()
    sim = hpic.Sim(cfg["target"], cfg["laser"], run, precision=prec, device=local,
                   stream=stream.cuda_stream, sort_interval=SORT_INTERVAL)
    # setup: the injection window (200 steps) builds the 1e7-electron state
    sim.step(200)
    sim.step(args.warmup)
    live = sim.n
    # the state at the start of the timed steps, so that the end-to-end leg
    # below runs the same steps (the beam spreads and later steps cost more)
    snap_p = sim.particles()
    snap_g = {k: sim.grid(k) for k in ("T", "eta", "Ti", "Ex", "Ey", "Ez", "Bx", "By", "Bz")}
    snap_clock = sim.clock()
    t0 = sim.tallies()
    launches0 = hpic.hpic_launch_count(sim.h)
    hpic.hpic_profile(sim.h, True)
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler()
    clocks.start()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    sim.step(args.steps)
    end.record(stream)
    end.synchronize()
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = start.elapsed_time(end)
    t1 = sim.tallies()
    k_ms, k_launches, k_ps = hpic.hpic_kernel_time(sim.h)
    hpic.hpic_profile(sim.h, False)
    launches = hpic.hpic_launch_count(sim.h) - launches0
    ps = t1["particle_steps"] - t0["particle_steps"]
    value, ms_max, ps_sum = replica_rate(world, ms, ps)

    # end to end through the C-ABI with host buffers, over the same K steps:
    # the grids and the clock of the timed start are restored untimed, then
    # the electron state is uploaded from host arrays, K steps run, and the
    # tallies and the state are read back
    for k, v in snap_g.items():
        sim.set_grid(k, v)
    sim.set_clock(*snap_clock)
    # the C-ABI moves FP64 arrays (and u32 ids) across; conversion is on the
    # device.  Both directions use page-locked host buffers allocated (and
    # filled with the start state) before the timed region; no electron is
    # injected after the injection window, so the read-back fits in as many.
    host, back_buf = pinned_state(snap_p), pinned_state(snap_p, fill=False)
    nbytes_state = len(host["id"]) * (7 * 8 + 4)
    torch.cuda.synchronize()
    barrier(world)
    w0 = time.perf_counter()
    e_t0 = sim.tallies()
    sim.set_particles(host)
    sim.step(args.steps)
    e_t1 = sim.tallies()
    back = sim.particles(out=back_buf)
    wall = time.perf_counter() - w0
    e_ps = e_t1["particle_steps"] - e_t0["particle_steps"]
    wall_max, = allreduce(world, [wall], "max")
    e_ps_sum, = allreduce(world, [e_ps], "sum")
    tally_bytes = 19 * 8
    e2e = {"value": e_ps_sum / wall_max, "unit": UNIT,
           "h2d_bytes_per_step": nbytes_state / args.steps,
           "d2h_bytes_per_step": (len(back["id"]) * (7 * 8 + 4) + 2 * tally_bytes) / args.steps,
           "what": ("hpic_load_particles from page-locked host arrays + hpic_step(K) + "
                    "hpic_read_tallies + hpic_read_particles into page-locked host arrays, "
                    "wall clock, over the timed steps again (grids and clock of their start "
                    "restored untimed)")}

    # FP64 reference path on the same workload (shorter run), for "FP32 vs FP64",
    # and the accuracy gate: both precisions from t = 0 through the injection
    # window and 1 ps beyond, CE(>1 MeV) and energy closure of each
    fp64, accuracy = None, None
    if args.precision == "fp32" and not args.no_fp64 and world == 1:
        s64 = hpic.Sim(cfg["target"], cfg["laser"], run, precision=hpic.HPIC_FP64, device=local,
                       stream=stream.cuda_stream, sort_interval=SORT_INTERVAL)
        s64.step(200 + args.warmup)
        k64 = max(args.steps // 4, 10)
        a0 = s64.tallies()["particle_steps"]
        hpic.hpic_profile(s64.h, True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s64.step(k64)
        e1.record(stream)
        e1.synchronize()
        m64 = e0.elapsed_time(e1)
        a1 = s64.tallies()["particle_steps"]
        km, kl, kp = hpic.hpic_kernel_time(s64.h)
        hpic.hpic_profile(s64.h, False)
        fp64 = {"value": (a1 - a0) / (m64 / 1e3), "unit": UNIT, "steps": k64,
                "ms_per_step": m64 / k64,
                "push_kernel_gbs": (push_bytes("fp64", kp, kl, 200 + args.warmup, k64) / (km / 1e3) / 1e9
                                    if km > 0 else None)}
        if km > 0:
            tf = NCU_FP64_FLOP_PER_PSTEP * kp / (km / 1e3) / 1e12
            fp64["alu"] = {"bound": "fp64", "achieved_tflops": tf, "peak_tflops": FP64_STATED_TFLOPS,
                           "frac": tf / FP64_STATED_TFLOPS, "peak_source": "stated (GB300 FP64 rate)",
                           "flop_per_particle_step": NCU_FP64_FLOP_PER_PSTEP,
                           "flop_source": "ncu DFMA/DADD/DMUL counts on config 1 in FP64"}
        if not args.no_accuracy:
            done64 = 200 + args.warmup + k64
            acc_steps = max(ACCURACY_STEPS, done64)
            s64.step(acc_steps - done64)
            s32 = hpic.Sim(cfg["target"], cfg["laser"], run, precision=hpic.HPIC_FP32_MIXED,
                           device=local, stream=stream.cuda_stream, sort_interval=SORT_INTERVAL)
            s32.step(acc_steps)
            acc = {}
            for name, s_ in (("fp32", s32), ("fp64", s64)):
                t = s_.tallies()
                rhs = (t["E_live"] + t["W_field"] + t["E_drag"] + t["E_xray"] + t["E_escaped"]
                       + t["E_reflux"])
                acc[name] = {"ce_above_1MeV": t["E_xray_above"] / (t["E_injected"] / cfg["laser"]["eta_l2e"]),
                             "closure": (t["E_injected"] - rhs) / t["E_injected"],
                             "particle_steps": t["particle_steps"]}
            s32.close()
            ce_rel = acc["fp32"]["ce_above_1MeV"] / acc["fp64"]["ce_above_1MeV"] - 1.0
            accuracy = {"window": f"steps 0..{acc_steps - 1} (injection + {(acc_steps - 200) * 0.5e-3:g} ps), same seed",
                        "ce_fp32": acc["fp32"]["ce_above_1MeV"], "ce_fp64": acc["fp64"]["ce_above_1MeV"],
                        "ce_rel_diff": ce_rel, "closure_fp32": acc["fp32"]["closure"],
                        "closure_fp64": acc["fp64"]["closure"],
                        "particle_steps_per_run": acc["fp64"]["particle_steps"],
                        "bar": {"ce_rel": 0.01, "closure": 1e-3},
                        "pass": bool(abs(ce_rel) < 0.01 and abs(acc["fp32"]["closure"]) < 1e-3
                                     and abs(acc["fp64"]["closure"]) < 1e-3)}
        s64.close()

    if rank != 0:
        sim.close()
        return
    pk = peaks()
    k_avg_ms = k_ms / max(k_launches, 1)
    k_bytes = push_bytes(args.precision, k_ps, k_launches, int(snap_clock[0]), args.steps)
    achieved = k_bytes / max(k_launches, 1) / (k_avg_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"],
                "traffic": push_traffic(NCU_DRAM_BYTES_PER_PSTEP, args.precision, k_ps, k_launches,
                                        int(snap_clock[0]), args.steps),
                "traffic_unit": "bytes per launch (ncu dram read+write, scaled by particle-steps)",
                "kernel": "k_push (push/collide/emit/deposit)",
                "kernel_ms_avg": k_avg_ms, "kernel_share_of_step": k_ms / ms if ms > 0 else None,
                "bytes_per_particle_step": k_bytes / k_ps if k_ps > 0 else None,
                "peak_source": pk["source"]}
    cpu = None
    if not args.no_cpu_baseline:
        keys = ("value", "unit", "cores", "kind", "sample", "cpu_model", "host_cores")
        r1 = oracle_rate(200, 2, budget_s=20.0)
        if oracle_threads_ok():
            r = oracle_rate(400, 2, budget_s=20.0, threads=True)
            cpu = dict({k: r[k] for k in keys}, single_core={k: r1[k] for k in keys})
        else:
            cpu = {k: r1[k] for k in keys}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD,
                       "precision": ("fp32-mixed: particles and fields f32; T, eta, tallies f64"
                                     if args.precision == "fp32" else "fp64 throughout"),
                       "sort_interval": SORT_INTERVAL, "live_electrons_at_start": live,
                       "l2": "inputs larger than L2 (particle state >= 320 MB per step)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk, "fp64": fp64, "accuracy": accuracy}
    if world == 1 and not args.no_sub:
        # the other single-GPU workloads, short windows: the batched scan
        # (64 targets, 200 timed steps after the injection window and the
        # autotuner) and the emission microbenchmark (2^27 electrons)
        sim.close()
        sim = None
        bl = batch_result(64, 200, 200)
        line["batched_scan"] = {k: bl[k] for k in ("metric", "value", "unit", "steps", "warmup",
                                                   "ms_per_step", "dtype", "config", "roofline",
                                                   "gpu_launches", "clocks", "ce_above_1MeV")}
        line["emission"] = emission_result(2 ** 27, {"fp32": 50, "fp64": 5}, 3)
    print(json.dumps(line), flush=True)
    if sim is not None:
        sim.close()


def run_full(args):
    """The whole 10 ps (20000-step) headline run in FP32-mixed and in FP64:
    X-ray conversion efficiency above 1 MeV, CE = E_xray(k >= 1 MeV) /
    E_laser with E_laser = E_injected / eta_l2e, and the energy-budget
    closure, for both precisions."""
    import torch

    from paper_2107_01723_gb300 import build as B
    from paper_2107_01723_gb300 import hpic
    from paper_2107_01723_gb300 import workloads as W
    B.build()
    cfg = W.config2()
    steps = cfg["steps"] if args.full_steps <= 0 else args.full_steps
    out = {"what": "full headline run, CE(>1 MeV) FP32-mixed vs FP64", "steps": steps}
    stream = torch.cuda.Stream()
    legs = [(n, p) for n, p in (("fp32", hpic.HPIC_FP32_MIXED), ("fp64", hpic.HPIC_FP64))
            if args.full_precision in ("both", n)]
    for name, prec in legs:
        sim = hpic.Sim(cfg["target"], cfg["laser"], cfg["run"], precision=prec,
                       stream=stream.cuda_stream, sort_interval=SORT_INTERVAL)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        e1.synchronize()
        t = sim.tallies()
        E_laser = t["E_injected"] / cfg["laser"]["eta_l2e"]
        rhs = t["E_live"] + t["W_field"] + t["E_drag"] + t["E_xray"] + t["E_escaped"] + t["E_reflux"]
        out[name] = {"CE_above_1MeV": t["E_xray_above"] / E_laser,
                     "eta_e2g": t["E_xray_above"] / t["E_injected"],
                     "closure": (t["E_injected"] - rhs) / t["E_injected"],
                     "particle_steps": t["particle_steps"], "seconds": e0.elapsed_time(e1) / 1e3,
                     "particle_steps_per_s": t["particle_steps"] / (e0.elapsed_time(e1) / 1e3),
                     "live_at_end": sim.n, "tallies": t}
        sim.close()
    if len(legs) == 2:
        out["CE_rel_diff"] = out["fp32"]["CE_above_1MeV"] / out["fp64"]["CE_above_1MeV"] - 1.0
    print(json.dumps(out), flush=True)


def run_thick(args):
    """The thick-target long run (not the headline line): 500 x 256 x 256 cells
    of 1 um gold, 1e8 electrons injected over 100 fs at 1e22 W/cm^2, reflux on
    all faces, FP32-mixed with FP64 tallies, stepped `--full-steps` steps
    (default 40,000 = 20 ps) in chunks.  Reports per chunk the conversion
    efficiency above 1 MeV (Sec. III.A), the energy closure and the live
    count, and at the end the angular distribution of the X-ray energy,
    dE/dOmega per polar bin about the laser axis (+x), and the
    particle-steps/s of the whole run."""
    import math

    import numpy as np
    import torch

    from paper_2107_01723_gb300 import build as B
    from paper_2107_01723_gb300 import hpic
    from paper_2107_01723_gb300 import workloads as W
    B.build()
    cfg = W.config3()
    steps = args.full_steps if args.full_steps > 0 else 40_000
    chunk = 2_000
    stream = torch.cuda.Stream()
    sim = hpic.Sim(cfg["target"], cfg["laser"], cfg["run"], precision=hpic.HPIC_FP32_MIXED,
                   stream=stream.cuda_stream, sort_interval=SORT_INTERVAL)
    eta = cfg["laser"]["eta_l2e"]
    series = []
    ms_total = 0.0
    done = 0
    while done < steps:
        k = min(chunk, steps - done)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(k)
        e1.record(stream)
        e1.synchronize()
        ms_total += e0.elapsed_time(e1)
        done += k
        t = sim.tallies()
        rhs = t["E_live"] + t["W_field"] + t["E_drag"] + t["E_xray"] + t["E_escaped"] + t["E_reflux"]
        series.append({"step": done, "t_ps": done * cfg["run"]["dt"] * 1e12,
                       "ce_above_1MeV": t["E_xray_above"] / (t["E_injected"] / eta),
                       "closure": (t["E_injected"] - rhs) / t["E_injected"], "live": sim.n,
                       "particle_steps": t["particle_steps"]})
    t = sim.tallies()
    hE, _ = sim.hist()
    nth = cfg["run"]["n_theta"]
    edges = np.linspace(0.0, math.pi, nth + 1)
    dOmega = 2 * math.pi * (np.cos(edges[:-1]) - np.cos(edges[1:]))
    E_th = hE.sum(axis=0)  # photon energy per polar bin (J), all energies
    dEdO = E_th / dOmega
    sim.close()
    out = {"what": "thick-target long run, FP32-mixed, FP64 tallies", "workload": (
               "500 x 256 x 256 cells x 1 um Au, 1e8 e- over 100 fs at 1e22 W/cm^2, reflux on all "
               "faces, dt = 0.5 fs"),
           "steps": steps, "t_ps": steps * cfg["run"]["dt"] * 1e12,
           "particle_steps_per_s": t["particle_steps"] / (ms_total / 1e3), "seconds": ms_total / 1e3,
           "ce_above_1MeV": t["E_xray_above"] / (t["E_injected"] / eta),
           "eta_e2g": t["E_xray_above"] / t["E_injected"],
           "closure": series[-1]["closure"], "series": series,
           "dE_dOmega_J_per_sr": {"theta_deg_bin_centres": list(np.degrees(0.5 * (edges[:-1] + edges[1:]))),
                                  "values": list(dEdO)},
           "dE_dOmega_peak_deg": float(np.degrees(0.5 * (edges[:-1] + edges[1:]))[int(np.argmax(dEdO))]),
           "forward_fraction_0_30deg": float(E_th[edges[1:] <= math.radians(30.0) + 1e-12].sum() / E_th.sum())}
    print(json.dumps(out), flush=True)


def run_small(args):
    """Config 1 (32^3 cells of 1 um gold, 1e5 electrons over 100 fs at
    1e20 W/cm^2) stepped `--full-steps` steps (default 200) in the chosen
    precision: particle-steps/s and the live count (not the headline line;
    a small case for counter captures)."""
    import torch

    from paper_2107_01723_gb300 import build as B
    from paper_2107_01723_gb300 import hpic
    from paper_2107_01723_gb300 import workloads as W
    B.build()
    cfg = W.config1()
    steps = args.full_steps if args.full_steps > 0 else cfg["steps"]
    prec = hpic.HPIC_FP32_MIXED if args.precision == "fp32" else hpic.HPIC_FP64
    stream = torch.cuda.Stream()
    sim = hpic.Sim(cfg["target"], cfg["laser"], cfg["run"], precision=prec,
                   stream=stream.cuda_stream, sort_interval=SORT_INTERVAL)
    live = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        sim.step(1)
        live.append(sim.n)
    e1.record(stream)
    e1.synchronize()
    t = sim.tallies()
    sim.close()
    print(json.dumps({"what": "config 1, " + args.precision, "steps": steps,
                      "particle_steps_per_s": t["particle_steps"] / (e0.elapsed_time(e1) / 1e3),
                      "live_after_step": live}), flush=True)


def emission_result(n: int, steps: dict, warmup: int) -> dict:
    """Emission microbenchmark: n electrons in an unbounded uniform gold medium,
    drag + scatter + bremsstrahlung only, in FP32 and FP64 (steps[precision]
    timed steps after `warmup`); k_push's particle-steps/s and HBM fraction."""
    import torch

    from paper_2107_01723_gb300 import hpic
    from paper_2107_01723_gb300 import workloads as W
    cfg = W.config5(n_electrons=n)
    pk = peaks()
    out = {"what": "emission microbenchmark: unbounded gold, drag+scatter+bremsstrahlung",
           "electrons": cfg["n_electrons"], "steps": steps, "warmup": warmup}
    stream = torch.cuda.Stream()
    for name, prec in (("fp32", hpic.HPIC_FP32_MIXED), ("fp64", hpic.HPIC_FP64)):
        sim = hpic.Sim(cfg["target"], cfg["laser"], cfg["run"], precision=prec,
                       stream=stream.cuda_stream)
        sim.seed(cfg["n_electrons"], cfg["mean_energy"])
        sim.step(warmup)
        hpic.hpic_profile(sim.h, True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(steps[name])
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        km, kl, kp = hpic.hpic_kernel_time(sim.h)
        hpic.hpic_profile(sim.h, False)
        gbs = ALG_BYTES[name] * kp / (km / 1e3) / 1e9
        out[name] = {"particle_steps_per_s": kp / (ms / 1e3), "ms_per_step": ms / steps[name],
                     "k_push_ms": km / kl, "achieved_GBs": gbs, "frac_of_hbm": gbs / pk["hbm_gbs"],
                     "peak_source": pk["source"], "emissions": sim.tallies()["n_emitted"]}
        sim.close()
    return out


def run_emission(args):
    """The emission microbenchmark alone (not the headline line)."""
    from paper_2107_01723_gb300 import build as B
    B.build()
    print(json.dumps(emission_result(args.emission_n, {"fp32": args.steps, "fp64": args.steps},
                                     args.warmup)), flush=True)


def batch_result(n_targets: int, warm: int, steps: int, precision: str = "fp32",
                 tuning: str = "", world: int = 1, rank: int = 0, local: int = 0):
    """Batched scan: n_targets targets of uneven thickness, element and
    intensity (6e7 electrons for 64), one launch per kernel kind per step,
    steps replayed from CUDA graphs.  Under torchrun the targets are sharded
    over the ranks (greedy LPT on electron counts, no exchange until an
    end-of-run tally sum).  The first `warm` steps (at least the 200-step
    injection window) run first, the autotuner then picks blocks per SM and
    the sort interval from a snapshot, and `steps` steps are timed.  Returns
    rank 0's line (None on other ranks)."""
    import torch

    from paper_2107_01723_gb300 import hpic
    from paper_2107_01723_gb300 import shard
    from paper_2107_01723_gb300 import workloads as W
    cfg = W.config4(n_targets=n_targets, total_macro=int(6e7 * n_targets / 64))
    # whole targets to ranks by electron count (greedy LPT); global indices
    # keep each target's random numbers
    mine = shard.lpt_assign([l["n_macro"] for l in cfg["lasers"]], world)[rank]
    targets = [cfg["targets"][t] for t in mine]
    lasers = [cfg["lasers"][t] for t in mine]
    prec = hpic.HPIC_FP32_MIXED if precision == "fp32" else hpic.HPIC_FP64
    stream = torch.cuda.Stream()
    b = hpic.Batch(targets, lasers, cfg["run"], precision=prec, device=local,
                   stream=stream.cuda_stream, sort_interval=SORT_INTERVAL, target_index=mine)
    b.step(warm)
    if tuning:
        bps, si = (int(v) for v in tuning.split(","))
        b.set_tuning(bps, si)
        tune = dict(b.tuning(), chosen="fixed by --batch-tuning")
    else:
        tune = dict(b.autotune(trial_steps=40), chosen="autotuned")
    b.step(1)  # captures and uploads the graphs of the chosen tuning
    torch.cuda.synchronize()
    live = sum(b.target(t).n for t in range(len(b)))
    launches0 = hpic.hpic_batch_launch_count(b.b)
    ps0 = sum(b.target(t).tallies()["particle_steps"] for t in range(len(b)))
    barrier(world)
    clocks = ClockSampler()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = hpic.hpic_batch_launch_count(b.b) - launches0
    ps1 = sum(b.target(t).tallies()["particle_steps"] for t in range(len(b)))
    value, ms_max, _ = replica_rate(world, ms, ps1 - ps0)
    # the particle kernel alone, from direct launches bracketed by events
    step0 = int(b.target(0).clock()[0])
    hpic.hpic_batch_profile(b.b, True)
    b.step(40)
    km, kl, kp = hpic.hpic_batch_kernel_time(b.b)
    hpic.hpic_batch_profile(b.b, False)
    pk = peaks()
    si = int(tune["sort_interval"])
    kbytes = push_bytes(precision, kp, kl, step0, 40, si, keyed=False)
    achieved = kbytes / kl / (km / kl / 1e3) / 1e9
    ce, tot = [], {"E_xray_above": 0.0, "E_injected": 0.0}
    for t in range(len(b)):
        T = b.target(t).tallies()
        ce.append(T["E_xray_above"] / (T["E_injected"] / lasers[t]["eta_l2e"]))
        for k in tot:
            tot[k] += T[k]
    tot = shard.reduce_tallies(world, tot)  # the scan's only exchange, at the end
    b.close()
    if rank != 0:
        return None
    return {"metric": f"particle-steps/s, batched scan of {n_targets} targets", "value": value,
            "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": warm, "ms_per_step": ms_max / steps,
            "higher_is_better": True, "scaling": "strong" if world > 1 else "weak",
            "dtype": "f32" if precision == "fp32" else "f64",
            "data": "synthetic",
            "config": {"parallelism": f"{world} ranks, whole targets by LPT" if world > 1 else "single GPU",
                       "workload": (f"{n_targets} targets: thickness U{{5..200}} x 64 x 64 cells of 1 um, "
                                    "Z in {13, 29, 79}, log10 I ~ U[20, 22] W/cm^2, "
                                    f"{sum(l['n_macro'] for l in cfg['lasers']):.3g} e- in all "
                                    "(1e5..4e6 per target)"),
                       "live_electrons_at_start": live, "tuning": tune,
                       "graphs": "plain and sorting steps replayed from captured CUDA graphs"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / pk["hbm_gbs"],
                         "traffic": (push_traffic(NCU_BATCH_DRAM_BYTES_PER_PSTEP, precision, kp, kl,
                                                  step0, 40, si, keyed=False)
                                     if int(tune["blocks_per_sm"]) == NCU_BATCH_CAPTURE_BLOCKS
                                     else None),
                         "bytes_per_particle_step": kbytes / kp if kp > 0 else None,
                         "traffic_unit": ("bytes per launch (ncu dram read+write on 16 targets at "
                                          f"{NCU_BATCH_CAPTURE_BLOCKS} blocks of 256 threads per SM, "
                                          "scaled by particle-steps; null at another launch shape)"),
                         "kernel": "k_batch_push", "kernel_ms_avg": km / kl,
                         "measured_over": f"{kl} direct launches after the timed window",
                         "peak_source": pk["source"]},
            "gpu_launches": launches, "clocks": clk,
            "ce_above_1MeV": {"rank0_min": min(ce), "rank0_max": max(ce),
                              "scan_eta_e2g": tot["E_xray_above"] / tot["E_injected"]}}


def run_batch(args):
    """The batched scan alone (not the headline line): the 1 ps window after
    the injection window."""
    import torch

    from paper_2107_01723_gb300 import build as B
    from paper_2107_01723_gb300 import workloads as W
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if rank == 0 or not os.path.exists(B.LIB):
        B.build()
    barrier(world)
    warm = args.warmup if args.warmup >= 200 else 200
    steps = args.steps if args.steps != 1000 else W.config4()["steps"] - warm - 1
    line = batch_result(args.batch_targets, warm, steps, args.precision, args.batch_tuning,
                        world, rank, local)
    if line is not None:
        print(json.dumps(line), flush=True)


def run_model(args):
    """The paper's loss-channel estimate (Sec. III.B) over its heatmap
    (intensity x Z), one GPU thread per parameter set, FP64; not the headline
    line.  value: parameter sets per second with inputs resident on the
    device; e2e: through hpic_model with host arrays."""
    import ctypes as C

    import torch

    from paper_2107_01723_gb300 import build as B
    from paper_2107_01723_gb300 import hpic
    from paper_2107_01723_gb300 import workloads as W
    B.build()
    pts = W.model_heatmap(n_I=args.model_n_I, n_Z=92)
    n = len(pts)
    host_in = (hpic.hpic_model_in * n)(*[hpic.model_in(p) for p in pts])
    nb_in, nb_out = C.sizeof(hpic.hpic_model_in) * n, C.sizeof(hpic.hpic_model_out) * n
    d_in = torch.empty(nb_in, dtype=torch.uint8, device="cuda")
    d_out = torch.empty(nb_out, dtype=torch.uint8, device="cuda")
    d_in.copy_(torch.frombuffer(bytearray(bytes(host_in)), dtype=torch.uint8))
    stream = torch.cuda.Stream()
    s = stream.cuda_stream
    for _ in range(args.warmup):
        hpic.hpic_model_device(n, d_in.data_ptr(), d_out.data_ptr(), 0, s)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        hpic.hpic_model_device(n, d_in.data_ptr(), d_out.data_ptr(), 0, s)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    out = (hpic.hpic_model_out * n).from_buffer_copy(bytes(d_out.cpu().numpy()))
    steps = sum(o.steps for o in out)
    t0 = time.perf_counter()
    res = hpic.hpic_model(pts, 0, s)
    wall = time.perf_counter() - t0
    # the oracle on a sample of the same sets
    from oracle import oracle as O
    t1 = time.perf_counter()
    k = 0
    while k < n and time.perf_counter() - t1 < 10.0:
        O.model(pts[(k * 97) % n])
        k += 1
    cpu_rate = k / (time.perf_counter() - t1)
    eta = [r["E_xray_above"] / r["E_injected"] for r in res]
    line = {"metric": "loss-channel estimate (Sec. III.B): parameter sets per second",
            "value": n / (ms / 1e3), "unit": "parameter sets/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"heatmap {args.model_n_I} intensities (1e20-1e22 W/cm^2) x Z = 1..92, "
                                   "100^3 um^3, n_i = 6e28 m^-3, I_ex = 11 eV Z, RK4 rel_step 0.01",
                       "points": n, "rk4_steps_per_call": steps},
            "rk4_steps_per_s": steps / (ms / 1e3),
            "roofline": {"bound": "alu", "note": "FP64 transcendental-bound (log, exp per RK4 stage)"},
            "e2e": {"value": n / wall, "unit": "parameter sets/s", "h2d_bytes_per_step": nb_in,
                    "d2h_bytes_per_step": nb_out},
            "cpu_baseline": {"value": cpu_rate, "unit": "parameter sets/s", "cores": 1,
                             "kind": "oracle", "sample": f"{k} sets of the heatmap, 10 s"},
            "eta_e2g": {"min": min(eta), "max": max(eta)}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="headline",
                    choices=["headline", "emission", "batch", "model", "thick", "small"])
    ap.add_argument("--model-n-I", type=int, default=256, help="loss-channel heatmap: intensities")
    ap.add_argument("--emission-n", type=int, default=2 ** 27)
    ap.add_argument("--batch-targets", type=int, default=64,
                    help="batched scan: targets (electrons scale with the count)")
    ap.add_argument("--batch-tuning", default="",
                    help="batched scan: 'blocks_per_sm,sort_interval' instead of the autotuner")
    ap.add_argument("--full-run", action="store_true",
                    help="run the whole headline workload in FP32 and FP64 and compare CE")
    ap.add_argument("--full-steps", type=int, default=0)
    ap.add_argument("--full-precision", default="both", choices=["both", "fp32", "fp64"])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-sub", action="store_true",
                    help="skip the batched-scan and emission sub-lines")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the FP32-vs-FP64 CE and closure window")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.full_run:
        run_full(args)
        return
    if args.workload == "emission":
        run_emission(args)
        return
    if args.workload == "thick":
        run_thick(args)
        return
    if args.workload == "small":
        run_small(args)
        return
    if args.workload == "batch":
        run_batch(args)
        if int(os.environ.get("WORLD_SIZE", "1")) > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    if args.workload == "model":
        run_model(args)
        return
    if args.impl == "reference":
        # the oracle runs on rank 0 only; other ranks exit without work
        run_reference(args, int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")))
        return
    world, rank, local = dist_setup()
    run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
