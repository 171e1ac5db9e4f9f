#!/usr/bin/env python
"""Throughput of the fused volumetric-curvilinear stream-and-collide step.

Workload: D3Q19, 256^3 cells, FP32 populations, a channel with tanh wall-normal
stretching (factor 0.7) and a sinusoidal bump on the lower wall (amplitude
0.05 h, wavelength half the streamwise length), walls with halfway
bounce-back, periodic streamwise and spanwise axes, constant body force,
tau = 0.8, rho = 1 with seeded 1% velocity noise. (Stretching 2.5 makes the
rest equilibrium negative near the walls and the run fails within tens of
steps; at tau <= 0.6 this bumped mesh is unstable at the lower wall after
about 300 steps. The per-cell work does not depend on either value.) A step is one time step over the whole lattice
(one fused kernel launch). Metric: MLUPS (million cell updates per second) and
the fraction of the measured HBM copy bandwidth that the algorithmic traffic
(each population read and written once, 2 * 19 * 4 = 152 bytes per cell
update) reaches.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
                  [--storage f32|f16|bf16 --reference rest|uniform]
                  [--workload batch --nmesh M]   (M uneven D2Q9 meshes, one launch per step)
                  [--workload warmstart --ntrain N --ntest M --iters K]   (learned warm start)
                  [--workload d3q39 --n N]   (6th-order isotropic set, FP64, N^3 periodic box)
                  [--workload precision --n 384 --drift-steps 10000]   (FP32 / FP16 / BF16
                      storage: MLUPS at N^3, error against the FP64 GPU path and the
                      oracle on a 64^3 instance, total-mass drift)
                  [--workload nn-forward]   (warm-start network forward pass, tensor cores
                      against CUDA cores)

Multi-GPU (torchrun, one rank per GPU): independent replicas of the workload,
no collective on the data path (weak scaling); timing is the max over ranks.
"""
import argparse
import hashlib
import json
import os
import re
import signal
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_CELL = {("19", "f32"): 2 * 19 * 4, ("19", "f64"): 2 * 19 * 8, ("9", "f32"): 2 * 9 * 4,
                  ("9", "f64"): 2 * 9 * 8, ("19", "f16"): 2 * 19 * 2, ("19", "bf16"): 2 * 19 * 2}
STEP_SOURCES = ["vlb_step.cu", "vlb_step.cuh", "vlb_collide.cuh", "vlb_addr.cuh", "vlb_internal.cuh"]
# the coefficient record values the D3Q19 FP32 step kernel reads per cell
# with one record per cell (CoefLayout<19>::RR: everything before the rest
# state, which that mode forms from J and g^ij; the wall velocity after it is
# read in moving-wall cells only)
RECORD_FLOATS_READ = 136


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--n", type=int, default=None,
                    help="cells per axis (default 256; 64 for --workload d3q39)")
    ap.add_argument("--stretch", type=float, default=0.7)
    ap.add_argument("--bump", type=float, default=0.05)
    ap.add_argument("--tau", type=float, default=0.8)
    ap.add_argument("--coef-mode", default="auto", choices=["auto", "full", "plane"])
    ap.add_argument("--mesh", default="channel", choices=["channel", "bump3d"],
                    help="bump3d: the lower-wall bump also varies spanwise (per-cell coefficient records)")
    ap.add_argument("--general-n", type=int, default=256,
                    help="cells per axis of the general-mesh leg (0 skips it)")
    ap.add_argument("--general-steps", type=int, default=200)
    ap.add_argument("--no-time-to-steady", action="store_true",
                    help="skip the reduced warm-start comparison of the default run")
    ap.add_argument("--tts-train", type=int, default=512)
    ap.add_argument("--tts-test", type=int, default=64)
    ap.add_argument("--tts-iters", type=int, default=1000)
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"],
                    help="population storage (arithmetic stays FP32)")
    ap.add_argument("--reference", default="rest", choices=["uniform", "rest"],
                    help="storage reference of 16-bit populations")
    ap.add_argument("--no-storage16", action="store_true",
                    help="skip the FP16-storage leg of the default run")
    ap.add_argument("--drift-steps", type=int, default=10000,
                    help="precision workload: steps of the total-mass drift runs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="channel",
                    choices=["channel", "batch", "warmstart", "d3q39", "precision", "nn-forward"],
                    help="batch: many uneven D2Q9 meshes advanced by one launch per step; "
                         "warmstart: train the warm-start network and compare time to steady")
    ap.add_argument("--ntrain", type=int, default=2048)
    ap.add_argument("--ntest", type=int, default=256)
    ap.add_argument("--iters", type=int, default=3000)
    ap.add_argument("--nmesh", type=int, default=512)
    a = ap.parse_args()
    if a.n is None:
        a.n = 64 if a.workload == "d3q39" else 256
    return a


def source_sha():
    h = hashlib.sha256()
    for f in STEP_SOURCES:
        with open(os.path.join(ROOT, "paper_2401_17183_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def ncu_traffic(ncell, name="step_d3q19_f32_channel_ncu.md"):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current step-kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", name)
    try:
        txt = open(p).read()
    except OSError:
        return None
    m_sha = re.search(r"source_sha:\s*([0-9a-f]+)", txt)
    m_b = re.search(r"dram_bytes_per_cell_update:\s*([0-9.]+)", txt)
    if not m_sha or not m_b or m_sha.group(1) != source_sha():
        return None
    return float(m_b.group(1)) * ncell


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.proc = None
        self.path = os.path.join("/tmp", "vlb_clocks_%d_%d.csv" % (os.getpid(), int(time.time())))
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(gpu_id)], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        os.remove(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def max_over_ranks(x, device=None):
    """Max of a per-rank float over all ranks of the default process group
    (returned unchanged when no group is initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(world, ncell, steps, seconds):
    """Whole-job cell updates per second (millions): every rank advances its own
    replica of ncell cells by steps steps; seconds is the slowest rank's time."""
    return world * ncell * steps / seconds / 1e6


def cpu_model():
    """Host CPU model and logical CPU count, from lscpu (else /proc/cpuinfo)."""
    info = {"model": None, "cpus": os.cpu_count(), "source": "os"}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            k, v = k.strip(), v.strip()
            if k == "Model name" and info["model"] is None:
                info["model"] = v
            elif k == "CPU(s)":
                info["cpus"] = int(v)
            elif k == "Vendor ID":
                info["vendor"] = v
        info["source"] = "lscpu"
    except Exception:
        pass
    if info["model"] is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    info["model"] = line.split(":", 1)[1].strip()
                    break
        except OSError:
            info["model"] = os.uname().machine
    return info


def _oracle_sample(n, tau, stretch, bump):
    from oracle import OracleSim
    from paper_2401_17183_gb300 import workloads as W
    mesh = W.channel_mesh(*n, stretch=stretch, bump=bump)
    rho, u = W.noise_fields(mesh, amp=0.01, seed=2)
    o = OracleSim(mesh, W.params(tau, body_force=(1e-6, 0.0, 0.0)))
    o.init(rho, u)
    return o


def _oracle_timed(o, min_steps, min_s, max_steps=200):
    """Steps of a running oracle until both min_steps and min_s are reached."""
    t = time.perf_counter()
    k = 0
    while k < min_steps or (time.perf_counter() - t < min_s and k < max_steps):
        o.step(1)
        k += 1
    return k, time.perf_counter() - t


def reference_sample_run(steps, warmup, tau, stretch, bump, budget_s=120.0):
    """The FP64 oracle as it stands, its time step on every host core
    (OpenMP over the cells), on a bounded sample of the channel family sized
    so that warmup + steps fit budget_s."""
    from oracle import set_threads
    cpu = cpu_model()
    procs = max(1, int(cpu["cpus"] or 1))
    set_threads(procs)
    o = _oracle_sample((8, 8, 8), tau, stretch, bump)
    t = time.perf_counter()
    o.step(1)
    per_cell = (time.perf_counter() - t) / 512
    per_step_budget = budget_s / max(1, steps + warmup)
    s = 8
    while (s + 4) ** 3 * per_cell <= per_step_budget and s < 48:
        s += 4
    o = _oracle_sample((s, s, s), tau, stretch, bump)
    o.step(warmup)
    t = time.perf_counter()
    o.step(steps)
    el = time.perf_counter() - t
    return {"value": s ** 3 * steps / el / 1e6, "cells": s ** 3, "steps": steps, "seconds": el, "cores": procs,
            "cpu": cpu,
            "sample": "%d^3 cells of the same channel family (stretch %g, bump %g h, walls, body force, "
                      "tau %g), %d timed steps, OpenMP over the cells on %d cores" % (s, stretch, bump, tau, steps, procs)}


def cpu_baseline_leg(tau, stretch, bump):
    """Oracle MLUPS on a bounded sample (32 x 32 x 16 cells of the channel
    family), its time step on every host core (OpenMP over the cells) and on
    one thread; at least 10 s of stepping each (the single-thread leg) or
    3 s (all cores)."""
    from oracle import set_threads
    n = (32, 32, 16)
    nc = n[0] * n[1] * n[2]
    cpu = cpu_model()
    procs = max(1, int(cpu["cpus"] or 1))
    before = set_threads(0)
    try:
        set_threads(1)
        o = _oracle_sample(n, tau, stretch, bump)
        o.step(1)
        k1, el1 = _oracle_timed(o, 3, 10.0)
        set_threads(procs)
        o = _oracle_sample(n, tau, stretch, bump)
        o.step(1)
        kp, elp = _oracle_timed(o, 10, 3.0, 2000)
    finally:
        set_threads(before)
    return {"value": nc * kp / elp / 1e6, "unit": "MLUPS", "cores": procs, "kind": "oracle", "cpu": cpu,
            "sample": "32x32x16 cells of the same channel family (D3Q19, FP64, stretch %g, bump %g h, "
                      "tau %g), %d steps with OpenMP over the cells on %d cores (%.1f s)"
                      % (stretch, bump, tau, kp, procs, elp),
            "single_thread": {"value": nc * k1 / el1 / 1e6, "unit": "MLUPS", "cores": 1, "steps": k1,
                              "seconds": el1}}


def general_mesh_leg(a, stream):
    """The same fused step on a mesh whose geometry varies along every axis (a
    channel whose lower-wall bump also varies spanwise): one coefficient record
    per cell, streamed from HBM with the populations. FP32, --general-n^3 cells,
    --general-steps timed steps after 5 warm-up steps."""
    import torch

    from paper_2401_17183_gb300 import vlb
    from paper_2401_17183_gb300 import workloads as W
    n = a.general_n
    mesh = W.channel_bump3d_mesh(n, n, n, stretch=a.stretch, bump=a.bump)
    prm = W.params(a.tau, body_force=(1e-6, 0.0, 0.0))
    rho, u = W.noise_fields(mesh, amp=0.01, seed=2)
    ncell = W.ncell(mesh)
    gm = vlb.Mesh(mesh)
    del mesh
    sim = vlb.Sim(gm, prm, rho, u, precision=vlb.VLB_F32, coef_mode=vlb.VLB_COEF_FULL,
                  stream=stream.cuda_stream)
    lay = sim.layout()
    sim.step(5)
    sim.sync()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(a.general_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    sim.sync()
    value = ncell * a.general_steps / (ms / 1e3) / 1e6
    peak, peak_kind = measured_peak_hbm()
    # bytes the kernel moves per cell update: populations read and written, and
    # the part of the cell's coefficient record it reads
    rec_bytes = 4 * RECORD_FLOATS_READ
    per_launch = ms / 1e3 / a.general_steps
    out = {"workload": "channel_bump3d_d3q19_%d^3_fp32_full_records" % n, "cells": ncell,
           "value": value, "unit": "MLUPS", "steps": a.general_steps,
           "ms_per_step": ms / a.general_steps, "coef_mode": "plane" if lay["plane"] else "full",
           "record_floats_stored": lay["coef_per_cell"], "record_bytes_read_per_cell": rec_bytes,
           "roofline": {"bound": "hbm", "peak": peak, "unit": "GB/s", "peak_kind": peak_kind,
                        "achieved_populations": 152 * ncell / per_launch / 1e9,
                        "frac_populations": 152 * ncell / per_launch / 1e9 / peak,
                        "achieved_with_records": (152 + rec_bytes) * ncell / per_launch / 1e9,
                        "frac_with_records": (152 + rec_bytes) * ncell / per_launch / 1e9 / peak,
                        "traffic": ncu_traffic(ncell, "step_d3q19_f32_bump3d_full_ncu.md")}}
    sim.close()
    gm.close()
    return out


def batch_meshes(nmesh, seed=4):
    """Seeded uneven 2D channels: streamwise (periodic, fastest) size
    log-uniform in [64, 512], wall-normal size half of it, tanh stretching
    uniform in [0.3, 0.9]."""
    import numpy as np
    from paper_2401_17183_gb300 import workloads as W
    u = W.uniform(seed, nmesh, 2)
    out = []
    for k in range(nmesh):
        n1 = int(round(64 * 8 ** u[k, 0]))
        n0 = max(4, n1 // 2)
        out.append(W.channel2d_mesh(n0, n1, stretch=0.3 + 0.6 * u[k, 1]))
    return out


def bench_batch(a):
    """One kernel launch per time step for the whole set (CUDA graph replays),
    against stepping every mesh on its own."""
    import numpy as np
    import torch

    from paper_2401_17183_gb300 import build as B
    B.build()
    from paper_2401_17183_gb300 import vlb
    from paper_2401_17183_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    meshes = batch_meshes(a.nmesh)
    sims = []
    for k, mesh in enumerate(meshes):
        rho, u = W.noise_fields(mesh, amp=0.01, seed=100 + k)
        sims.append(vlb.Sim(vlb.Mesh(mesh), W.params(a.tau, body_force=(0.0, 1e-6, 0.0)), rho, u,
                            precision=vlb.VLB_F32, stream=stream.cuda_stream))
    ncell = sum(W.ncell(m) for m in meshes)
    batch = vlb.Batch(sims)

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    # every block shape at its default run length (for the record), then the
    # tuner's choice of shape and run length
    shapes, k_shape = [], max(32, a.steps // 4)
    for i in range(4):
        batch.set_shape(i)
        batch.step(a.warmup)
        ms_i = timed(lambda: batch.step(k_shape))
        ly = batch.layout()
        shapes.append({"threads": ly["threads"], "min_blocks_per_sm": ly["min_blocks"],
                       "tiles_per_block": ly["run_length"], "value": ncell * k_shape / (ms_i / 1e3) / 1e6})
    run = batch.tune(4)
    batch.step(a.warmup)
    torch.cuda.synchronize()

    sampler = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    ms = timed(lambda: batch.step(a.steps))
    clocks = sampler.stop()
    for s in sims:
        s.sync()
    k_alone = max(2, a.steps // 10)
    ms_alone = timed(lambda: [s.step(k_alone) for s in sims])
    for s in sims:
        s.sync()
    value = ncell * a.steps / (ms / 1e3) / 1e6
    alone = ncell * k_alone / (ms_alone / 1e3) / 1e6
    bpc = BYTES_PER_CELL[("9", "f32")]
    peak, peak_kind = measured_peak_hbm()
    achieved = bpc * ncell / (ms / 1e3 / a.steps) / 1e9
    lay = batch.layout()
    line = {
        "metric": "MLUPS, batch of uneven D2Q9 meshes in one launch per step", "value": value,
        "unit": "MLUPS", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded meshes and 1% velocity noise)",
        "config": {"workload": "batch_%d_channel2d_d2q9_fp32" % a.nmesh, "meshes": a.nmesh, "cells": ncell,
                   "sizes": "streamwise log-uniform 64..512, wall-normal half", "tau": a.tau,
                   "blocks_per_launch": lay["blocks"], "tiles_per_block": run,
                   "threads_per_block": lay["threads"], "min_blocks_per_sm": lay["min_blocks"],
                   "graph": "32 launches per CUDA graph"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                     "bytes_per_cell_update": bpc},
        "shapes_at_default_run": shapes,
        "one_launch_per_mesh": {"value": alone, "unit": "MLUPS", "steps": k_alone,
                                "speedup_of_batch": value / alone},
        "clocks": clocks, "gpu_launches": a.steps,
    }
    print(json.dumps(line))


def bench_d3q39(a):
    """The 6th-order isotropic velocity set D3Q39 (FP64, pair-form
    collision) on a periodic sine-mapped box of --n^3 cells."""
    import torch

    from paper_2401_17183_gb300 import build as B
    B.build()
    from paper_2401_17183_gb300 import vlb
    from paper_2401_17183_gb300 import workloads as W
    n = a.n
    mesh = W.periodic_sine_mesh3d(n, 0.01, q=39)
    rho, u = W.noise_fields(mesh, amp=0.01, seed=2)
    stream = torch.cuda.current_stream()
    sim = vlb.Sim(vlb.Mesh(mesh), W.params(a.tau, body_force=(1e-6, 0.0, 0.0)), rho, u,
                  precision=vlb.VLB_F64, stream=stream.cuda_stream)
    sim.step(a.warmup)
    sim.sync()
    torch.cuda.synchronize()
    sampler = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(a.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    sim.sync()
    ms = e0.elapsed_time(e1)
    ncell = n ** 3
    value = ncell * a.steps / (ms / 1e3) / 1e6
    bpc = 2 * 39 * 8
    peak, peak_kind = measured_peak_hbm()
    achieved = bpc * ncell / (ms / 1e3 / a.steps) / 1e9
    line = {
        "metric": "MLUPS, D3Q39 (6th-order isotropic) fused step", "value": value, "unit": "MLUPS",
        "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded periodic sine-mapped box, 1% velocity noise)",
        "config": {"workload": "d3q39_sine_box_%d^3_fp64" % n, "cells": ncell, "lattice": "D3Q39",
                   "amplitude": "0.01 L", "tau": a.tau},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                     "bytes_per_cell_update": bpc,
                     "limiter": "FP64 arithmetic of the per-direction collision, not DRAM"},
        "clocks": clocks, "gpu_launches": a.steps,
    }
    print(json.dumps(line))


def time_steps(sim, steps, warmup, stream):
    """Device time (ms) of `steps` time steps of one simulation after `warmup`
    untimed ones: CUDA events on the launching stream, synchronised on both
    sides."""
    import torch
    sim.step(warmup)
    sim.sync()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    sim.sync()
    return e0.elapsed_time(e1)


def storage16_leg(a, gmesh, prm, rho, u, stream, storage="f16"):
    """The same workload with 16-bit population storage relative to the rest
    state (FP32 arithmetic), timed like the headline."""
    from paper_2401_17183_gb300 import vlb
    prec = {"f16": vlb.VLB_F16, "bf16": vlb.VLB_BF16}[storage]
    sim = vlb.Sim(gmesh, prm, rho, u, precision=prec, stream=stream.cuda_stream,
                  reference=vlb.VLB_REF_REST)
    ms = time_steps(sim, a.steps, a.warmup, stream)
    sim.close()
    ncell = a.n ** 3
    peak, peak_kind = measured_peak_hbm()
    bpc = BYTES_PER_CELL[("19", storage)]
    achieved = bpc * ncell / (ms / 1e3 / a.steps) / 1e9
    return {"storage": storage, "reference": "rest", "value": ncell * a.steps / (ms / 1e3) / 1e6,
            "unit": "MLUPS", "ms_per_step": ms / a.steps, "steps": a.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind, "bytes_per_cell_update": bpc,
                         "traffic": ncu_traffic(ncell, "step_d3q19_f16_channel_ncu.md") if storage == "f16" else None,
                         "kernel": "k_step<19,%s,float>" % ("__half" if storage == "f16" else "__nv_bfloat16"),
                         "source_sha": source_sha()}}


PRECISION_FORMS = [("f64", "uniform"), ("f32", "uniform"), ("f16", "rest"), ("f16", "uniform"),
                   ("bf16", "rest"), ("bf16", "uniform")]


def precision_accuracy(stream, drift_steps):
    """Every storage form on the 64^3 instance of workloads.precision_instance:
    max |rho - rho_ref| and max |u - u_ref| / max |u_ref| against the FP64 GPU
    run and, where tests/golden/precision64_oracle.npz exists (written by
    tests/golden/precision_reference.py, which runs only the oracle), against
    the oracle, at its checkpoints; and the relative drift of the total mass
    over drift_steps steps from the run's own start."""
    import numpy as np

    from paper_2401_17183_gb300 import vlb
    from paper_2401_17183_gb300 import workloads as W
    n = 64
    mesh, prm, rho, u = W.precision_instance(n)
    gm = vlb.Mesh(mesh)
    ref_path = os.path.join(ROOT, "tests", "golden", "precision%d_oracle.npz" % n)
    orc = dict(np.load(ref_path)) if os.path.exists(ref_path) else None
    marks = [int(s) for s in orc["steps"]] if orc is not None else [200, 1000]
    prec = {"f64": vlb.VLB_F64, "f32": vlb.VLB_F32, "f16": vlb.VLB_F16, "bf16": vlb.VLB_BF16}

    def errs(mo, r, uu):
        su = np.abs(uu).max()
        return {"rho_abs": float(np.abs(mo["rho"] - r).max()), "u_rel": float(np.abs(mo["u"] - uu).max() / su)}

    fields, out = {}, {}
    for st, rf in PRECISION_FORMS:
        name = st if st in ("f64", "f32") else "%s_%s" % (st, rf)
        sim = vlb.Sim(gm, prm, rho, u, precision=prec[st], stream=stream.cuda_stream,
                      reference=vlb.VLB_REF_REST if rf == "rest" else vlb.VLB_REF_UNIFORM)
        res, done = {}, 0
        for k in marks:
            sim.step(k - done)
            done = k
            mo = sim.moments()
            fields[(name, k)] = mo
            r = {}
            if name != "f64":
                f64 = fields[("f64", k)]
                r["vs_fp64_gpu"] = errs(mo, f64["rho"], f64["u"])
            if orc is not None:
                r["vs_oracle"] = errs(mo, orc["rho_%d" % k], orc["u_%d" % k])
            res[str(k)] = r
        sim.close()
        # total-mass drift from the run's own (rounded) start
        sim = vlb.Sim(gm, prm, rho, u, precision=prec[st], stream=stream.cuda_stream,
                      reference=vlb.VLB_REF_REST if rf == "rest" else vlb.VLB_REF_UNIFORM)
        m0 = sim.moments(fields=False)["mass"]
        sim.step(drift_steps)
        m1 = sim.moments(fields=False)["mass"]
        sim.close()
        res["mass_drift"] = {"steps": drift_steps, "relative": float(m1 / m0 - 1.0)}
        out[name] = res
    oracle = None
    if orc is not None:
        oracle = {"file": os.path.relpath(ref_path, ROOT), "steps": marks,
                  "mass_drift": {"steps": marks[-1], "relative": float(orc["mass_%d" % marks[-1]] / orc["mass0"] - 1.0)}}
    return {"instance": "channel_d3q19_64^3 (stretch 0.7, bump 0.05 h, tau 0.8, body force 1e-5, "
                        "seeded 1% noise, seed 3)",
            "checkpoints": marks, "metrics": "rho_abs = max|rho - rho_ref|; u_rel = max|u - u_ref| / max|u_ref|",
            "oracle": oracle if oracle is not None else "absent (run tests/golden/precision_reference.py)",
            "forms": out}


def bench_precision(a):
    """The storage-precision forms: throughput of FP32, FP16 and BF16 (rest
    reference, FP32 arithmetic) on the --n^3 channel of the headline workload
    (default 256^3; the 384^3 channel of the precision configuration needs
    --steps 400, since the scheme goes unstable there between 500 and 600
    steps), timed the same way in the same run, and their accuracy and mass
    drift (precision_accuracy)."""
    import torch

    from paper_2401_17183_gb300 import build as B
    B.build()
    from paper_2401_17183_gb300 import vlb
    from paper_2401_17183_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    n = a.n
    mesh = W.channel_mesh(n, n, n, stretch=a.stretch, bump=a.bump)
    prm = W.params(a.tau, body_force=(1e-6, 0.0, 0.0))
    rho, u = W.noise_fields(mesh, amp=0.01, seed=2)
    gm = vlb.Mesh(mesh)
    del mesh
    ncell = n ** 3
    peak, peak_kind = measured_peak_hbm()
    sampler = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    thr = {}
    for st in ("f32", "f16", "bf16"):
        p = {"f32": vlb.VLB_F32, "f16": vlb.VLB_F16, "bf16": vlb.VLB_BF16}[st]
        sim = vlb.Sim(gm, prm, rho, u, precision=p, stream=stream.cuda_stream,
                      reference=vlb.VLB_REF_REST if st != "f32" else vlb.VLB_REF_UNIFORM)
        ms = time_steps(sim, a.steps, a.warmup, stream)
        sim.close()
        bpc = BYTES_PER_CELL[("19", st)]
        ach = bpc * ncell / (ms / 1e3 / a.steps) / 1e9
        thr[st] = {"value": ncell * a.steps / (ms / 1e3) / 1e6, "unit": "MLUPS", "ms_per_step": ms / a.steps,
                   "reference": "rest" if st != "f32" else "uniform", "bytes_per_cell_update": bpc,
                   "achieved_gbs": ach, "frac": ach / peak}
    clocks = sampler.stop()
    del gm
    acc = precision_accuracy(stream, a.drift_steps)
    line = {
        "metric": "MLUPS of the 16-bit storage forms (FP32 arithmetic) and their error against the FP64 GPU "
                  "path and the oracle", "value": thr["f16"]["value"], "unit": "MLUPS",
        "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": thr["f16"]["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f16 storage, f32 arithmetic", "data": "synthetic (seeded mesh and 1% velocity noise)",
        "config": {"workload": "channel_d3q19_%d^3_precision_forms" % n, "cells": ncell, "lattice": "D3Q19",
                   "stretch": a.stretch, "bump": a.bump, "tau": a.tau, "body_force": 1e-6,
                   "l2": "no flush: populations >= %.2f GB > 129 MB L2" % (ncell * 19 * 2 / 1e9)},
        "throughput": thr, "peak": peak, "peak_kind": peak_kind, "clocks": clocks,
        "f16_over_f32": thr["f16"]["value"] / thr["f32"]["value"], "accuracy": acc,
        "gpu_launches": 3 * a.steps,
    }
    print(json.dumps(line))


def bench_nn_forward(a):
    """Forward passes of the warm-start network (width 64, 8 input channels,
    32 x 64 grid, batch 32, bfloat16 storage): the 3x3 layers on the tensor
    cores (tcgen05) against every layer on the CUDA cores."""
    import torch

    from paper_2401_17183_gb300 import build as B
    B.build()
    from paper_2401_17183_gb300 import nn
    nn.load()
    H, W, bt, wd = 32, 64, 32, 64
    net = nn.Net(8, 3, wd, H, W, bt, storage=nn.VLB_NN_BF16, seed=7)
    g = torch.Generator(device="cuda").manual_seed(7)
    x = torch.rand((bt, 8, H, W), device="cuda", generator=g) * 2 - 1
    y = torch.zeros((bt, 3, H, W), device="cuda")
    res = {}
    for tc in (True, False):
        net.set_tensor_cores(tc)
        for _ in range(a.warmup):
            net.forward(x.data_ptr(), y.data_ptr(), bt)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.steps):
            net.forward(x.data_ptr(), y.data_ptr(), bt)
        e1.record()
        torch.cuda.synchronize()
        res["tensor_cores" if tc else "cuda_cores"] = e0.elapsed_time(e1) / a.steps
    line = {"metric": "warm-start network forward pass, ms per batch", "value": res["tensor_cores"], "unit": "ms",
            "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16 storage, f32 accumulation", "data": "synthetic (uniform inputs)",
            "config": {"workload": "unet_w64_8ch_32x64_batch32_bf16"},
            "cuda_cores_ms": res["cuda_cores"], "speedup": res["cuda_cores"] / res["tensor_cores"],
            "gpu_launches": None}
    print(json.dumps(line))


def warmstart_leg(ntrain, ntest, iters):
    """Steps and wall time to a 1e-6 residual from the learned prediction and
    from rest, on held-out members of the bumped 2D channel family."""
    import numpy as np

    from paper_2401_17183_gb300 import warmstart as WS
    t0 = time.perf_counter()
    X, Y, keep = WS.dataset(WS.family(4, ntrain))
    t_data = time.perf_counter() - t0
    ws = WS.WarmStart()
    losses, t_train = ws.train(X, Y, iters)
    test = WS.family(5, ntest)
    Xt, Yt, kt = WS.dataset(test)
    tspec = [test[k] for k in kt]
    t1 = time.perf_counter()
    pred = ws.predict(Xt)
    t_pred = time.perf_counter() - t1
    err = [float(np.linalg.norm(np.stack([p[1][..., 0], p[1][..., 1]]) - Yt[i, 1:]) / np.linalg.norm(Yt[i, 1:]))
           for i, p in enumerate(pred)]
    cold = [m[2] for m in WS.make_sims(tspec)]
    sc, tc = WS.run_to_steady(cold)
    warm = [m[2] for m in WS.make_sims(tspec, init=pred)]
    sw, tw = WS.run_to_steady(warm)
    return {
        "value": float(sc.mean() / sw.mean()), "unit": "x fewer steps (mean over held-out members)",
        "config": {"workload": "warmstart_channel2d_32x64_d2q9", "train_members": len(keep),
                   "test_members": len(kt), "iters": iters, "batch": ws.batch,
                   "params": ws.net.nparams, "tau": WS.TAU, "residual": 1e-6},
        "cold": {"steps_mean": float(sc.mean()), "steps_max": int(sc.max()), "wall_s": tc},
        "warm": {"steps_mean": float(sw.mean()), "steps_max": int(sw.max()), "wall_s": tw + t_pred,
                 "inference_s": t_pred},
        "wall_speedup": float(tc / (tw + t_pred)),
        "prediction_u_rel_err": {"mean": float(np.mean(err)), "max": float(np.max(err))},
        "train": {"loss_first": losses[0], "loss_last": losses[-1], "seconds": t_train,
                  "data_seconds": t_data},
    }


def bench_warmstart(a):
    from paper_2401_17183_gb300 import build as B
    B.build()
    r = warmstart_leg(a.ntrain, a.ntest, a.iters)
    line = {
        "metric": "time-to-steady (1e-6 residual), learned warm start vs plain cold start",
        "value": r["value"], "unit": r["unit"],
        "n_gpus": 1, "steps": None, "warmup": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 solver; bf16 network storage with f32 accumulation",
        "data": "synthetic (seeded bumped 2D channels; steady targets from the solver)",
        "config": r["config"], "cold": r["cold"], "warm": r["warm"], "wall_speedup": r["wall_speedup"],
        "prediction_u_rel_err": r["prediction_u_rel_err"], "train": r["train"],
    }
    print(json.dumps(line))


def main():
    a = args_parse()
    if a.workload == "batch":
        return bench_batch(a)
    if a.workload == "warmstart":
        return bench_warmstart(a)
    if a.workload == "d3q39":
        return bench_d3q39(a)
    if a.workload == "precision":
        return bench_precision(a)
    if a.workload == "nn-forward":
        return bench_nn_forward(a)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    metric = "MLUPS & % HBM roofline (fused D3Q19 stream-and-collide step)"
    cfg = {"workload": "channel_d3q19_%d^3_%s" % (a.n, "fp32" if a.storage == "f32" else a.storage),
           "cells": a.n ** 3, "lattice": "D3Q19",
           "stretch": a.stretch, "bump": a.bump, "tau": a.tau, "walls": "eta (halfway bounce-back)",
           "periodic": "xi, zeta", "body_force": 1e-6,
           "l2": "no flush: populations %.2f GB > 129 MB L2"
                 % (a.n ** 3 * BYTES_PER_CELL[("19", a.storage)] / 2 / 1e9)}
    if a.storage != "f32":
        cfg["storage_reference"] = a.reference

    if a.impl == "reference":
        if rank != 0:
            return
        r = reference_sample_run(a.steps, a.warmup, a.tau, a.stretch, a.bump)
        line = {"impl": "reference", "metric": metric, "value": r["value"], "unit": "MLUPS",
                "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
                "ms_per_step": 1e3 * r["seconds"] / r["steps"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": cfg,
                "cpu_baseline": {"value": r["value"], "unit": "MLUPS", "cores": r["cores"],
                                 "kind": "oracle", "sample": r["sample"], "cpu": r["cpu"]},
                "e2e": {"value": r["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import numpy as np
    import torch

    from paper_2401_17183_gb300 import build as B
    B.build()
    from paper_2401_17183_gb300 import vlb
    from paper_2401_17183_gb300 import workloads as W

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)

    make = W.channel_bump3d_mesh if a.mesh == "bump3d" else W.channel_mesh
    mesh = make(a.n, a.n, a.n, stretch=a.stretch, bump=a.bump)
    if a.mesh == "bump3d":
        cfg["workload"] = cfg["workload"].replace("channel_", "channel_bump3d_")
    prm = W.params(a.tau, body_force=(1e-6, 0.0, 0.0))
    rho, u = W.noise_fields(mesh, amp=0.01, seed=2)
    ncell = W.ncell(mesh)
    gmesh = vlb.Mesh(mesh)
    info = gmesh.info()
    mode = {"auto": vlb.VLB_COEF_AUTO, "full": vlb.VLB_COEF_FULL, "plane": vlb.VLB_COEF_PLANE}[a.coef_mode]
    prec = {"f32": vlb.VLB_F32, "f16": vlb.VLB_F16, "bf16": vlb.VLB_BF16}[a.storage]
    ref = vlb.VLB_REF_REST if a.reference == "rest" else vlb.VLB_REF_UNIFORM
    sim = vlb.Sim(gmesh, prm, rho, u, precision=prec, coef_mode=mode, stream=stream.cuda_stream,
                  reference=ref)
    lay = sim.layout()
    cfg["coef_mode"] = "plane" if lay["plane"] else "full"
    cfg["feq_rest_min"] = info["feq_rest_min"]

    # ---- device-resident timing
    sim.step(a.warmup)
    sim.sync()
    gpu_id = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local if world > 1 else 0]
    sampler = ClockSampler(gpu_id) if rank == 0 else None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(a.steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1)
    sim.sync()     # raises on a kernel-reported error (e.g. a non-converged solve)
    ms = max_over_ranks(ms, dev)
    value = job_mlups(world, ncell, a.steps, ms / 1e3)
    per_launch_s = ms / 1e3 / a.steps
    bpc = BYTES_PER_CELL[("19", a.storage)]
    peak, peak_kind = measured_peak_hbm()
    achieved = bpc * ncell / per_launch_s / 1e9
    traffic = ncu_traffic(ncell) if a.storage == "f32" else None

    # ---- end to end through the public API with host buffers
    e2e = None
    if not a.no_e2e:
        pin_rho = torch.from_numpy(rho).pin_memory()
        pin_u = torch.from_numpy(np.ascontiguousarray(u)).pin_memory()
        out_rho = torch.empty(ncell, dtype=torch.float64).pin_memory()
        out_u = torch.empty(ncell * 3, dtype=torch.float64).pin_memory()
        out_ut = torch.empty(ncell * 3, dtype=torch.float64).pin_memory()
        out_t = torch.empty(7, dtype=torch.float64).pin_memory()
        # one untimed pass through the same buffers (first-touch of the pinned pages)
        sim.reset_ptr(pin_rho.data_ptr(), pin_u.data_ptr())
        sim.moments_ptr(out_rho.data_ptr(), out_u.data_ptr(), out_ut.data_ptr(), out_t.data_ptr())
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        # the steps of this run carry events of their own: they start from the
        # reset state, whose first steps take more chord evaluations than the
        # warmed-up steps of the device-resident timing
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        sim.reset_ptr(pin_rho.data_ptr(), pin_u.data_ptr())
        t1 = time.perf_counter()
        f0.record(stream)
        sim.step(a.steps)
        f1.record(stream)
        sim.moments_ptr(out_rho.data_ptr(), out_u.data_ptr(), out_ut.data_ptr(), out_t.data_ptr())
        t3 = time.perf_counter()
        e2e_steps_s = f0.elapsed_time(f1) / 1e3
        el = max_over_ranks(t3 - t0, dev)
        # after the timed region: the moments kernels alone (totals only to the
        # host), so that the device-to-host copy of the fields can be told apart
        sim.moments_ptr(0, 0, 0, out_t.data_ptr())
        t4 = time.perf_counter()
        sim.moments_ptr(0, 0, 0, out_t.data_ptr())
        t5 = time.perf_counter()
        h2d = 8 * ncell * 4
        d2h = 8 * ncell * 7 + 56
        e2e = {"value": job_mlups(world, ncell, a.steps, el), "unit": "MLUPS",
               "h2d_bytes_per_step": h2d / a.steps, "d2h_bytes_per_step": d2h / a.steps,
               "api": "vlb_reset(host rho,u) + vlb_step(K) + vlb_moments(host rho,u,u~,totals)",
               # reset: H2D of rho and u plus the initialisation kernel; steps:
               # this run's K steps, device-timed; moments: the moments and totals
               # kernels with only the totals copied back; d2h: the rest of the
               # time from the step launches to the end of vlb_moments (the
               # fields' copy)
               "phases_s": {"reset": t1 - t0, "steps": e2e_steps_s, "moments_kernels": t5 - t4,
                            "fields_d2h": max(0.0, (t3 - t1) - e2e_steps_s - (t5 - t4))}}

    general = tts = s16 = None
    if a.mesh == "channel" and a.storage == "f32" and world == 1 and not a.no_storage16:
        # the FP16-storage form of the same workload (rest reference)
        s16 = storage16_leg(a, gmesh, prm, rho, u, stream)
    if a.general_n > 0 and a.mesh == "channel" and a.storage == "f32" and world == 1:
        del sim, gmesh
        general = general_mesh_leg(a, stream)
    if not a.no_time_to_steady and a.mesh == "channel" and a.storage == "f32" and world == 1:
        # the second half of the metric: time to a 1e-6 residual, learned warm
        # start against the cold start (a reduced training set that fits the run)
        tts = warmstart_leg(a.tts_train, a.tts_test, a.tts_iters)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    cpu = None if (a.no_cpu_baseline or world > 1) else cpu_baseline_leg(a.tau, a.stretch, a.bump)
    line = {
        "metric": metric, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if a.storage == "f32" else "%s storage, f32 arithmetic" % a.storage,
        "data": "synthetic (seeded mesh and 1% velocity noise)", "config": cfg,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)",
                     "bytes_per_cell_update": bpc,
                     "kernel": "k_step<19,%s,float>" % {"f32": "float", "f16": "__half",
                                                        "bf16": "__nv_bfloat16"}[a.storage],
                     "source_sha": source_sha()},
        "clocks": clocks, "e2e": e2e, "gpu_launches": a.steps, "cpu_baseline": cpu,
        "storage16": s16, "general_mesh": general, "time_to_steady": tts,
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
