"""Throughput of the GR PIC hot path (push + deposit + field update) on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                [--workload wald512] [--precision both|fp64|mixed] [--sort-every 10]

A step is one full PIC step (Sec. 3.4 of arXiv:2511.17701) over the whole workload:
field predict, (sort), fused push + deposit of both species, field advance. The default
workload is the 512^2 Kerr (a = 0.9) Wald configuration with 32 particles per cell per
species (16,777,216 particles), synthetic and seeded. By default it is timed in FP64 (the
line's value, with the end-to-end leg and the CPU oracle beside it) and then in mixed
precision on the same workload (the "mixed" object). Prints one JSON line.

--impl reference times the CPU oracle (FP64, OpenMP over particles) on the host cores,
each step on a bounded sample of the same workload.
Under torchrun with N > 1 every rank runs an independent replica of the workload on its
own GPU (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = ("particle-steps/sec (push+deposit+field) & % HBM roofline, FP64 vs mixed, 1 GB300")

# Algorithmic bytes of one particle-step of the dominant kernel of each precision.
# FP64 k_push<deposit> (SoA; read: i1, i2, dx1, dx2, u1, u2, u3, phi, w, tag; write: the same
# minus w plus the previous position i1p, i2p, dx1p, dx2p): 4+4+8+8+24+8+8+1 = 65 B read,
# 4+4+8+8+24+8+1 + 4+4+8+8 = 81 B written.
FP64_BYTES_PER_PARTICLE_STEP = 65 + 81
# Mixed k_push32<deposit> (FP32 offsets, momenta, phi and w; the guard bitmask): 4+4+4+4+12+4+4
# +1 + 1/8 = 37 B read; i1p, i2p, dx1p, dx2p, i1, i2, dx1, dx2 (32) + u (12) + phi (4) = 48 B
# written.
MIXED_BYTES_PER_PARTICLE_STEP = 37 + 48
# FP64 pipe operations (DFMA + DMUL + DADD thread instructions) per particle-step of
# k_push<deposit> on the wald512 workload, counted by ncu, and as flops (2 DFMA + DMUL +
# DADD): with the implicit iterations refined from an FP32 predictor and one Newton step on
# its FP32 Jacobian (iter_tol > 0): 303 + 354 + 109 = 767 (1070 flop); stopped at an exact
# repeat (iter_tol = 0): 476 + 548 + 120 = 1144 (1620 flop). The FP64 pipe issues 2 such
# operations per clock per SM.
FP64_PIPE_OPS_PER_PARTICLE_STEP = {True: 767, False: 1144}
FP64_FLOP_PER_PARTICLE_STEP = {True: 1070, False: 1620}
SMS, MAX_SM_GHZ = 152, 2.07
FP64_PIPE_PEAK_GOPS = 2 * SMS * MAX_SM_GHZ  # 629 G operations/s
# Warp instructions issued per particle by k_push32<deposit> on the wald512 workload (ncu:
# 384.9 M over 8.39 M particles with 12 resident blocks per SM, spills included); an SM
# issues at most 4 warp instructions per clock.
MIXED_WARP_INST_PER_PARTICLE = 45.9
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per particle of the dominant
# kernels on the wald512 workload, from one ncu capture each: k_push<deposit> at 4 particles
# per cell and species (87.5 + 32.5 MB over 1,048,576 particles; traffic grows with the
# particles, so a full launch is this times its particles), k_push32<deposit> at the full
# size (314.6 + 615.9 MB over 8,388,608 particles).
TRAFFIC_BYTES_PER_PARTICLE = {"fp64": (87.5e6 + 32.5e6) / 1048576,
                              "mixed": (314.6e6 + 615.9e6) / 8388608}
ISSUE_PEAK_GINST = 4 * SMS * MAX_SM_GHZ  # 1259 G warp instructions/s


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                rows.append(p)
            except ValueError:
                pass
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, name in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(ws, x, device):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(ws, x, device):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


PRECISION_DESC = {"fp64": "FP64",
                  "mixed": "mixed precision (FP32 state, fields and currents; FP64 metric "
                           "within 4 cells of the horizon and the axes)"}


def field_kind(cfg, lib_side=True):
    """The initial field of a workload: Wald (default) or the BZ monopole."""
    if cfg.get("field") == "monopole":
        if lib_side:
            from paper_2511_17701_gb300 import FIELD_MONOPOLE
            return FIELD_MONOPOLE
        from oracle import oracle as O
        return O.FIELD_MONOPOLE
    if lib_side:
        from paper_2511_17701_gb300 import FIELD_WALD
        return FIELD_WALD
    from oracle import oracle as O
    return O.FIELD_WALD


def workload_desc(name, cfg, n_total, precision="fp64"):
    field = ("monopole A_phi=-B0 cos(theta)" if cfg.get("field") == "monopole" else "Wald")
    return ("%s: Kerr a=%g, %s B0=%g, %dx%d log-r grid, r in [%.4g, %g], e+- pairs %d "
            "per cell per species (%d particles), Maxwell-Juttner theta_T=%g, density ~ r^-%g, "
            "%s" % (name, cfg["a"], field, cfg["B0"], cfg["n_r"], cfg["n_theta"], cfg["r_min"],
                    cfg["r_max"], cfg["ppc"], n_total, cfg["theta_T"],
                    cfg.get("density_power", 0.0), PRECISION_DESC[precision]))


def oracle_workload(cfg, frac, seed=99):
    """The oracle holding the workload's grid and, when frac < 1, the particles of a
    seeded random fraction of the cells (a bounded sample)."""
    from oracle import oracle as O
    cells = None
    if frac < 1.0:
        cells = W.random_cells(cfg, max(1, int(cfg["n_r"] * cfg["n_theta"] * frac)), seed)
    osim = O.OracleSim(cfg)
    osim.init_fields(field_kind(cfg, lib_side=False), cfg["B0"])
    pl = W.pair_plasma(cfg, cells=cells)
    for s in range(2):
        osim.add_species(pl["pos"], pl["uhat"][s], pl["w0"], pl["qm"][s], pl["qc"][s],
                         pl["density_power"])
    return osim


def oracle_steps(osim, steps):
    """Seconds of each of `steps` full oracle PIC steps, and the particles pushed."""
    times, parts = [], 0
    for _ in range(steps):
        parts += sum(s.n for s in osim.species)
        t0 = time.perf_counter()
        osim.step(1)
        times.append(time.perf_counter() - t0)
    return times, parts


def host_cores():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def run_reference(args, ws, rank):
    if rank != 0:
        return
    cfg = W.grid_config(args.workload)
    frac = args.ref_frac
    osim = oracle_workload(cfg, frac)
    n = sum(s.n for s in osim.species)
    oracle_steps(osim, args.warmup)
    times, parts = oracle_steps(osim, args.steps)
    value = parts / sum(times)
    line = {"metric": METRIC, "value": value,
            "unit": "particle-steps/s", "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_desc(args.workload, cfg,
                                                 2 * cfg["n_r"] * cfg["n_theta"] * cfg["ppc"])},
            "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": host_cores(),
                             "kind": "oracle",
                             "sample": "full %dx%d grid with the particles of %.1f%% of the "
                                       "cells (%d particles), %d warm-up + %d timed steps" % (
                                           cfg["n_r"], cfg["n_theta"], 100 * frac, n,
                                           args.warmup, args.steps)},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


_PLASMA = {}


def measure(args, precision, ws, rank, local, workload=None, photons=False, extra=None):
    """Time args.steps full steps of the workload at one precision; returns the pieces of
    the JSON line (and the Sim for the end-to-end leg). photons: one species of massless
    particles at the electrons' positions and momenta instead of the e+- pairs; extra:
    further configuration (e.g. n_filter)."""
    import torch

    from paper_2511_17701_gb300 import Sim

    device = torch.device("cuda", local)
    workload = workload or args.workload
    cfg = W.grid_config(workload, sort_every=args.sort_every, tile_r=args.tile,
                        tile_theta=args.tile, precision=precision,
                        tiled_push=1 if args.tiled_push else 0, iter_tol=args.iter_tol)
    if args.ppc and workload == args.workload:
        cfg["ppc"] = args.ppc
    cfg.update(extra or {})
    # the seeded plasma of a workload is drawn once per process (the two precisions and the
    # photon run share it: drawing 377 M particles takes a minute and a half)
    key = (workload, cfg["seed"] + 1000 * rank, cfg["ppc"], cfg["n_r"], cfg["n_theta"])
    if key not in _PLASMA:
        _PLASMA.clear()
        _PLASMA[key] = W.pair_plasma(cfg, seed=cfg["seed"] + 1000 * rank)
    pl = _PLASMA[key]
    n = pl["pos"]["i1"].size
    nsp = 1 if photons else 2
    sim = Sim(dict(cfg, massless=[0] if photons else []), [n] * nsp, device=device)
    sim.init_metric()
    sim.init_fields(field_kind(cfg), cfg["B0"])
    for s in range(nsp):
        sim.load_particles(s, pl["pos"], pl["uhat"][s], pl["w0"], pl["qm"][s], pl["qc"][s],
                           pl["density_power"])
    for _ in range(args.warmup):
        sim.step(1)
    sim.sync()
    n_before = sum(sim.count(s) for s in range(nsp))
    sim.timing()  # reset counters
    sim.set_timing(True)
    stream = sim.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier(ws)
        torch.cuda.synchronize(device)
        e0.record(stream)
        for _ in range(args.steps):
            sim.step(1)
        e1.record(stream)
        torch.cuda.synchronize(device)
        barrier(ws)
    sim.set_timing(False)
    ms = e0.elapsed_time(e1)
    tim = sim.timing()
    # the pusher alone (grpic_push: steps 1-11 of Sec. 3.1, no deposit), one launch per
    # species after the timed steps, the component the paper times per particle (Sec. 3.5)
    push_ms, push_n = 0.0, 0
    for sp in range(nsp):
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        cnt = sim.count(sp)
        torch.cuda.synchronize(device)
        p0.record(stream)
        sim.push(sp)
        p1.record(stream)
        torch.cuda.synchronize(device)
        push_ms += p0.elapsed_time(p1)
        push_n += cnt
    n_after = sum(sim.count(s) for s in range(nsp))
    psteps_local = 0.5 * (n_before + n_after) * args.steps
    ms_max = allreduce_max(ws, ms, device)
    psteps = allreduce_sum(ws, psteps_local, device)
    value = psteps / (ms_max * 1e-3)

    # the dominant kernel, timed by the library's events around each launch on its stream
    calls = max(tim["push_calls"], 1)
    kernel_ms = tim["kernel_ms"] / calls
    parts_per_launch = 0.5 * (n_before + n_after) / nsp
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs")
    bpp = FP64_BYTES_PER_PARTICLE_STEP if precision == "fp64" else MIXED_BYTES_PER_PARTICLE_STEP
    hbm_achieved = parts_per_launch * bpp / (kernel_ms * 1e-3) / 1e9
    if precision == "fp64":
        refined = args.iter_tol > 0
        ops = parts_per_launch * FP64_PIPE_OPS_PER_PARTICLE_STEP[refined] / (kernel_ms * 1e-3) / 1e9
        roofline = {"bound": "alu", "achieved": ops, "peak": FP64_PIPE_PEAK_GOPS,
                    "unit": "G FP64-pipe op/s", "frac": ops / FP64_PIPE_PEAK_GOPS,
                    "traffic": None,
                    "peak_source": "nominal: 2 FP64 operations/clk/SM x 152 SMs x 2.07 GHz",
                    "tflops": parts_per_launch * FP64_FLOP_PER_PARTICLE_STEP[refined]
                    / (kernel_ms * 1e-3) / 1e12,
                    "kernel": "k_push<deposit> (fused FP64 push + deposit)"}
    else:
        gi = parts_per_launch * MIXED_WARP_INST_PER_PARTICLE / (kernel_ms * 1e-3) / 1e9
        roofline = {"bound": "alu", "achieved": gi, "peak": ISSUE_PEAK_GINST,
                    "unit": "G warp-instructions/s", "frac": gi / ISSUE_PEAK_GINST,
                    "traffic": None,
                    "peak_source": "nominal: 4 warp instructions/clk/SM x 152 SMs x 2.07 GHz",
                    "kernel": "k_push32<deposit> (FP32 push + warp-reduced deposit; the "
                              "guard-zone kernels run beside it on a second stream)"}
    roofline["avg_launch_ms"] = kernel_ms
    if (workload == "wald512" and args.iter_tol == 1e-12 and not photons and not extra
            and not args.ppc):
        roofline["traffic"] = TRAFFIC_BYTES_PER_PARTICLE[precision] * parts_per_launch
        roofline["traffic_source"] = ("ncu dram bytes per particle of the same kernel on this "
                                      "workload, times the particles of one launch")
    hbm = {"achieved_gbs": hbm_achieved, "peak_gbs": hbm_peak or 6800.0,
           "frac": hbm_achieved / (hbm_peak or 6800.0),
           "peak_source": "measured" if hbm_peak else "fallback",
           "bytes_per_particle_step": bpp, "kernel": roofline["kernel"]}
    out = {"value": value, "ms_per_step": ms_max / args.steps, "roofline": roofline,
           "hbm_roofline": hbm,
           "phase_ms_per_step": {k: tim[k] / args.steps for k in
                                 ("predict_ms", "sort_ms", "push_ms", "advance_ms")},
           "gpu_launches": tim["launches"], "clocks": clk.summary(),
           "workload": workload_desc(workload, cfg, nsp * n, precision),
           "particles": nsp * n, "psteps": psteps, "timing": tim, "cfg": cfg,
           "pusher_ns_per_particle": push_ms * 1e6 / max(push_n, 1)}
    return out, sim


# the particle state a step reads: position, momenta, phi, weight, tag (the previous
# position is written by the step's push, Sec. 3.2, so it is not an input)
STATE_ARRAYS = ("i1", "i2", "dx1", "dx2", "u1", "u2", "u3", "phi", "w", "tag")


def end_to_end(args, sim, psteps, ws, device):
    """Through the C ABI with host buffers (grpic_step_host): every step the particle state
    (the arrays the step reads) goes from pinned host memory to the device and comes back
    once its species is pushed, the copies of one species overlapping the work on the
    other."""
    import torch
    host = []
    types = [(k, t) for k, t in sim.ptypes if k in STATE_ARRAYS]
    for s in range(2):
        st = sim.get_particles(s)
        hs = {}
        for k, t in types:
            ht = torch.empty(st[k].shape, dtype=getattr(torch, np.dtype(t).name),
                             pin_memory=True)
            ht.numpy()[:] = st[k]
            hs[k] = ht
        host.append((hs, len(st["i1"])))
    bi = sum(n_s * sum(np.dtype(t).itemsize for _, t in types) for _, n_s in host)
    torch.cuda.synchronize(device)
    barrier(ws)
    t0 = time.perf_counter()
    count = [n_s for _, n_s in host]
    for _ in range(args.steps):
        count = sim.step_host([h for h, _ in host], count)  # returns after the copies back
    t_e2e = time.perf_counter() - t0
    t_e2e = allreduce_max(ws, t_e2e, device)
    return {"value": psteps / t_e2e, "unit": "particle-steps/s", "h2d_bytes_per_step": bi,
            "d2h_bytes_per_step": bi, "api": "grpic_step_host"}


def run_gpu(args, ws, rank, local):
    import torch

    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    precisions = ["fp64", "mixed"] if args.precision == "both" else [args.precision]
    res = {}
    e2e = None
    for prec in precisions:
        out, sim = measure(args, prec, ws, rank, local)
        if prec == precisions[0] and not args.no_e2e:
            e2e = end_to_end(args, sim, out["psteps"], ws, device)
        del sim
        torch.cuda.empty_cache()
        res[prec] = out
    main = res[precisions[0]]

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        ocfg = W.grid_config(args.workload)
        if args.ppc:
            ocfg["ppc"] = args.ppc
        osim = oracle_workload(ocfg, args.cpu_frac)
        times, parts = oracle_steps(osim, args.cpu_steps)
        cpu = {"value": parts / sum(times), "unit": "particle-steps/s", "cores": host_cores(),
               "kind": "oracle",
               "sample": "%d full FP64 PIC steps of the %s workload (%d particles%s), %.1f s" % (
                   args.cpu_steps, args.workload, parts // max(args.cpu_steps, 1),
                   "" if args.cpu_frac >= 1 else ", particles of %.1f%% of the cells"
                   % (100 * args.cpu_frac), sum(times))}
        del osim
    if rank == 0:
        line = {"metric": METRIC, "precision": precisions[0],
                "value": main["value"], "unit": "particle-steps/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": main["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if precisions[0] == "fp64" else "f32 (f64 metric in the guard zones)",
                "data": "synthetic (seeded workload generator)",
                "config": {"workload": main["workload"],
                           "sort_every": args.sort_every, "tile": args.tile,
                           "iter_tol": args.iter_tol,
                           "l2": "inputs larger than L2: particle state %.2f GB" % (
                               main["particles"] * (89 if precisions[0] == "fp64" else 49) / 1e9),
                           "parallelism": "replica per GPU" if ws > 1 else "1 GPU"},
                "roofline": main["roofline"], "hbm_roofline": main["hbm_roofline"],
                "phase_ms_per_step": main["phase_ms_per_step"],
                "pusher_ns_per_particle": main["pusher_ns_per_particle"],
                "gpu_launches": main["gpu_launches"], "e2e": e2e, "cpu_baseline": cpu,
                "clocks": main["clocks"]}
        if args.workload == "bz2048":
            line["paper_context"] = {
                "pusher_ns_per_particle": 6.2, "hardware": "1x A100, precision not stated",
                "workload": "BZ monopole test, 2048^2 log-r mesh, 90 particles per cell "
                            "(Sec. 3.5)"}
        if len(precisions) == 2:
            m = res["mixed"]
            line["mixed"] = {"value": m["value"], "unit": "particle-steps/s",
                             "ms_per_step": m["ms_per_step"],
                             "speedup_vs_fp64": m["value"] / main["value"],
                             "workload": m["workload"], "roofline": m["roofline"],
                             "hbm_roofline": m["hbm_roofline"],
                             "phase_ms_per_step": m["phase_ms_per_step"],
                             "pusher_ns_per_particle": m["pusher_ns_per_particle"],
                             "gpu_launches": m["gpu_launches"], "clocks": m["clocks"],
                             "error_bound": "<= 1e-5 relative per step on particle state vs "
                                            "the FP64 oracle (tests/test_gpu_mixed.py)"}
        print(json.dumps(line), flush=True)


def run_extensions(args, ws, rank, local):
    """The rows beyond the base path, each on the bench's grid: (1) massless particles: one
    species of photons at the electrons' positions and momenta (16,777,216 on wald512,
    gamma without the mass term, no EM push, no deposit), FP64 and mixed, against the e+-
    pairs' push; (2) the current filter: the e+- workload with n_f = 4 passes (the grid
    starts 7.3 cells inside the horizon), its share of the step, and the filter kernel's
    HBM roofline on the 2048^2 grid (8 passes, planes larger than L2). Prints one JSON
    line."""
    import torch

    torch.cuda.set_device(local)
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs") or 6800.0
    out = {"metric": "extensions: massless particles, the current filter, pair injection, "
                     "quasi-spherical grids",
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup}
    parts = set(args.only.split(",")) if args.only else {"photons", "filter512", "filter2048",
                                                          "inject", "qks"}
    ph = {}
    for prec in (("fp64", "mixed") if "photons" in parts else ()):
        pairs, sim = measure(args, prec, ws, rank, local)
        del sim
        phot, sim = measure(args, prec, ws, rank, local, photons=True)
        del sim
        torch.cuda.empty_cache()
        ph[prec] = {"photon_steps_per_s": phot["value"],
                    "pair_particle_steps_per_s": pairs["value"],
                    "push_kernel_ns_per_photon": phot["roofline"]["avg_launch_ms"] * 1e6 /
                    (phot["particles"]),
                    "push_kernel_ns_per_pair_particle": pairs["roofline"]["avg_launch_ms"] * 1e6 /
                    (pairs["particles"] / 2),
                    "photon_hbm_gbs": phot["hbm_roofline"]["achieved_gbs"],
                    "clocks": phot["clocks"], "workload": phot["workload"]}
    if ph:
        out["massless"] = ph
    # the filter on the bench workload: the step with and without it
    if "filter512" in parts:
        base, sim = measure(args, "fp64", ws, rank, local)
        del sim
        filt, sim = measure(args, "fp64", ws, rank, local, extra={"n_filter": 4})
        del sim
        torch.cuda.empty_cache()
        f_ms = filt["timing"]["deposit_ms"] / args.steps
        cfg = filt["cfg"]
        plane = (cfg["n_r"] + 5) * (cfg["n_theta"] + 5) * 8
        out["filter_wald512"] = {
            "n_filter": 4, "step_ms": filt["ms_per_step"],
            "step_ms_without": base["ms_per_step"], "filter_ms_per_step": f_ms,
            "share_of_step": f_ms / filt["ms_per_step"], "algorithmic_bytes_per_step": 6 * plane,
            "note": "3 current planes read and written once per step (one launch runs the 4 "
                    "passes in shared memory); at 512^2 the planes (12.8 MB) stay in L2"}
    if "filter2048" in parts:
        out["filter_wald2048"] = measure_filter_2048(args, ws, rank, local, peaks)
    if "inject" in parts:
        out["inject_bz2048"] = measure_injection(args, local, peaks)
    if "qks" in parts:
        # the bench workload on a quasi-spherical grid (App. A): r0 = 0.4, h0 = 0.45
        q = {}
        for prec in ("fp64", "mixed"):
            base, sim = measure(args, prec, ws, rank, local)
            del sim
            qk, sim = measure(args, prec, ws, rank, local, extra={"r0": 0.4, "h0": 0.45})
            del sim
            torch.cuda.empty_cache()
            q[prec] = {"particle_steps_per_s": qk["value"], "plain_grid": base["value"],
                       "ratio": qk["value"] / base["value"],
                       "push_kernel_ms": qk["roofline"]["avg_launch_ms"],
                       "push_kernel_ms_plain": base["roofline"]["avg_launch_ms"],
                       "clocks": qk["clocks"]}
        out["qks_wald512"] = q
    if rank == 0:
        print(json.dumps(out), flush=True)


def measure_filter_2048(args, ws, rank, local, peaks):
    """The filter kernel against the FP64 pipe and HBM: 2048^2 planes (33.7 MB each, above
    L2), 8 passes in one launch, on the wald2048 grid with args.ext_ppc particles per cell
    per species."""
    import torch

    hbm_peak = peaks.get("hbm_gbs") or 6800.0
    big, sim = measure(args, "fp64", ws, rank, local, workload="wald2048",
                       extra={"n_filter": 8, "ppc": args.ext_ppc or 1})
    del sim
    torch.cuda.empty_cache()
    cfg = big["cfg"]
    plane = (cfg["n_r"] + 5) * (cfg["n_theta"] + 5) * 8
    f_ms = big["timing"]["deposit_ms"] / args.steps
    gbs = 6 * plane / (f_ms * 1e-3) / 1e9
    # FP64 operations the 8 passes need at least: per pass, cell and component one DFMA and
    # one DADD along each of x1 and x2 (the kernel also recomputes its tiles' halos, 1.4x)
    ops = 4 * 8 * 3 * (plane // 8) / (f_ms * 1e-3) / 1e9
    return {
        "n_filter": 8, "filter_ms_per_step": f_ms, "algorithmic_bytes_per_launch": 6 * plane,
        "algorithmic_fp64_ops_per_launch": 4 * 8 * 3 * (plane // 8),
        "roofline": {"bound": "alu", "achieved": ops, "peak": FP64_PIPE_PEAK_GOPS,
                     "unit": "G FP64-pipe op/s", "frac": ops / FP64_PIPE_PEAK_GOPS,
                     "traffic": None,
                     "peak_source": "nominal: 2 FP64 operations/clk/SM x 152 SMs x 2.07 GHz",
                     "kernel": "k_filter<double> (8 passes fused in shared memory)"},
        "hbm_roofline": {"achieved_gbs": gbs, "peak_gbs": hbm_peak, "frac": gbs / hbm_peak,
                         "peak_source": "measured" if peaks.get("hbm_gbs") else "fallback"},
        "clocks": big["clocks"]}


def measure_injection(args, local, peaks):
    """Pair injection (Sec. 4.5) on the 2048^2 monopole grid with 4 particles per cell per
    species (33.6 M particles; args.ext_ppc when given): a full FP64 step followed by
    grpic_inject with sigma_th = 2000, args.steps times after args.warmup; the injection's
    time per call and its share of the step. The density scatter reads 17 B per particle
    (cell indices, weight, tag); the per-cell part reads B (3 planes) and writes about 24 B
    per cell."""
    import torch

    from paper_2511_17701_gb300 import FIELD_MONOPOLE, Sim

    device = torch.device("cuda", local)
    cfg = W.grid_config("bz2048", ppc=args.ext_ppc or 4, sort_every=args.sort_every,
                        tile_r=args.tile, tile_theta=args.tile, iter_tol=args.iter_tol)
    pl = W.pair_plasma(cfg)
    n = pl["pos"]["i1"].size
    nc = cfg["n_r"] * cfg["n_theta"]
    room = (args.warmup + args.steps + 1) * nc  # at most one pair per cell and call
    sim = Sim(cfg, [n + room, n + room], device=device)
    sim.init_metric()
    sim.init_fields(FIELD_MONOPOLE, cfg["B0"])
    for s in range(2):
        sim.load_particles(s, pl["pos"], pl["uhat"][s], pl["w0"], pl["qm"][s], pl["qc"][s],
                           pl["density_power"])
    del pl
    pool = torch.tensor(W.injection_pool(cfg, 1 << 20, seed=cfg["seed"] + 7),
                        dtype=torch.float64, device=device)
    sim.inject(cfg["sigma0"], cfg["sigma_th"], cfg["B0"], pool, pool_offset=0)
    for _ in range(args.warmup):
        sim.step(1)
        sim.inject(cfg["sigma0"], cfg["sigma_th"], cfg["B0"], pool)
    sim.sync()
    sim.diagnostics()
    sim.timing()
    sim.set_timing(True)
    n0 = sim.count(0) + sim.count(1)
    stream = sim.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        sim.step(1)
        sim.inject(cfg["sigma0"], cfg["sigma_th"], cfg["B0"], pool)
    e1.record(stream)
    torch.cuda.synchronize(device)
    sim.set_timing(False)
    ms = e0.elapsed_time(e1) / args.steps
    tim = sim.timing()
    d = sim.diagnostics()
    n1 = sim.count(0) + sim.count(1)
    inj_ms = tim["inject_ms"] / args.steps
    parts = 0.5 * (n0 + n1)
    bytes_ = parts * 17 + nc * (3 * 8 + 24)
    hbm_peak = peaks.get("hbm_gbs") or 6800.0
    gbs = bytes_ / (inj_ms * 1e-3) / 1e9
    del sim
    torch.cuda.empty_cache()
    return {"workload": "bz2048 grid, %d ppc per species, FP64, sigma0 = %g, sigma_th = %g"
                        % (cfg["ppc"], cfg["sigma0"], cfg["sigma_th"]),
            "particles_before": n0, "particles_after": n1, "cells": nc,
            "pairs_added_per_step": d["injected"] / args.steps,
            "inject_ms_per_call": inj_ms, "step_plus_inject_ms": ms,
            "share_of_step": inj_ms / ms,
            "hbm_roofline": {"achieved_gbs": gbs, "peak_gbs": hbm_peak,
                             "frac": gbs / hbm_peak,
                             "algorithmic_bytes_per_call": bytes_}}


def run_adjoint(args, ws, rank, local):
    """The adjoint of the pusher over a frozen field: test particles in the 512^2 Kerr
    (a = 0.9) Wald field, forward n steps with checkpoints, then the reverse sweep for the
    gradient of L = sum(v . final state) with respect to the initial state and B0, both timed
    with CUDA events; central differences of the forward on a sample of particles."""
    import torch

    from paper_2511_17701_gb300 import FIELD_WALD, Sim

    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    cfg = W.grid_config("wald512", r_absorb=1e300)
    n, steps, every = args.adjoint_particles, args.adjoint_steps, args.adjoint_ckpt
    tp = W.probe_particles(cfg, n, 77 + rank, (0.2 * cfg["n_r"], 0.8 * cfg["n_r"]),
                           (0.15 * cfg["n_theta"], 0.85 * cfg["n_theta"]), 0.5)
    qm, qc = W.species_coefficients(1.0)
    sim = Sim(cfg, [n], device=device)
    sim.init_metric()
    sim.init_fields(FIELD_WALD, cfg["B0"])
    sim.load_particles(0, tp["pos"], tp["uhat"], tp["w0"], qm, qc)  # u_i = e_i^j u_j^ on the GPU
    v = sim.species_views(0)
    st0 = torch.stack([v["i1"].double() + v["dx1"], v["i2"].double() + v["dx2"], v["phi"],
                       v["u1"], v["u2"], v["u3"]]).contiguous()
    gen = torch.Generator(device=device).manual_seed(5)
    cot = torch.randn((6, n), dtype=torch.float64, device=device, generator=gen)
    n_iter = 64
    b0 = cfg["B0"]
    stream = sim.stream
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    sim.adjoint_forward(st0[:, :1024].contiguous(), qm, b0, 4, 2, n_iter)  # warm-up
    torch.cuda.synchronize(device)
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        out, ckpt = sim.adjoint_forward(st0, qm, b0, steps, every, n_iter)
        ev[1].record(stream)
        ok = ~torch.isnan(out[0])
        gout = cot * ok
        gin, gpp, gsum = sim.adjoint_backward(ckpt, gout, qm, b0, steps, every, n_iter)
        ev[2].record(stream)
        torch.cuda.synchronize(device)
    fwd_ms, bwd_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    n_ok = int(ok.sum())
    # central differences of the forward on a sample of particles that stayed inside
    idx = torch.nonzero(ok).flatten()[: args.adjoint_fd_sample]
    sub = st0[:, idx].contiguous()
    csub = gout[:, idx]
    h = 1e-6

    def loss(st, b):
        o, _ = sim.adjoint_forward(st, qm, b, steps, every, n_iter)
        return (o * csub).sum(dim=0)

    def central(hh):
        fd = torch.zeros((7, idx.numel()), dtype=torch.float64, device=device)
        for q in range(6):
            sp_, sm_ = sub.clone(), sub.clone()
            sp_[q] += hh
            sm_[q] -= hh
            fd[q] = (loss(sp_, b0) - loss(sm_, b0)) / (2 * hh)
        fd[6] = (loss(sub, b0 + hh) - loss(sub, b0 - hh)) / (2 * hh)
        return fd

    fd_h, fd_h2 = central(h), central(0.5 * h)
    fd_r = (4.0 * fd_h2 - fd_h) / 3.0  # Richardson: the h^2 term of the central difference cancels
    ad = torch.cat([gin[:, idx], gpp[idx][None]])
    good = ~(torch.isnan(fd_h).any(dim=0) | torch.isnan(fd_r).any(dim=0))

    def rel(fd):
        return ((fd - ad).abs().amax(dim=0) / ad.abs().amax(dim=0))[good].cpu().numpy()

    err, err_r = rel(fd_h), rel(fd_r)
    psteps = n_ok * steps
    line = {"metric": "adjoint push: particle-steps/s (frozen field, forward + reverse sweep)",
            "value": psteps / ((fwd_ms + bwd_ms) * 1e-3), "unit": "particle-steps/s",
            "n_gpus": ws, "steps": steps, "warmup": 1, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic (seeded test particles)",
            "config": {"workload": "adjoint: %d test particles (x1 in [0.2, 0.8] n_r, x2 in "
                                   "[0.15, 0.85] n_theta, |u^| uniform in [0, 0.5]) in the frozen "
                                   "Wald field, Kerr a=0.9, B0 as parameter, 512x512 log-r grid "
                                   "r in [0.95 r_h, 50]; %d FP64 steps, checkpoints every %d"
                                   % (n, steps, every)},
            "forward_ms": fwd_ms, "backward_ms": bwd_ms,
            "forward_particle_steps_per_s": n * steps / (fwd_ms * 1e-3),
            "particles_kept": n_ok,
            "dL_dB0": float(gsum.cpu()[0]),
            "fd_check": {"sample": int(good.sum()), "step": h,
                         "median_rel_err": float(np.median(err)) if err.size else None,
                         "p90_rel_err": float(np.quantile(err, 0.9)) if err.size else None,
                         "max_rel_err": float(err.max()) if err.size else None,
                         "frac_within_1e-6": float((err < 1e-6).mean()) if err.size else None,
                         "richardson": {
                             "median_rel_err": float(np.median(err_r)) if err.size else None,
                             "p90_rel_err": float(np.quantile(err_r, 0.9)) if err.size else None,
                             "max_rel_err": float(err_r.max()) if err.size else None,
                             "frac_within_1e-6": float((err_r < 1e-6).mean()) if err.size
                             else None}},
            "gpu_launches": None, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


def bz_diagnostics(sim, cfg, radii):
    """The closed-form quantities of Sec. 4.5 from one snapshot of the em planes: per radius,
    the field-line angular velocity Omega = -E_theta / (sqrt(h) B^r) averaged over theta in
    [pi/6, 5 pi/6] with weight sin^2(theta) (BZ: omega_h / 2 at every latitude to O(a^2)), the
    amplitude of H_phi fitted to sin^2(theta) by least squares (BZ: -B0 a / 8), and the
    Poynting flux L = 2 pi int P^r sqrt(h) dtheta = (1/2) int (E_theta H_phi - E_phi H_theta)
    dtheta. In the code coordinates E_theta dtheta = E_2 dx2 and H_phi = H_3, so L is half the
    sum over rows of E_2 H_3 - E_3 H_2; E_2, B^1 at (i, j + 1/2), H_3 at (i + 1/2, j + 1/2)
    and H_2 at (i + 1/2, j) are averaged to column i. sqrt(h) is the Kerr-Schild volume
    element sin(theta) Sigma sqrt(1 + 2 r / Sigma) times dr/dx1 dtheta/dx2."""
    F = sim.planes()
    E, H = sim.aux_fields()
    a, nr, nt, G = cfg["a"], cfg["n_r"], cfg["n_theta"], 2
    dxi = math.log(cfg["r_max"] / cfg["r_min"]) / nr
    dth = math.pi / nt
    thc = (np.arange(nt) + 0.5) * dth
    out = {}
    for rr in radii:
        i = int(round(math.log(rr / cfg["r_min"]) / dxi))
        r = cfg["r_min"] * math.exp(i * dxi)
        sig = r * r + a * a * np.cos(thc) ** 2
        sq = dxi * r * dth * sig * np.sin(thc) * np.sqrt(1.0 + 2.0 * r / sig)
        om = -E[1][G:G + nt, G + i] / (sq * F[0][G:G + nt, G + i])
        mid = (thc > math.pi / 6) & (thc < 5 * math.pi / 6)
        w = np.sin(thc[mid]) ** 2
        h3 = 0.5 * (H[2][G:G + nt, G + i - 1] + H[2][G:G + nt, G + i])
        s2 = np.sin(thc) ** 2
        h2 = 0.5 * (H[1][G:G + nt + 1, G + i - 1] + H[1][G:G + nt + 1, G + i])
        wn = np.ones(nt + 1)
        wn[0] = wn[-1] = 0.5
        out[rr] = {"omega": float(np.sum(w * om[mid]) / np.sum(w)),
                   "hphi_amp": float(np.sum(h3 * s2) / np.sum(s2 * s2)),
                   "L": float(0.5 * (np.sum(E[1][G:G + nt, G + i] * h3) -
                                     np.sum(wn * E[2][G:G + nt + 1, G + i] * h2)))}
    return out


def run_bz_physics(args, local):
    """The BZ monopole test of Sec. 4.5: the monopole A_phi = -B0 cos(theta) on the Kerr (a =
    0.2) log-r grid r in [1, 10] with its absorbing layer, a thin e+- plasma (density ~ r^-2)
    and pair injection where sigma > sigma_th = 2000 after every step, run to args.bz_time
    r_g; then Omega / omega_h (BZ: 1/2), H_phi / (-B0 a / 8) (BZ: 1) and L / L_BZ, L_BZ =
    B0^2 omega_h^2 / 6 (BZ: 1), each averaged over snapshots every r_g in the last third of
    the run. omega_h = a / (2 r_h) = -g_03 / g_33 at the horizon (M = 1)."""
    import torch

    from paper_2511_17701_gb300 import FIELD_MONOPOLE, Sim

    device = torch.device("cuda", local)
    n_g = args.bz_n
    prec = args.bz_precision
    cfg = W.grid_config("bz1024", n_r=n_g, n_theta=n_g, ppc=2, sort_every=args.sort_every,
                        tile_r=args.tile, tile_theta=args.tile, precision=prec,
                        iter_tol=args.iter_tol if prec == "fp64" else 0.0)
    a, B0 = cfg["a"], cfg["B0"]
    rh = 1.0 + math.sqrt(1.0 - a * a)
    wh = a / (2.0 * rh)
    LBZ = B0 * B0 * wh * wh / 6.0
    pl = W.pair_plasma(cfg)
    n = pl["pos"]["i1"].size
    cap = n + 48 * n_g * n_g
    sim = Sim(cfg, [cap, cap], device=device)
    sim.init_metric()
    sim.init_fields(FIELD_MONOPOLE, B0)
    for sp in range(2):
        sim.load_particles(sp, pl["pos"], pl["uhat"][sp], pl["w0"], pl["qm"][sp], pl["qc"][sp],
                           pl["density_power"])
    del pl
    pool = torch.tensor(W.injection_pool(cfg, 1 << 22, seed=cfg["seed"] + 7),
                        dtype=torch.float64, device=device)
    radii = (2.0, 3.0, 5.0, 8.0)
    dt = sim.dt
    t0 = time.perf_counter()
    sim.inject(cfg["sigma0"], cfg["sigma_th"], B0, pool, pool_offset=0)
    t, snaps = 0.0, []
    n_mark = int(math.floor(args.bz_time))
    for mark in range(1, n_mark + 1):
        k = int(round((mark - t) / dt))
        for _ in range(k):
            sim.step(1)
            sim.inject(cfg["sigma0"], cfg["sigma_th"], B0, pool)
        t += k * dt
        if mark > 2 * n_mark / 3:
            snaps.append(bz_diagnostics(sim, cfg, radii))
            sn = snaps[-1]
            print(json.dumps({"t": t, "omega_over_omega_h": {str(r): sn[r]["omega"] / wh
                                                             for r in radii},
                              "hphi_over_bz": {str(r): sn[r]["hphi_amp"] / (-B0 * a / 8.0)
                                               for r in radii},
                              "L_over_LBZ": {str(r): sn[r]["L"] / LBZ for r in radii}}),
                  file=sys.stderr, flush=True)
    sim.sync()
    wall = time.perf_counter() - t0
    d = sim.diagnostics()

    def avg(key, norm):
        return {str(rr): float(np.mean([sn[rr][key] for sn in snaps]) / norm) for rr in radii}

    def spread(key, norm):
        return {str(rr): float(np.std([sn[rr][key] for sn in snaps]) / abs(norm)) for rr in radii}

    line = {"metric": "BZ monopole closed-form checks (Sec. 4.5)", "n_gpus": 1,
            "precision": prec, "data": "synthetic (seeded workload generator)",
            "config": {"workload": "bz monopole, Kerr a=%.1f, %dx%d log-r grid, r in [1, 10], "
                                   "absorbing layer from r=9, rho0=5e-5, d0=2.5e-3, sigma0=2500, "
                                   "sigma_th=2000, initial e+- 2 per cell per species, density "
                                   "~ r^-2" % (a, n_g, n_g),
                       "t_end_rg": t, "dt": dt, "average_over_rg": [t - len(snaps), t],
                       "omega_h": wh, "L_BZ": LBZ},
            "omega_over_omega_h": avg("omega", wh), "omega_spread": spread("omega", wh),
            "hphi_over_bz": avg("hphi_amp", -B0 * a / 8.0),
            "hphi_spread": spread("hphi_amp", -B0 * a / 8.0),
            "L_over_LBZ": avg("L", LBZ), "L_spread": spread("L", LBZ),
            "expected": {"omega_over_omega_h": 0.5, "hphi_over_bz": 1.0, "L_over_LBZ": 1.0},
            "particles": [sim.count(0), sim.count(1)], "injected": d["injected"],
            "inject_dropped": d["inject_dropped"], "nonfinite": d["nonfinite"],
            "wall_s": wall}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="wald512", choices=sorted(W.CONFIGS))
    ap.add_argument("--sort-every", type=int, default=10)
    ap.add_argument("--tile", type=int, default=16)
    ap.add_argument("--precision", default="both", choices=["fp64", "mixed", "both"],
                    help="both: FP64 (the line's value) and then mixed on the same workload")
    ap.add_argument("--ppc", type=int, default=0, help="override particles per cell per species "
                    "(a smaller case of the same workload, e.g. for profiling)")
    ap.add_argument("--cpu-frac", type=float, default=1.0,
                    help="fraction of the cells whose particles the CPU baseline pushes")
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--ref-frac", type=float, default=0.25,
                    help="fraction of the cells whose particles the reference arm pushes")
    ap.add_argument("--adjoint", action="store_true",
                    help="time the adjoint of the pusher over a frozen field instead")
    ap.add_argument("--extensions", action="store_true",
                    help="time the rows beyond the base path instead: massless particles and "
                         "the current filter")
    ap.add_argument("--only", default="",
                    help="--extensions: a comma list of photons, filter512, filter2048, inject, "
                         "qks")
    ap.add_argument("--ext-ppc", type=int, default=0,
                    help="--extensions: particles per cell per species of the 2048^2 filter "
                         "and injection cases (default 1 and 4)")
    ap.add_argument("--adjoint-particles", type=int, default=1 << 20)
    ap.add_argument("--adjoint-steps", type=int, default=2000)
    ap.add_argument("--adjoint-ckpt", type=int, default=100)
    ap.add_argument("--adjoint-fd-sample", type=int, default=256)
    ap.add_argument("--iter-tol", type=float, default=1e-12,
                    help="implicit pushes: FP64 iterations from an FP32 predictor to this "
                         "tolerance (0: exact-repeat stop, bit-identical to n_iter iterations)")
    ap.add_argument("--tiled-push", action="store_true",
                    help="mixed path: the shared-memory tiled FP32 kernel instead of the default "
                         "one thread per particle")
    ap.add_argument("--bz-physics", action="store_true",
                    help="run the BZ monopole test of Sec. 4.5 and report its closed-form checks")
    ap.add_argument("--bz-n", type=int, default=512, help="--bz-physics: cells per direction")
    ap.add_argument("--bz-time", type=float, default=60.0, help="--bz-physics: run time, r_g")
    ap.add_argument("--bz-precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    ws, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.adjoint:
        run_adjoint(args, ws, rank, local)
    elif args.extensions:
        run_extensions(args, ws, rank, local)
    elif args.bz_physics:
        if rank == 0:
            run_bz_physics(args, local)
    else:
        run_gpu(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
