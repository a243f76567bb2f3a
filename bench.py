"""Throughput of the GR PIC hot path (push + deposit + field update) on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                [--workload wald512] [--sort-every 10]

A step is one full PIC step (Sec. 3.4 of arXiv:2511.17701) over the whole workload:
field predict, (sort), fused push + deposit of both species, field advance. The default
workload is the 512^2 Kerr (a = 0.9) Wald configuration with 32 particles per cell per
species (16,777,216 particles), FP64, synthetic and seeded. Prints one JSON line.

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

# Algorithmic bytes of one particle-step of the fused FP64 push + deposit kernel
# (SoA, read: i1, i2, dx1, dx2, u1, u2, u3, phi, w, tag; write: the same minus w plus the
# previous position i1p, i2p, dx1p, dx2p): 4+4+8+8+24+8+8+1 = 65 B read,
# 4+4+8+8+24+8+1 + 4+4+8+8 = 81 B written.
BYTES_PER_PARTICLE_STEP = 65 + 81
# FP64 operations per particle-step of the same kernel, counted by ncu on this kernel
# (2 x dfma + dmul + dadd instructions executed / particles); see profiles/.
FP64_FLOP_PER_PARTICLE_STEP = 3806
FP64_PEAK_TFLOPS = 1.25  # GB300 nominal FP64 (2 DFMA / clk / SM x 152 SMs x 2.07 GHz)


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
        import torch.distributed as dist
        dist.init_process_group("nccl")
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


def workload_desc(name, cfg, n_total, precision="fp64"):
    return ("%s: Kerr a=%g Wald B0=%g, %dx%d log-r grid, r in [0.95 r_h, %g], e+- pairs %d "
            "per cell per species (%d particles), Maxwell-Juttner theta_T=%g, density ~ r^-%g, "
            "%s" % (name, cfg["a"], cfg["B0"], cfg["n_r"], cfg["n_theta"], cfg["r_max"],
                    cfg["ppc"], n_total, cfg["theta_T"], cfg.get("density_power", 0.0),
                    PRECISION_DESC[precision]))


def oracle_workload(cfg, frac, seed=99):
    """The oracle holding the workload's grid and, when frac < 1, the particles of a
    seeded random fraction of the cells (a bounded sample)."""
    from oracle import oracle as O
    cells = None
    if frac < 1.0:
        cells = W.random_cells(cfg, max(1, int(cfg["n_r"] * cfg["n_theta"] * frac)), seed)
    osim = O.OracleSim(cfg)
    osim.init_fields(O.FIELD_WALD, cfg["B0"])
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
    line = {"metric": "particle-steps/s (push+deposit+field), FP64", "value": value,
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


def run_gpu(args, ws, rank, local):
    import torch

    from paper_2511_17701_gb300 import FIELD_WALD, Sim

    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    cfg = W.grid_config(args.workload, sort_every=args.sort_every, tile_r=args.tile,
                        tile_theta=args.tile, precision=args.precision)
    if args.ppc:
        cfg["ppc"] = args.ppc
    pl = W.pair_plasma(cfg, seed=cfg["seed"] + 1000 * rank)
    n = pl["pos"]["i1"].size
    sim = Sim(cfg, [n, n], device=device)
    sim.init_metric()
    sim.init_fields(FIELD_WALD, cfg["B0"])
    for s in range(2):
        sim.load_particles(s, pl["pos"], pl["uhat"][s], pl["w0"], pl["qm"][s], pl["qc"][s],
                           pl["density_power"])
    del pl
    for _ in range(args.warmup):
        sim.step(1)
    sim.sync()
    n_before = sum(sim.count(s) for s in range(2))
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
    n_after = sum(sim.count(s) for s in range(2))
    psteps_local = 0.5 * (n_before + n_after) * args.steps
    ms_max = allreduce_max(ws, ms, device)
    psteps = allreduce_sum(ws, psteps_local, device)
    value = psteps / (ms_max * 1e-3)

    # dominant kernel: fused FP64 push + deposit, average launch time from events
    push_ms = tim["push_ms"] / max(tim["push_calls"], 1)
    parts_per_launch = 0.5 * (n_before + n_after) / 2
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs")
    bytes_launch = parts_per_launch * BYTES_PER_PARTICLE_STEP
    hbm_achieved = bytes_launch / (push_ms * 1e-3) / 1e9
    if FP64_FLOP_PER_PARTICLE_STEP:
        fl = parts_per_launch * FP64_FLOP_PER_PARTICLE_STEP / (push_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": fl, "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": fl / FP64_PEAK_TFLOPS, "traffic": None,
                    "peak_source": "nominal FP64 rate from unit counts and clocks"}
    else:
        roofline = {"bound": "hbm", "achieved": hbm_achieved,
                    "peak": hbm_peak or 6800.0, "unit": "GB/s",
                    "frac": hbm_achieved / (hbm_peak or 6800.0), "traffic": None,
                    "peak_source": "measured" if hbm_peak else "fallback"}
    roofline["kernel"] = "k_push<deposit> (fused FP64 push + deposit)"
    roofline["avg_launch_ms"] = push_ms
    hbm = {"achieved_gbs": hbm_achieved, "peak_gbs": hbm_peak,
           "frac": hbm_achieved / hbm_peak if hbm_peak else None,
           "bytes_per_particle_step": BYTES_PER_PARTICLE_STEP}

    # end to end through the C ABI with host buffers: per step the particle state goes
    # from pinned host memory to the device, one step runs, and the state comes back
    e2e = None
    if not args.no_e2e:
        host = []
        for s in range(2):
            st = sim.get_particles(s)
            hs = {}
            for k, t in sim.ptypes:
                ht = torch.empty(st[k].shape, dtype=getattr(torch, np.dtype(t).name),
                                 pin_memory=True)
                ht.numpy()[:] = st[k]
                hs[k] = ht
            host.append((hs, len(st["i1"])))
        bi = sum(n_s * sum(np.dtype(t).itemsize for _, t in sim.ptypes) for _, n_s in host)
        torch.cuda.synchronize(device)
        barrier(ws)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for s in range(2):
                sim.set_particles(s, host[s][0], sim.qm[s], sim.qc[s])
            sim.step(1)
            for s in range(2):
                v = sim.species_views(s)
                for k, _ in sim.ptypes:
                    host[s][0][k][: v[k].numel()].copy_(v[k], non_blocking=True)
            torch.cuda.synchronize(device)
        t_e2e = time.perf_counter() - t0
        t_e2e = allreduce_max(ws, t_e2e, device)
        e2e = {"value": psteps / t_e2e, "unit": "particle-steps/s", "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bi}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        ocfg = W.grid_config(args.workload)
        if args.ppc:
            ocfg["ppc"] = args.ppc
        osim = oracle_workload(ocfg, args.cpu_frac)
        times, parts = oracle_steps(osim, args.cpu_steps)
        cpu = {"value": parts / sum(times), "unit": "particle-steps/s", "cores": host_cores(),
               "kind": "oracle",
               "sample": "%d full PIC steps of the %s workload (%d particles%s), %.1f s" % (
                   args.cpu_steps, args.workload, parts // max(args.cpu_steps, 1),
                   "" if args.cpu_frac >= 1 else ", particles of %.1f%% of the cells"
                   % (100 * args.cpu_frac), sum(times))}
        del osim
    if rank == 0:
        line = {"metric": "particle-steps/s (push+deposit+field), FP64",
                "precision": args.precision,
                "value": value, "unit": "particle-steps/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.precision == "fp64" else "f32 (f64 within the guard cells)",
                "data": "synthetic (seeded workload generator)",
                "config": {"workload": workload_desc(args.workload, cfg, 2 * n, args.precision),
                           "sort_every": args.sort_every, "tile": args.tile,
                           "l2": "inputs larger than L2: particle state %.2f GB" % (
                               2 * n * 89 / 1e9),
                           "parallelism": "replica per GPU" if ws > 1 else "1 GPU"},
                "roofline": roofline, "hbm_roofline": hbm,
                "phase_ms_per_step": {k: tim[k] / args.steps for k in
                                      ("predict_ms", "sort_ms", "push_ms", "advance_ms")},
                "gpu_launches": tim["launches"], "e2e": e2e, "cpu_baseline": cpu,
                "clocks": clk.summary()}
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
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--ppc", type=int, default=0, help="override particles per cell per species "
                    "(a smaller case of the same workload, e.g. for profiling)")
    ap.add_argument("--cpu-frac", type=float, default=1.0,
                    help="fraction of the cells whose particles the CPU baseline pushes")
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--ref-frac", type=float, default=0.25,
                    help="fraction of the cells whose particles the reference arm pushes")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    ws, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_gpu(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
