"""Throughput of the GR PIC hot path (push + deposit + field update) on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                [--workload wald2048] [--precision both|fp64|mixed] [--sort-every 10]

A step is one full PIC step (Sec. 3.4 of arXiv:2511.17701) over the whole workload: field
predict, (sort), fused push + deposit of both species, field advance. The default workload
is the 2048^2 Kerr (a = 0.9) Wald configuration: r in [0.95 r_h, 200], 16 particles per cell
per species (134,217,728 particles), density ~ 1/r, Maxwell-Juttner theta_T = 1, synthetic
and seeded. It is timed in FP64 (the line's value, with the end-to-end leg through the C ABI
and the CPU oracle beside it) and then in mixed precision on the same workload (the "mixed"
object, with its per-step error against the FP64 path and the invariant drift of both
precisions). The rooflines divide by peaks measured in the same run: the FP64 and FP32 FMA
rates of the library's probe kernel, and the HBM copy bandwidth of MEASURED_PEAKS.json.
Prints one JSON line.

--impl reference times the CPU oracle (FP64, OpenMP over particles) on the host cores on a
bounded sample of the same workload.
Under torchrun with N > 1 every rank runs an independent replica of the workload on its
own GPU (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
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

# Algorithmic bytes of one particle-step of the dominant kernel of each precision, as the
# bench runs it (the fused push + deposit stores no previous positions):
# FP64 k_push<deposit> reads i1, i2, dx1, dx2, u1, u2, u3, phi, w, tag (4+4+8+8+24+8+8+1 =
# 65 B) and writes all of them but w (57 B): 122 B.
FP64_BYTES_PER_PARTICLE_STEP = 65 + 57
# Mixed k_push32<deposit>: FP32 offsets, momenta, phi and w and the guard bitmask read
# (4+4+4+4+12+4+4+1 + 1/8 = 37 B), the same but w and the mask written (33 B): 70 B.
MIXED_BYTES_PER_PARTICLE_STEP = 37 + 33
# The grid's share of a step: em (6 planes), em0 (6), cur0 (3) and cur (3) read, em, em0 and
# cur0 written: 33 plane elements per cell (264 B in FP64, 132 B in FP32), per particle the
# cell's share 264 / (particles per cell).
GRID_BYTES_PER_CELL = {"fp64": 33 * 8, "mixed": 33 * 4}

# Executed work and DRAM traffic per particle of the dominant kernels, from ncu captures of
# the kernel sources whose digest is `src` (profiles/): FP64-pipe operations (DFMA + DMUL +
# DADD thread instructions) of k_push<deposit>, warp instructions of k_push32<deposit>, and
# dram__bytes_read.sum + dram__bytes_write.sum per particle. When the sources change the
# counts are reported as stale and the traffic as null until they are captured again.
KERNEL_COUNTS = {
    "fp64": {"src": "396195e5c4b7c291",
             "workload": "wald2048; operations from ncu --set full of one launch at 1 particle "
                         "per cell per species (4,194,304 particles), DRAM bytes from a one-pass "
                         "capture of a full launch (67,108,864 particles)",
             "fp64_ops": 198.63 + 269.56 + 94.10, "flop": 2 * 198.63 + 269.56 + 94.10,
             "dram_bytes": (4712624896 + 3813730816) / 67108864},
    "mixed": {"src": "396195e5c4b7c291",
              "workload": "wald2048; warp instructions from ncu --set full of one launch at 1 "
                          "particle per cell per species, DRAM bytes from a one-pass capture of a "
                          "full launch (67,108,864 particles)",
              "warp_inst": 168257970 / 4194304,
              "dram_bytes": (2653071872 + 2371053056) / 67108864},
}
KERNEL_SOURCES = ("particles.cu", "pusher.cuh", "dfloat.cuh", "grpic_internal.cuh")


def kernel_src_digest() -> str:
    """sha256 (first 16 hex digits) of the sources that define the push kernels."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2511_17701_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def hbm_peak():
    """(GB/s, source): the measured copy bandwidth, else the stated fallback."""
    p = measured_peaks().get("hbm_gbs")
    if p:
        return float(p), "measured (MEASURED_PEAKS.json: device copy on this pool's GB300s)"
    return 6800.0, "fallback (6.8 TB/s, one earlier GB300 measurement; no MEASURED_PEAKS.json)"


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
            if len(p) >= 9:
                rows.append(p)
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


# ---------------------------------------------------------------------------------------
# The CPU oracle (cpu_baseline and the reference arm only)
# ---------------------------------------------------------------------------------------
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


def oracle_phases(osim, threads):
    """One oracle PIC step in its phases, timed: (field seconds: predict + advance,
    particle seconds: both pushes + the deposit, particles pushed)."""
    from oracle import oracle as O
    O.set_threads(threads)
    n = sum(s.n for s in osim.species)
    t0 = time.perf_counter()
    osim.predict()
    t1 = time.perf_counter()
    for s in range(len(osim.species)):
        osim.push(s)
    osim.deposit()
    t2 = time.perf_counter()
    osim.advance()
    t3 = time.perf_counter()
    return (t1 - t0) + (t3 - t2), t2 - t1, n


def host_cores():
    from oracle import oracle as O
    return O.max_threads()


def projected_rate(n_total, t_field, t_part, n_sample):
    """Particle-steps/s of a full-workload step from a step on the whole grid with a sample
    of the particles: the particle phases scale with the particles, the field phases do not."""
    return n_total / (t_field + t_part * n_total / n_sample)


def cpu_baseline(args):
    """The oracle as it stands on the host cores: --cpu-steps full steps on the workload's
    whole grid with the particles of a seeded fraction of the cells (all cores), then the
    particle phases of --cpu-steps-1core more steps on one core; the particle phases projected
    to the full workload (no projection at --cpu-frac 1)."""
    cfg = W.grid_config(args.workload)
    if args.ppc:
        cfg["ppc"] = args.ppc
    n_total = 2 * cfg["n_r"] * cfg["n_theta"] * cfg["ppc"]
    t_set = time.perf_counter()
    osim = oracle_workload(cfg, args.cpu_frac)
    setup = time.perf_counter() - t_set
    cores = host_cores()
    tf = tp = 0.0
    n_s = 0
    for _ in range(args.cpu_steps):
        f, p, n_s = oracle_phases(osim, cores)
        tf += f
        tp += p
    tf /= args.cpu_steps
    tp /= args.cpu_steps
    all_core = projected_rate(n_total, tf, tp, n_s)
    from oracle import oracle as O
    O.set_threads(1)
    t0 = time.perf_counter()
    for _ in range(args.cpu_steps_1core):
        for s in range(len(osim.species)):
            osim.push(s)
        osim.deposit()
    tp1 = (time.perf_counter() - t0) / args.cpu_steps_1core
    O.set_threads(cores)
    one_core = projected_rate(n_total, tf, tp1, n_s)
    if n_s == n_total:
        who = "all %d particles of the workload (no projection)" % n_total
    else:
        who = ("the particles of %.1f%% of the cells (%d particles, seeded); particle phases "
               "scaled to the %d particles of the workload" % (100 * args.cpu_frac, n_s, n_total))
    sample = ("%s: the full %dx%d grid (field predict + advance, which the oracle runs on one "
              "core, %.2f s per step) with %s: %d full steps on %d cores (push + deposit %.2f s "
              "per step), then the particle phases of %d more step(s) on 1 core (%.2f s per "
              "step); set-up %.0f s"
              % (args.workload, cfg["n_r"], cfg["n_theta"], tf, who, args.cpu_steps, cores, tp,
                 args.cpu_steps_1core, tp1, setup))
    return {"value": all_core, "unit": "particle-steps/s", "cores": cores, "kind": "oracle",
            "sample": sample, "one_core": {"value": one_core, "cores": 1},
            "field_s_per_step": tf, "particle_s_per_sample_step": tp,
            "particle_s_per_sample_step_1core": tp1, "sample_particles": n_s}


def run_reference(args, ws, rank):
    """The reference arm: the oracle timed on the host cores. Each step runs the particle
    phases (push of both species + deposit) on a bounded sample of the workload's particles;
    the field phases on the whole grid (one core in the oracle, several seconds at 2048^2)
    are timed on the first timed step and charged to every step."""
    if rank != 0:
        return
    cfg = W.grid_config(args.workload)
    frac = args.ref_frac
    n_total = 2 * cfg["n_r"] * cfg["n_theta"] * cfg["ppc"]
    osim = oracle_workload(cfg, frac)
    cores = host_cores()
    n = sum(s.n for s in osim.species)

    def particles_only():
        t0 = time.perf_counter()
        for s in range(len(osim.species)):
            osim.push(s)
        osim.deposit()
        return time.perf_counter() - t0

    for _ in range(args.warmup):
        particles_only()
    tf, tp0, n = oracle_phases(osim, cores)
    tps = [tp0] + [particles_only() for _ in range(args.steps - 1)]
    step_s = [tf + t * n_total / n for t in tps]
    value = n_total * len(step_s) / sum(step_s)
    line = {"metric": METRIC, "value": value,
            "unit": "particle-steps/s", "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(step_s)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_desc(args.workload, cfg, n_total)},
            "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": cores,
                             "kind": "oracle",
                             "sample": "full %dx%d grid (field phases timed once, %.2f s, "
                                       "charged to every step) with the particles of %.1f%% "
                                       "of the cells (%d particles, push + deposit timed "
                                       "every step, scaled to %d particles); %d warm-up + %d "
                                       "timed steps" % (cfg["n_r"], cfg["n_theta"], tf,
                                                         100 * frac, n, n_total, args.warmup,
                                                         args.steps)},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------
# GPU measurements
# ---------------------------------------------------------------------------------------
def device_facts(device):
    import torch
    p = torch.cuda.get_device_properties(device)
    return {"name": p.name, "sms": int(p.multi_processor_count)}


def measure_alu_peaks(device, launches=5):
    """Throughput of the library's probe kernel (grpic_probe_alu), timed with CUDA events on
    the current stream: FP64 fused multiply-add, multiply and add (thread operations/s; the
    FP64 pipe's peak is the fastest of them, the rate the FP64 kernel's DFMA/DMUL/DADD mixture
    is measured against) and FP32 fused multiply-add as warp instructions/s (the issue peak).
    Each launch runs ~0.1 s; the median of `launches` launches after one warm-up."""
    import torch

    from paper_2511_17701_gb300.binding import probe_alu
    stream = torch.cuda.current_stream(device)
    sink = torch.zeros(1, dtype=torch.float64, device=device)
    sms = device_facts(device)["sms"]
    out = {}
    for prec, op, iters in (("fp64", "fma", 800), ("fp64", "mul", 800), ("fp64", "add", 800),
                            ("fp32", "fma", 50000)):
        iters = max(1, int(iters * 152 / sms))
        probe_alu(prec, op, iters, 8, sink, stream)
        rates = []
        for _ in range(launches):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ops = probe_alu(prec, op, iters, 8, sink, stream)
            e1.record(stream)
            e1.synchronize()
            rates.append(ops / (e0.elapsed_time(e1) * 1e-3))
        out[prec + "_" + op] = float(np.median(rates)) / 1e9
    fp64 = {k: out["fp64_" + k] for k in ("fma", "mul", "add")}
    return {"fp64_gops": max(fp64.values()), "fp64_by_op_gops": fp64,
            "warp_ginst": out["fp32_fma"] / 32, "fp32_gops": out["fp32_fma"], "sms": sms}


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
                        tiled_push=args.tiled_push, iter_tol=args.iter_tol)
    if args.ppc and workload == args.workload:
        cfg["ppc"] = args.ppc
    cfg.update(extra or {})
    # the seeded plasma of a workload is drawn once per process (the two precisions and the
    # photon run share it: drawing 134 M particles takes most of a minute)
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
    # nothing reads the previous positions inside the timed steps: the fused push skips them
    sim.set_keep_prev(False)
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
    ppc_total = nsp * cfg["ppc"]
    out = {"value": value, "ms_per_step": ms_max / args.steps, "kernel_ms": kernel_ms,
           "parts_per_launch": parts_per_launch, "ppc_total": ppc_total,
           "phase_ms_per_step": {k: tim[k] / args.steps for k in
                                 ("predict_ms", "sort_ms", "push_ms", "advance_ms")},
           "gpu_launches": tim["launches"], "clocks": clk.summary(),
           "workload": workload_desc(workload, cfg, nsp * n, precision),
           "particles": nsp * n, "psteps": psteps, "timing": tim, "cfg": cfg,
           "pusher_ns_per_particle": push_ms * 1e6 / max(push_n, 1)}
    return out, sim


def rooflines(out, precision, alu, args, photons=False):
    """roofline (the bound that applies to the dominant kernel, against the peak measured in
    this run), hbm_roofline (the dominant kernel's algorithmic bytes against the HBM peak)
    and hbm_roofline_step (the whole step's algorithmic bytes per particle-step, grid
    included, at the line's particle-steps/s)."""
    kc = KERNEL_COUNTS[precision]
    fresh = kc["src"] == kernel_src_digest() and not photons
    kms, parts = out["kernel_ms"], out["parts_per_launch"]
    sms = alu.get("sms")
    mhz = out["clocks"].get("sm_mhz")
    if precision == "fp64":
        ach = parts * kc["fp64_ops"] / (kms * 1e-3) / 1e9
        peak = alu.get("fp64_gops")
        roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "G FP64-pipe op/s",
                "frac": ach / peak if peak else None,
                "peak_source": "measured in this run: grpic_probe_alu FP64, the fastest of "
                               "DFMA, DMUL and DADD chains (8 per thread, %d SMs x 8 blocks of "
                               "256 threads)" % sms,
                "nominal_peak_at_sampled_clock": 2 * sms * mhz / 1e3 if (sms and mhz) else None,
                "ops_per_particle": kc["fp64_ops"],
                "tflops": parts * kc["flop"] / (kms * 1e-3) / 1e12,
                "kernel": "k_push<deposit> (fused FP64 push + deposit)"}
        bpp = FP64_BYTES_PER_PARTICLE_STEP
    else:
        ach = parts * kc["warp_inst"] / (kms * 1e-3) / 1e9
        peak = alu.get("warp_ginst")
        roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "G warp-instructions/s",
                "frac": ach / peak if peak else None,
                "peak_source": "measured in this run: grpic_probe_alu FP32 (one warp FMA "
                               "instruction per clock per SM sub-partition), / 32 lanes",
                "nominal_peak_at_sampled_clock": 4 * sms * mhz / 1e3 if (sms and mhz) else None,
                "warp_inst_per_particle": kc["warp_inst"],
                "kernel": "k_push32<deposit> (FP32 push + warp-reduced deposit; the "
                          "guard-zone kernels run beside it on a second stream)"}
        bpp = MIXED_BYTES_PER_PARTICLE_STEP
    roof["avg_launch_ms"] = kms
    roof["traffic"] = kc["dram_bytes"] * parts if (fresh and kc["dram_bytes"]) else None
    roof["counts"] = ("ncu, kernel sources %s (%s)" % (kc["src"], kc["workload"]) if fresh else
                      "stale: ncu counts of kernel sources %s, now %s"
                      % (kc["src"] or "-", kernel_src_digest()))
    hp, hsrc = hbm_peak()
    gbs = parts * bpp / (kms * 1e-3) / 1e9
    hbm = {"achieved_gbs": gbs, "peak_gbs": hp, "frac": gbs / hp, "peak_source": hsrc,
           "bytes_per_particle_step": bpp, "kernel": roof["kernel"]}
    step_bpp = bpp + GRID_BYTES_PER_CELL[precision] / out["ppc_total"]
    sgbs = out["value"] * step_bpp / 1e9
    step = {"achieved_gbs": sgbs, "peak_gbs": hp, "frac": sgbs / hp,
            "bytes_per_particle_step": step_bpp,
            "bytes": "%d B per particle (dominant kernel) + %d B per cell / %d particles per "
                     "cell (field planes)" % (bpp, GRID_BYTES_PER_CELL[precision],
                                              out["ppc_total"]),
            "timed": "the line's particle-steps/s over the whole timed step"}
    return roof, hbm, step


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
        del st
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


def mixed_step_error(sim64, sim32):
    """Per-result error of one mixed-precision step against the FP64 path from the same
    state: the mixed context's particles and planes after its timed steps are copied, widened,
    into the FP64 context; both run predict, the push of each species, the deposit and the
    advance; then per quantity the largest difference over all particles (positions x = i +
    dx relative to max(1, |x|), momenta relative to |u_c| + median |u_c|, phi relative to
    max(1, |phi|)) and per field plane the normwise difference. The FP64 path matches the
    oracle to 1e-12 per step (tests), so these are the errors against the FP64 oracle to that
    level."""
    import torch

    from paper_2511_17701_gb300 import NPLANES
    for s in range(2):
        v = sim32.species_views(s)
        arrays = {k: (t.double() if t.dtype == torch.float32 else t.clone())
                  for k, t in v.items()}
        sim64.set_particles(s, arrays, sim32.qm[s], sim32.qc[s])
        del arrays
    for k in range(NPLANES):
        sim64.plane(k).copy_(sim32.plane(k))
    for sim in (sim64, sim32):
        sim.set_keep_prev(True)
        sim.predict()
        for s in range(2):
            sim.push(s)
        sim.deposit()
        sim.advance()
        sim.sync()
    err = {}
    for s in range(2):
        a, b = sim32.species_views(s), sim64.species_views(s)
        if not torch.equal(a["tag"], b["tag"]):
            err["tag_mismatch_species_%d" % s] = int((a["tag"] != b["tag"]).sum())
        for i, d in (("i1", "dx1"), ("i2", "dx2")):
            xa = a[i].double() + a[d].double()
            xb = b[i].double() + b[d]
            e = float(((xa - xb).abs() / xb.abs().clamp(min=1.0)).max())
            err["x" + i[1]] = max(err.get("x" + i[1], 0.0), e)
        for c in ("u1", "u2", "u3"):
            sc = float(b[c].abs().median())
            e = float(((a[c].double() - b[c]).abs() / (b[c].abs() + sc + 1e-300)).max())
            err[c] = max(err.get(c, 0.0), e)
        e = float(((a["phi"].double() - b["phi"]).abs() / b["phi"].abs().clamp(min=1.0)).max())
        err["phi"] = max(err.get("phi", 0.0), e)
    names = {0: "B1", 1: "B2", 2: "B3", 3: "D1", 4: "D2", 5: "D3"}
    for k, nm in names.items():
        pa, pb = sim32.plane(k).double(), sim64.plane(k)
        err["plane_" + nm] = float((pa - pb).abs().max() / pb.abs().max().clamp(min=1e-300))
    return err


def invariant_drift(device, steps=10000):
    """Relative drift of the conserved energy and angular momentum (Sec. 2.3) of 4096 test
    particles over `steps` pushes in the frozen Wald field, FP64 and mixed: a = 0.9 on a
    128^2 grid, r in [0.95 r_h, 20], particles at x1 in [40, 100], x2 in [20, 108],
    tetrad-frame |u| uniform in [0, 0.5]; the largest and the median |E1/E0 - 1|, |L1/L0 - 1|
    over the particles that stay inside (x1 in (10, 118))."""
    import torch

    from paper_2511_17701_gb300 import FIELD_WALD, Sim
    cfg = W.grid_config("wald64", n_r=128, n_theta=128, r_max=20.0, r_absorb=1e300)
    tp = W.probe_particles(cfg, 4096, 7, (40.0, 100.0), (20.0, 108.0), 0.5)
    qm, qc = W.species_coefficients(1.0)
    out = {}
    for prec in ("fp64", "mixed"):
        sim = Sim(dict(cfg, precision=prec), [4096], device=device)
        sim.init_metric()
        sim.init_fields(FIELD_WALD, 1.0)
        sim.load_particles(0, tp["pos"], tp["uhat"], tp["w0"], qm, qc)
        sim.predict()
        sim.push(0)
        E0, L0 = sim.invariants(0, FIELD_WALD, 1.0)
        for _ in range(steps - 1):
            sim.push(0)
        E1, L1 = sim.invariants(0, FIELD_WALD, 1.0)
        p = sim.get_particles(0)
        keep = (p["tag"] == 1) & (p["i1"] > 10) & (p["i1"] < 118)
        dE = np.abs(E1[keep] / E0[keep] - 1)
        dL = np.abs(L1[keep] / L0[keep] - 1)
        out[prec] = {"E_max": float(dE.max()), "E_median": float(np.median(dE)),
                     "L_max": float(dL.max()), "L_median": float(np.median(dL)),
                     "particles": int(keep.sum())}
        sim.close()
        del sim
        torch.cuda.empty_cache()
    out["mixed_over_fp64"] = {k: out["mixed"][k] / out["fp64"][k]
                              for k in ("E_max", "E_median", "L_max", "L_median")}
    out["setup"] = ("4096 test particles, frozen Wald field (a = 0.9, 128^2 grid, r in [0.95 "
                    "r_h, 20]), %d pushes" % steps)
    return out


def run_gpu(args, ws, rank, local):
    import torch

    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    alu = measure_alu_peaks(device) if not args.no_probe else {"sms": device_facts(device)["sms"]}
    precisions = ["fp64", "mixed"] if args.precision == "both" else [args.precision]
    res, sims = {}, {}
    e2e = None
    for prec in precisions:
        out, sim = measure(args, prec, ws, rank, local)
        if prec == precisions[0] and not args.no_e2e:
            e2e = end_to_end(args, sim, out["psteps"], ws, device)
        res[prec] = out
        sims[prec] = sim
    err = None
    if len(precisions) == 2 and not args.no_error:
        err = mixed_step_error(sims["fp64"], sims["mixed"])
    for s in sims.values():
        s.close()
    del sims
    torch.cuda.empty_cache()
    drift = invariant_drift(device) if len(precisions) == 2 and not args.no_drift else None
    main = res[precisions[0]]
    roof, hbm, step = rooflines(main, precisions[0], alu, args)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args)
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
                               main["particles"] * (65 if precisions[0] == "fp64" else 37) / 1e9),
                           "parallelism": "replica per GPU" if ws > 1 else "1 GPU"},
                "roofline": roof, "hbm_roofline": hbm, "hbm_roofline_step": step,
                "alu_peaks_measured": alu,
                "phase_ms_per_step": main["phase_ms_per_step"],
                "pusher_ns_per_particle": main["pusher_ns_per_particle"],
                "gpu_launches": main["gpu_launches"], "e2e": e2e, "cpu_baseline": cpu,
                "clocks": main["clocks"]}
        if args.workload == "bz2048":
            line["paper_context"] = {
                "pusher_ns_per_particle": 6.2, "hardware": "1x A100, precision not stated",
                "workload": "BZ monopole test, 2048^2 log-r mesh, 90 particles per cell "
                            "(Sec. 3.5)"}
        else:
            line["paper_context"] = {
                "pusher_ns_per_particle": 6.2, "hardware": "1x A100, precision not stated",
                "workload": "BZ monopole test, 2048^2 log-r mesh, 90 particles per cell "
                            "(Sec. 3.5); bench.py --workload bz2048 times that shape"}
        if len(precisions) == 2:
            m = res["mixed"]
            mroof, mhbm, mstep = rooflines(m, "mixed", alu, args)
            line["mixed"] = {"value": m["value"], "unit": "particle-steps/s",
                             "ms_per_step": m["ms_per_step"],
                             "speedup_vs_fp64": m["value"] / main["value"],
                             "workload": m["workload"], "roofline": mroof,
                             "hbm_roofline": mhbm, "hbm_roofline_step": mstep,
                             "phase_ms_per_step": m["phase_ms_per_step"],
                             "pusher_ns_per_particle": m["pusher_ns_per_particle"],
                             "gpu_launches": m["gpu_launches"], "clocks": m["clocks"],
                             "error_per_step_vs_fp64": err,
                             "error_bound": "<= 1e-5 relative per step on particle state "
                                            "(north-star bound; the FP64 path is the oracle "
                                            "to 1e-12)",
                             "invariant_drift": drift}
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
    alu = measure_alu_peaks(torch.device("cuda", local))
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
                    "push_kernel_ns_per_photon": phot["kernel_ms"] * 1e6 / (phot["particles"]),
                    "push_kernel_ns_per_pair_particle": pairs["kernel_ms"] * 1e6 /
                    (pairs["particles"] / 2),
                    "photon_hbm_gbs": rooflines(phot, prec, alu, args, photons=True)[1][
                        "achieved_gbs"],
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
        out["filter_wald2048"] = measure_filter_2048(args, ws, rank, local, alu)
    if "inject" in parts:
        out["inject_bz2048"] = measure_injection(args, local)
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
                       "push_kernel_ms": qk["kernel_ms"],
                       "push_kernel_ms_plain": base["kernel_ms"],
                       "clocks": qk["clocks"]}
        out["qks_wald512"] = q
    if rank == 0:
        print(json.dumps(out), flush=True)


def measure_filter_2048(args, ws, rank, local, alu):
    """The filter kernel against the FP64 pipe and HBM: 2048^2 planes (33.7 MB each, above
    L2), 8 passes in one launch, on the wald2048 grid with args.ext_ppc particles per cell
    per species."""
    import torch

    hp, hsrc = hbm_peak()
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
        "roofline": {"bound": "alu", "achieved": ops, "peak": alu["fp64_gops"],
                     "unit": "G FP64-pipe op/s", "frac": ops / alu["fp64_gops"],
                     "traffic": None,
                     "peak_source": "measured in this run: grpic_probe_alu FP64",
                     "kernel": "k_filter<double> (8 passes fused in shared memory)"},
        "hbm_roofline": {"achieved_gbs": gbs, "peak_gbs": hp, "frac": gbs / hp,
                         "peak_source": hsrc},
        "clocks": big["clocks"]}


def measure_injection(args, local):
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
    hp, _ = hbm_peak()
    gbs = bytes_ / (inj_ms * 1e-3) / 1e9
    del sim
    torch.cuda.empty_cache()
    return {"workload": "bz2048 grid, %d ppc per species, FP64, sigma0 = %g, sigma_th = %g"
                        % (cfg["ppc"], cfg["sigma0"], cfg["sigma_th"]),
            "particles_before": n0, "particles_after": n1, "cells": nc,
            "pairs_added_per_step": d["injected"] / args.steps,
            "inject_ms_per_call": inj_ms, "step_plus_inject_ms": ms,
            "share_of_step": inj_ms / ms,
            "hbm_roofline": {"achieved_gbs": gbs, "peak_gbs": hp,
                             "frac": gbs / hp,
                             "algorithmic_bytes_per_call": bytes_}}


def run_adjoint(args, ws, rank, local):
    """The adjoint of the pusher over a frozen field: test particles in the 512^2 Kerr
    (a = 0.9) Wald field, forward n steps with checkpoints, then the reverse sweep for the
    gradient of L = sum(v . final state) with respect to the initial state and B0, both timed
    with CUDA events; central differences of the forward on a sample of particles. With N
    ranks the particles are sharded (each rank a contiguous share of the same seeded set) and
    dL/dB0 is the exact binned sum over all ranks (one int64 all-reduce; strong scaling)."""
    import torch

    from paper_2511_17701_gb300 import FIELD_WALD, Sim
    from paper_2511_17701_gb300.binding import SUM_BINS, sum_bins_add, sum_bins_value
    from paper_2511_17701_gb300.sharded import shard_bounds

    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    cfg = W.grid_config("wald512", r_absorb=1e300)
    n_all, steps, every = args.adjoint_particles, args.adjoint_steps, args.adjoint_ckpt
    tp_all = W.probe_particles(cfg, n_all, 77, (0.2 * cfg["n_r"], 0.8 * cfg["n_r"]),
                               (0.15 * cfg["n_theta"], 0.85 * cfg["n_theta"]), 0.5)
    lo, hi = shard_bounds(n_all, rank, ws)
    n = hi - lo
    tp = {"pos": {k: a[lo:hi] for k, a in tp_all["pos"].items()}, "uhat": tp_all["uhat"][:, lo:hi],
          "w0": tp_all["w0"][lo:hi]}
    qm, qc = W.species_coefficients(1.0)
    sim = Sim(cfg, [n], device=device)
    sim.init_metric()
    sim.init_fields(FIELD_WALD, cfg["B0"])
    sim.load_particles(0, tp["pos"], tp["uhat"], tp["w0"], qm, qc)  # u_i = e_i^j u_j^ on the GPU
    v = sim.species_views(0)
    st0 = torch.stack([v["i1"].double() + v["dx1"], v["i2"].double() + v["dx2"], v["phi"],
                       v["u1"], v["u2"], v["u3"]]).contiguous()
    gen = torch.Generator(device=device).manual_seed(5)
    cot = torch.randn((6, n_all), dtype=torch.float64, device=device, generator=gen)[:, lo:hi]
    cot = cot.contiguous()
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
        # dL/dB0 over every rank's particles: exact bins, one int64 all-reduce, one rounding
        bins = torch.zeros(2 * SUM_BINS, dtype=torch.int64, device=device)
        sum_bins_add(gpp.contiguous(), bins, stream)
        if ws > 1:
            import torch.distributed as dist
            dist.all_reduce(bins, op=dist.ReduceOp.SUM)
        ev[2].record(stream)
        torch.cuda.synchronize(device)
    fwd_ms, bwd_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    fwd_ms, bwd_ms = allreduce_max(ws, fwd_ms, device), allreduce_max(ws, bwd_ms, device)
    dL_dB0 = sum_bins_value(bins.cpu())
    n_ok = int(allreduce_sum(ws, float(ok.sum()), device))
    # central differences of the forward on a sample of particles that stayed inside
    idx = torch.nonzero(ok).flatten()[: args.adjoint_fd_sample]
    sub = st0[:, idx].contiguous()
    csub = gout[:, idx]

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

    ad = torch.cat([gin[:, idx], gpp[idx][None]])

    def rel(fd):
        good = ~torch.isnan(fd).any(dim=0)
        return ((fd - ad).abs().amax(dim=0) / ad.abs().amax(dim=0))[good].cpu().numpy()

    # over 2000 steps the +-h orbits cross kinks of the bilinear interpolation: the quotient
    # converges to the derivative only as h shrinks, so it is reported at several steps
    fd_by_h = {}
    for hh in (1e-6, 2.5e-7, 6.25e-8):
        e = rel(central(hh))
        fd_by_h["%g" % hh] = {"sample": int(e.size),
                              "median_rel_err": float(np.median(e)) if e.size else None,
                              "p90_rel_err": float(np.quantile(e, 0.9)) if e.size else None,
                              "max_rel_err": float(e.max()) if e.size else None,
                              "frac_within_1e-6": float((e < 1e-6).mean()) if e.size else None}
    psteps = n_ok * steps
    line = {"metric": "adjoint push: particle-steps/s (frozen field, forward + reverse sweep)",
            "value": psteps / ((fwd_ms + bwd_ms) * 1e-3), "unit": "particle-steps/s",
            "n_gpus": ws, "steps": steps, "warmup": 1, "higher_is_better": True,
            "scaling": "strong", "dtype": "f64", "data": "synthetic (seeded test particles)",
            "config": {"workload": "adjoint: %d test particles (x1 in [0.2, 0.8] n_r, x2 in "
                                   "[0.15, 0.85] n_theta, |u^| uniform in [0, 0.5]) in the frozen "
                                   "Wald field, Kerr a=0.9, B0 as parameter, 512x512 log-r grid "
                                   "r in [0.95 r_h, 50]; %d FP64 steps, checkpoints every %d"
                                   % (n_all, steps, every),
                       "parallelism": "particles sharded over %d rank(s), dL/dB0 exact "
                                      "all-reduce" % ws},
            "forward_ms": fwd_ms, "backward_ms": bwd_ms,
            "forward_particle_steps_per_s": n_all * steps / (fwd_ms * 1e-3),
            "particles_kept": n_ok,
            "dL_dB0": dL_dB0, "dL_dB0_this_rank_library_sum": float(gsum.cpu()[0]),
            "fd_check": fd_by_h,
            "gpu_launches": None, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


def bz_diagnostics(sim, cfg, radii):
    """The closed-form quantities of Sec. 4.5 from one snapshot of the em planes: per radius,
    the field-line angular velocity Omega = -E_theta / (sqrt(h) B^r) averaged over theta in
    [pi/6, 5 pi/6] with weight sin^2(theta) (BZ: omega_h / 2 at every latitude to O(a^2)) and
    the peak of its theta profile (smoothed over 5 rows, theta in [0.1 pi, 0.9 pi]; the paper
    states where the profile peaks), the
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
        # the profile's peak (the paper's statement about Omega): the largest value of the
        # profile smoothed over 5 rows, within theta in [0.1 pi, 0.9 pi]
        sm = np.convolve(om, np.ones(5) / 5.0, mode="same")
        band = (thc > 0.1 * math.pi) & (thc < 0.9 * math.pi)
        kpk = int(np.argmax(np.where(band, sm, -np.inf)))
        out[rr] = {"omega": float(np.sum(w * om[mid]) / np.sum(w)),
                   "omega_peak": float(sm[kpk]), "omega_peak_theta": float(thc[kpk]),
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
    every = max(1, args.bz_inject_every)
    n_step = 0
    for mark in range(1, n_mark + 1):
        k = int(round((mark - t) / dt))
        for _ in range(k):
            sim.step(1)
            n_step += 1
            if n_step % every == 0:
                sim.inject(cfg["sigma0"], cfg["sigma_th"], B0, pool)
        t += k * dt
        if mark > 2 * n_mark / 3:
            snaps.append(bz_diagnostics(sim, cfg, radii))
            sn = snaps[-1]
            print(json.dumps({"t": t, "omega_over_omega_h": {str(r): sn[r]["omega"] / wh
                                                             for r in radii},
                              "omega_peak_over_omega_h": {str(r): sn[r]["omega_peak"] / wh
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
                                   "~ r^-2, injection after every %d step(s)" % (a, n_g, n_g, every),
                       "t_end_rg": t, "dt": dt, "average_over_rg": [t - len(snaps), t],
                       "omega_h": wh, "L_BZ": LBZ},
            "omega_over_omega_h": avg("omega", wh), "omega_spread": spread("omega", wh),
            "omega_peak_over_omega_h": avg("omega_peak", wh),
            "omega_peak_theta": avg("omega_peak_theta", 1.0),
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
    ap.add_argument("--workload", default=None, choices=sorted(W.CONFIGS),
                    help="default wald2048 (--extensions: wald512)")
    ap.add_argument("--sort-every", type=int, default=10)
    ap.add_argument("--tile", type=int, default=16)
    ap.add_argument("--precision", default="both", choices=["fp64", "mixed", "both"],
                    help="both: FP64 (the line's value) and then mixed on the same workload")
    ap.add_argument("--ppc", type=int, default=0, help="override particles per cell per species "
                    "(a smaller case of the same workload, e.g. for profiling)")
    ap.add_argument("--cpu-frac", type=float, default=0.03,
                    help="fraction of the cells whose particles the CPU baseline pushes")
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--cpu-steps-1core", type=int, default=1, choices=range(1, 11),
                    help="steps of the one-core particle phases in the CPU baseline")
    ap.add_argument("--ref-frac", type=float, default=0.01,
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
    ap.add_argument("--tiled-push", type=int, default=0, choices=[0, 1, 2],
                    help="mixed path: 1 = the shared-memory tiled FP32 kernel (window loaded by "
                         "the CTA's threads), 2 = the same with the window loaded by TMA bulk "
                         "tensor copies; 0 (default) = one thread per particle")
    ap.add_argument("--bz-physics", action="store_true",
                    help="run the BZ monopole test of Sec. 4.5 and report its closed-form checks")
    ap.add_argument("--bz-n", type=int, default=512, help="--bz-physics: cells per direction")
    ap.add_argument("--bz-time", type=float, default=60.0, help="--bz-physics: run time, r_g")
    ap.add_argument("--bz-precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--bz-inject-every", type=int, default=1,
                    help="--bz-physics: pair injection after every k-th step (reading R32: 1)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-probe", action="store_true",
                    help="skip the FMA-throughput probe (the ALU rooflines then have no peak)")
    ap.add_argument("--no-error", action="store_true",
                    help="skip the mixed path's per-step error against the FP64 path")
    ap.add_argument("--no-drift", action="store_true",
                    help="skip the 10^4-step invariant drift of test particles")
    args = ap.parse_args()
    if args.workload is None:
        args.workload = "wald512" if args.extensions else "wald2048"
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
