"""Benchmark of the CVF Metropolis hot path on GB300.

Workload (one "step"): 1000 MC steps -- each one volume move plus a full
checkerboard sweep of the four sigma_ij of every cell, with the N_HB /
N_sigma reductions -- of a 4096 x 4096 lattice (q = 6), cycling through the
six lattices of the 4096^2 configuration: random (seed 3) and ordered init at
270, 300 and 330 K, 0.1 MPa.  Inputs (the lattices) are resident in HBM when
the timed region starts; L2 is flushed between timed steps.

  value  = sigma updates per ns = 4 L^2 x sweeps / device time (CUDA events)
  e2e    = the same through the C ABI with host buffers: set_state (H2D),
           sweep, get_state (D2H) and observables inside the timed region
  --impl reference   times the CPU oracle on the same metric (bounded sample)

The line also carries the batched (256 replicas, one persistent launch),
serving (continuous batching of arriving jobs) and cubic (the paper's own 3D
model at 260^3) measurements.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time
from dataclasses import asdict

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CVF Metropolis updates/ns at 4096²; batched replica sweeps/s, p50/p99"
UNIT = "updates/ns"
L2_FLUSH_BYTES = 512 << 20  # > 126.5 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--L", type=int, default=4096)
    ap.add_argument("--sweeps", type=int, default=1000, help="MC steps per benchmark step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-sweeps", type=int, default=10)
    ap.add_argument("--mode", default="full", choices=["full", "kernel", "kernel3", "batch"],
                    help="kernel / kernel3: one square / cubic lattice; batch: the 256 "
                         "replicas of the batched configuration in one persistent launch "
                         "per call (tile shape from the autotuner); warm-up then timed sweeps "
                         "only (profiling cases)")
    ap.add_argument("--L3", type=int, default=260,
                    help="cube side of the 3D measurement (260: the paper's largest lattice)")
    ap.add_argument("--cubic-sweeps", type=int, default=320,
                    help="timed MC steps of the 3D measurement (0: skip)")
    ap.add_argument("--batch-sweeps", type=int, default=5000,
                    help="steps per replica in the batched measurement (0: skip)")
    ap.add_argument("--serve-seconds", type=float, default=8.0,
                    help="time budget of the serving measurement (0: skip)")
    ap.add_argument("--record-counters", default=None,
                    help="write the sweep's counters file from this ncu CSV and exit")
    ap.add_argument("--tiles", type=int, default=-1,
                    help="kernel mode: the sweep configuration (cvf_set_tiles; -1: automatic)")
    ap.add_argument("--counter-steps", type=int, default=1,
                    help="MC steps in the launch the counters CSV captured (the wavefront "
                         "sweep runs a whole call in one launch)")
    return ap.parse_args()


# Issue-rate peak: 152 SMs x 128 thread-instructions per clock x the 2070 MHz
# maximum clock (four schedulers of one warp-instruction per clock per SM).
ISSUE_PEAK_T = 152 * 128 * 2.070e9 / 1e12

# Counters of the 4096^2 sweep per MC step (ncu: DRAM read + write bytes,
# executed warp instructions of one launch of the sweep kernel the automatic
# configuration runs there -- k_sweep_wave, one launch per call -- divided
# by the launch's steps), recorded by `bench.py --record-counters` from an ncu
# capture together with a hash of the sweep kernels' sources; the bench uses
# them only while that hash matches the current sources (null otherwise: the
# kernel changed since the capture).
COUNTERS_FILE = os.path.join(ROOT, "profiles", "k_sweep_wave_L4096_counters.json")
# the device code of the sweeps (the public header's declarations and
# comments do not enter it and are left out)
SWEEP_SOURCES = ("paper_2505_05919_gb300/csrc/cvf_tile.cuh", "paper_2505_05919_gb300/csrc/cvf_lattice.cu",
                 "paper_2505_05919_gb300/csrc/cvf_lattice.cuh", "paper_2505_05919_gb300/csrc/cvf_device.cuh",
                 "paper_2505_05919_gb300/csrc/cvf_tma.cuh", "paper_2505_05919_gb300/csrc/cvf_wave.cu",
                 "paper_2505_05919_gb300/csrc/cvf_fastdiv.cuh")


def sweep_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in SWEEP_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def sweep_counters():
    """The recorded counters of the current sweep kernel, or None."""
    try:
        d = json.load(open(COUNTERS_FILE))
    except Exception:
        return None
    return d if d.get("source_hash") == sweep_source_hash() else None


def record_counters(csv_path: str, steps: int) -> int:
    """Write COUNTERS_FILE from an ncu CSV (--csv --log-file) of one launch
    of the 4096^2 sweep kernel (k_sweep_wave or k_sweep_tiled) covering
    `steps` MC steps, with the metrics dram__bytes_read.sum,
    dram__bytes_write.sum and smsp__inst_executed.sum."""
    import csv
    rows = [r for r in csv.reader(open(csv_path)) if len(r) > 5]
    hdr = rows[0]
    im, iv, ik = hdr.index("Metric Name"), hdr.index("Metric Value"), hdr.index("Kernel Name")
    vals, kernel = {}, None
    for r in rows[1:]:
        if "k_sweep_wave" in r[ik] or "k_sweep_tiled" in r[ik]:
            vals[r[im]] = float(r[iv].replace(",", ""))
            kernel = r[ik]
    cells = 4096 * 4096
    out = {"kernel": "%s (%d MC steps of the 4096^2 lattice in the launch, q = 6, 300 K)"
                     % (kernel, steps),
           "source_hash": sweep_source_hash(), "cells": cells, "steps_in_launch": steps,
           "dram_bytes": (vals["dram__bytes_read.sum"] + vals["dram__bytes_write.sum"]) / steps,
           "inst_executed_warp": vals["smsp__inst_executed.sum"] / steps,
           "instructions_per_update": vals["smsp__inst_executed.sum"] * 32 / (4 * cells * steps),
           "per": "MC step",
           "capture": os.path.basename(csv_path)}
    with open(COUNTERS_FILE, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out))
    return 0


def philox_ceiling(stream, n_cells, reps=50):
    """Event-timed rate of the random-number work of one step alone
    (cvf_philox_probe: one Philox4x32-10 block per cell, four sigma updates
    per block), in sigma-updates/ns: the most a sweep that draws its numbers
    this way can reach on this GPU."""
    import torch
    from paper_2505_05919_gb300 import _capi
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    sp = stream.cuda_stream
    for i in range(3):
        _capi.cvf_philox_probe(3, n_cells, i, out.data_ptr(), sp)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(reps):
        _capi.cvf_philox_probe(3, n_cells, 100 + i, out.data_ptr(), sp)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return 4.0 * n_cells / (ms * 1e6), ms


def dist_env():
    from paper_2505_05919_gb300 import dist
    return dist.env()


def workload_configs(L):
    from paper_2505_05919_gb300 import workloads
    cfgs = workloads.c3()
    for c in cfgs:
        c["L"] = L
    return cfgs


def oracle_params(cfg, seed_offset=0):
    import oracle
    return oracle.physical_params(cfg["T"], cfg["P"], L=cfg["L"], q=cfg["q"],
                                  seed=cfg["seed"] + seed_offset, init=cfg["init"])


def lib_params(cfg, seed_offset=0):
    """Library parameters from the workload recipe (library-side units)."""
    from paper_2505_05919_gb300 import params
    return params(cfg["T"], cfg["P"], L=cfg["L"], q=cfg["q"], seed=cfg["seed"] + seed_offset,
                  init=cfg["init"])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(parts)
            except ValueError:
                pass
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for i, n in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(n)
        loaded = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        out.update(sm_mhz=statistics.median(loaded) if loaded else None,
                   sm_max_mhz=max(mx) if mx else None, reasons=sorted(reasons), samples=len(rows))
        return out


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def cpu_baseline(cfg, sample_sweeps):
    """The oracle, single-threaded, on a bounded sample of the workload."""
    import oracle
    op = oracle_params(cfg)
    t0 = time.perf_counter()
    o = oracle.Oracle(op)
    t1 = time.perf_counter()
    o.run(sample_sweeps)
    t2 = time.perf_counter()
    upd = 4.0 * cfg["L"] * cfg["L"] * sample_sweeps
    return {"value": upd / ((t2 - t1) * 1e9), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "L=%d, %d MC steps from the random init (seed %d, %g K), one thread; "
                      "init %.1f s not counted" % (cfg["L"], sample_sweeps, cfg["seed"], cfg["T"], t1 - t0)}


def _oracle_replica(args):
    """One oracle replica for the all-cores baseline (runs in a spawned
    process): L x L lattice from the random init, `steps` MC steps."""
    cfg, seed_offset, steps = args
    sys.path.insert(0, ROOT)
    import oracle
    o = oracle.Oracle(oracle_params(cfg, seed_offset=seed_offset))
    t0 = time.perf_counter()
    o.run(steps)
    return time.perf_counter() - t0


def cpu_baseline_all_cores(cfg, L=1024, steps=20):
    """nproc independent oracle replicas run concurrently, one per host core
    (independent seeds): aggregate sigma updates per ns over the slowest."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    c = dict(cfg)
    c["L"] = L
    ctx = mp.get_context("spawn")  # never fork a process that holds a CUDA context
    with ctx.Pool(n) as pool:
        times = pool.map(_oracle_replica, [(c, i, steps) for i in range(n)])
    upd = 4.0 * L * L * steps * n
    return {"value": upd / (max(times) * 1e9), "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": "%d concurrent replicas (one per core), each L=%d, %d MC steps from the random "
                      "init (seeds %d..%d), %g K" % (n, L, steps, cfg["seed"], cfg["seed"] + n - 1, cfg["T"])}


def arm_config(L, S):
    """The `config` of the benchmark line (both arms)."""
    return {"workload": "CVF 2D L=%d q=6, %d MC steps/step, random(seed 3)+ordered init at "
                        "270/300/330 K, 0.1 MPa" % (L, S),
            "L": L, "sweeps_per_step": S, "l2": "flushed between timed steps (512 MB write)",
            "rng_words": 1, "schedule": "checkerboard"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    cfg = workload_configs(args.L)[1]  # random init, 300 K
    op = oracle_params(cfg)
    o = oracle.Oracle(op)
    per_step = max(1, args.cpu_sample_sweeps // 10)
    for _ in range(args.warmup):
        o.run(per_step)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.run(per_step)
    dt = time.perf_counter() - t0
    upd = 4.0 * args.L * args.L * per_step * args.steps
    value = upd / (dt * 1e9)
    sample = ("each step: %d MC step(s) of the L=%d lattice (random init seed %d, %g K, %g MPa; "
              "one of the configuration's six, a bounded sample of its 1000-step step) by the "
              "single-threaded oracle" % (per_step, args.L, cfg["seed"], cfg["T"], cfg["P"]))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u16+int64+f64", "data": "synthetic",
            "impl": "reference",
            "config": arm_config(args.L, args.sweeps),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_kernel_mode(args):
    """Small profiling case: one lattice (random init, 300 K), `warmup`
    sweeps, then `steps` sweeps timed with CUDA events; no flush buffer."""
    import torch
    from paper_2505_05919_gb300 import Lattice, _capi, build as libbuild
    libbuild.build()
    _capi.load()
    cfg = workload_configs(args.L)[1]
    stream = torch.cuda.Stream()
    lat = Lattice(lib_params(cfg), stream=stream)
    if args.tiles >= 0:
        lat.set_tiles(args.tiles)
    tiles = lat.tiles()[0]
    lat.sweep(args.warmup)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    lat.sweep(args.steps)
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    o = lat.observables()
    lat.close()
    print(json.dumps({"mode": "kernel", "L": args.L, "tiles": tiles, "sweeps": args.steps, "ms": ms,
                      "updates_per_ns": 4.0 * args.L * args.L * args.steps / (ms * 1e6),
                      "n_hb_raw": o["n_hb_raw"], "n_coop": o["n_coop"]}))
    return 0


# The paper's own 3D figure (context, other hardware): 280 ms per Metropolis
# MC step at N = 260^3 on an RTX 3060, cuRAND generation and copies included.
PAPER_3D_MS_PER_STEP_260 = 280.0
# The paper's linear fit of its time per Metropolis step against N (Fig. 4
# caption), for context beside the per-size timings.
PAPER_3D_FIT_A_MS = 4.11e-6
PAPER_3D_FIT_B_MS = 1.2e-2
def run_kernel3_mode(args):
    """Profiling case of the cubic lattice: one cube (random init seed 3,
    300 K, 0.1 MPa), `warmup` MC steps, then `steps` timed with CUDA events."""
    import torch
    from paper_2505_05919_gb300 import Lattice3, params3, _capi, build as libbuild
    libbuild.build()
    _capi.load()
    stream = torch.cuda.Stream()
    lat = Lattice3(params3(300.0, 0.1, L=args.L3, seed=3), stream=stream)
    lat.sweep(args.warmup)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    lat.sweep(args.steps)
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    o = lat.observables()
    lat.close()
    print(json.dumps({"mode": "kernel3", "L": args.L3, "sweeps": args.steps, "ms": ms,
                      "updates_per_ns": 6.0 * args.L3 ** 3 * args.steps / (ms * 1e6),
                      "n_hb_raw": o["n_hb_raw"], "n_coop": o["n_coop"]}))
    return 0


def run_batch_mode(args):
    """Profiling case of the batched sweep: the 256 replicas of the batched
    configuration (L from {32..512}, T x P grid), tile configuration from the
    autotuner, `warmup` MC steps each in one call, then one call of `steps`
    MC steps each (one persistent launch) timed with CUDA events."""
    import torch
    from paper_2505_05919_gb300 import Batch, params, workloads, _capi, build as libbuild
    from paper_2505_05919_gb300.autotune import autotune
    libbuild.build()
    _capi.load()
    reps = workloads.c4(sweeps=args.steps)
    ps = [params(r["T"], r["P"], L=r["L"], q=r["q"], seed=r["seed"]) for r in reps]
    stream = torch.cuda.Stream()
    best, _ = autotune(ps, probe_sweeps=20, stream=stream)
    with Batch(ps, stream=stream) as b:
        b.set_tiles(best)
        b.sweep([args.warmup] * len(ps))
        b.sync()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        b.sweep([args.steps] * len(ps))
        ev1.record(stream)
        ev1.synchronize()
        b.sync()
        ms = ev0.elapsed_time(ev1)
    cells = sum(r["L"] * r["L"] for r in reps)
    print(json.dumps({"mode": "batch", "replicas": len(ps), "sweeps": args.steps, "ms": ms,
                      "tile_config": best,
                      "replica_sweeps_per_s": len(ps) * args.steps / (ms / 1e3),
                      "updates_per_ns": 4.0 * cells * args.steps / (ms * 1e6)}))
    return 0


def measure_cubic(args, rank, world):
    if not hasattr(args, "philox_ceiling"):
        import torch
        args.philox_ceiling, _ = philox_ceiling(torch.cuda.Stream(), 4096 * 4096)
    """The paper's own 3D model at its largest size (260^3, q = 6, 300 K,
    0.1 MPa, random init seed 3): MC steps of the six-arm layered schedule
    timed with CUDA events on the lattice's stream (the 70 MB lattice stays
    in HBM/L2), next to the paper's 280 ms per step on an RTX 3060 and the 3D
    oracle on a bounded sample."""
    import torch
    from paper_2505_05919_gb300 import Lattice3, dist, params3
    L, S = args.L3, args.cubic_sweeps
    stream = torch.cuda.Stream()
    lat = Lattice3(params3(300.0, 0.1, L=L, seed=3 + dist.seed_offset(rank)), stream=stream)
    lat.sweep(64)
    torch.cuda.synchronize()
    ms = []
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.sweep(S)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1) / S)
    per_step = statistics.median(ms)
    dev_s = dist.max_over_ranks(per_step / 1e3)
    o = lat.observables()
    lat.close()
    upd = 6.0 * L ** 3
    out = {"value": upd * world / (dev_s * 1e9), "unit": UNIT, "L": L, "N": L ** 3,
           "ms_per_mc_step": dev_s * 1e3, "sweeps_timed": S,
           "paper_ms_per_mc_step": PAPER_3D_MS_PER_STEP_260 if L == 260 else None,
           "paper_hardware": "RTX 3060 (sm_86), cuRAND and copies included",
           "launches_per_mc_step": 5,
           "roofline": {"bound": "alu", "achieved": upd / (per_step * 1e6),
                        "peak": args.philox_ceiling, "unit": "sigma-updates/ns",
                        "frac": upd / (per_step * 1e6) / args.philox_ceiling if args.philox_ceiling else None,
                        "peak_kind": "measured: the Philox draws alone (cvf_philox_probe, four "
                                     "updates per Philox block, as the passes draw them)",
                        "traffic": None,
                        "kernel": "k_eta3 + k_pass3 (five launches per MC step)"},
           "eta_moves": 1,
           "acceptance": o["acc_sigma"] / max(1.0, upd * o["sweep"]),
           "workload": "CVF 3D cubic lattice L=%d q=6, layered six-arm schedule with the eta "
                       "update of the checkerboard cubes, random init (seed 3), 300 K, 0.1 MPa" % L}
    # time per MC step against N over the sizes of the paper's Fig. 4, next
    # to its linear fit t = a N + b (RTX 3060, 32768 <= N <= 2097152)
    sizes = []
    for Ls in (16, 32, 52, 64, 100, 128, 160, 200):
        lat = Lattice3(params3(300.0, 0.1, L=Ls, seed=3), stream=stream)
        lat.sweep(64)
        torch.cuda.synchronize()
        n_steps = 640 if Ls <= 64 else 320
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.sweep(n_steps)
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) / n_steps
        lat.close()
        Ns = Ls ** 3
        sizes.append({"L": Ls, "N": Ns, "ms_per_mc_step": t,
                      "paper_fit_ms_per_mc_step": PAPER_3D_FIT_A_MS * Ns + PAPER_3D_FIT_B_MS,
                      "updates_per_ns": 6.0 * Ns / (t * 1e6)})
    out["by_size"] = sizes
    out["paper_fit"] = "t = 4.11e-6 ms x N + 1.2e-2 ms (RTX 3060, fitted on 32768 <= N <= 2097152)"
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            import oracle
            Lc = min(L, 128)
            ref = oracle.Oracle3(oracle.physical_params3(300.0, 0.1, L=Lc, seed=3))
            t0 = time.perf_counter()
            ref.run(3)
            dt = time.perf_counter() - t0
            out["cpu_baseline"] = {"value": 6.0 * Lc ** 3 * 3 / (dt * 1e9), "unit": UNIT, "cores": 1,
                                   "kind": "oracle",
                                   "sample": "3D oracle, L=%d, 3 MC steps from the random init, "
                                             "one thread" % Lc}
        except Exception as e:
            out["cpu_baseline"] = {"value": None, "error": str(e)}
    return out


def copy_bandwidth_gbs(stream, nbytes, reps):
    """Event-timed bandwidth (read + write bytes / s) of this library's
    16-byte copy kernel between two device buffers of `nbytes`, copied back
    and forth `reps` times after three warm-up copies."""
    import torch
    from paper_2505_05919_gb300 import _capi
    a = torch.ones(nbytes, dtype=torch.uint8, device="cuda")
    b = torch.zeros_like(a)
    torch.cuda.synchronize()  # the fills run on torch's stream
    sp = stream.cuda_stream
    for _ in range(3):
        _capi.cvf_copy_probe(b.data_ptr(), a.data_ptr(), nbytes, sp)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for r in range(reps):
        src, dst = (a, b) if r % 2 == 0 else (b, a)
        _capi.cvf_copy_probe(dst.data_ptr(), src.data_ptr(), nbytes, sp)
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    del a, b
    return 2.0 * nbytes * reps / (ms * 1e-3) / 1e9


def cpu_small_configs():
    """The oracle, one thread, on configurations 1 (in full: L 64, 1000 MC
    steps) and 2 (L 1024, the first 50 of its 10^4 MC steps, recording every
    10 as the configuration does); the init is not timed."""
    import oracle
    from paper_2505_05919_gb300 import workloads
    out = {}
    for name, c, n in (("c1", workloads.c1(), 1000), ("c2", workloads.c2(), 50)):
        op = oracle.physical_params(c["T"], c["P"], L=c["L"], q=c["q"], seed=c["seed"],
                                    init=oracle.INIT_RANDOM)
        o = oracle.Oracle(op)
        t0 = time.perf_counter()
        o.run(n, c.get("record_every", 0))
        dt = time.perf_counter() - t0
        out[name] = {"value": 4.0 * c["L"] ** 2 * n / (dt * 1e9), "unit": UNIT, "cores": 1,
                     "kind": "oracle", "ms_per_mc_step": dt * 1e3 / n,
                     "sample": "L=%d, %d of the configuration's %d MC steps, random init seed %d, "
                               "one thread" % (c["L"], n, c["sweeps"], c["seed"])}
    return out


def measure_order_parameter(rank, L=32, steps=8000, skip=4000, max_lag=2000):
    """The order parameter M and its correlation time (Sec. III.A) at the
    paper's dynamics size N = 32^3 = 32768: a cube (300 K, 0.1 MPa, random
    init) recorded every MC step on the GPU (N_q' counted in the sweep),
    drained, and analysed: M = max N_q' / (6 N) at a few steps of the
    relaxation, and C_M(dt) and tau (first 1/e) over the second half."""
    import torch
    from paper_2505_05919_gb300 import Lattice3, analysis, dist, params3
    stream = torch.cuda.Stream()
    with Lattice3(params3(300.0, 0.1, L=L, seed=11 + dist.seed_offset(rank)), stream=stream) as lat:
        lat.sweep(8, 1)
        lat.drain()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        lat.sweep(steps, 1)
        ev1.record(stream)
        ev1.synchronize()
        recs, overflow = lat.drain(steps + 16)
    m = analysis.order_series(recs, L ** 3, arms=6)
    c = analysis.autocorrelation(m[skip:], max_lag)
    tau = analysis.correlation_time(c)  # None in the line when C_M stays above 1/e
    return {"L": L, "cells": L ** 3, "steps": steps, "recorded_every": 1,
            "ms_per_mc_step": ev0.elapsed_time(ev1) / steps, "records": len(recs),
            "overflow": bool(overflow),
            "M_at_step": {str(t + 1): float(m[t]) for t in (0, 9, 99, 999, 3999, steps - 1)},
            "M_mean_after_skip": float(m[skip:].mean()), "max_lag": max_lag,
            "tau_steps": tau if math.isfinite(tau) else None, "skip": skip,
            "workload": "CVF 3D cube L=%d q=6, 300 K, 0.1 MPa, random init (seed 11), "
                        "observables and N_q' recorded every MC step" % L}


def measure_small_configs(rank):
    """Configurations 1 and 2 as single lattices through the public API:
    C1 = L 64, 1000 MC steps (latency of one small lattice); C2 = L 1024,
    10^4 steps with the observables recorded every 10 steps (1000 ring
    records, drained at the end).  Wall-clock around sweep + drain +
    observables, after a warm-up call that instantiates the step graphs."""
    import torch
    from paper_2505_05919_gb300 import Lattice, dist, params, workloads
    out = {}
    for name, c in (("c1", workloads.c1()), ("c2", workloads.c2())):
        stream = torch.cuda.Stream()
        lat = Lattice(params(c["T"], c["P"], L=c["L"], q=c["q"], seed=c["seed"] + dist.seed_offset(rank)),
                      stream=stream)
        every = c.get("record_every", 0)
        lat.sweep(64, every)
        lat.drain()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.sweep(c["sweeps"], every)
        recs, overflow = lat.drain()
        o = lat.observables()
        dt = time.perf_counter() - t0
        lat.close()
        out[name] = {"L": c["L"], "sweeps": c["sweeps"], "record_every": every,
                     "records": len(recs), "wall_ms": dt * 1e3,
                     "ms_per_mc_step": dt * 1e3 / c["sweeps"],
                     "updates_per_ns": 4.0 * c["L"] ** 2 * c["sweeps"] / (dt * 1e9),
                     "acceptance": o["acc_sigma"] / max(1.0, 4.0 * c["L"] ** 2 * o["sweep"])}
    return out


def measure_batched(args, rank):
    """Configuration 4: 256 replicas (L from {32..512}, T x P grid), the same
    number of steps each, in one persistent launch per call; tile shape from
    the autotuner.  Baselines: the same replicas one at a time (a Lattice
    each, 200 steps) with one launch per MC step, and in their fastest
    single-lattice form, as replica-steps per second."""
    import torch
    from paper_2505_05919_gb300 import Batch, Lattice, dist, params, workloads
    from paper_2505_05919_gb300.autotune import autotune, cells_per_thread
    from paper_2505_05919_gb300.batch import tile_configs
    reps = workloads.c4(sweeps=args.batch_sweeps)
    ps = [params(r["T"], r["P"], L=r["L"], q=r["q"], seed=r["seed"] + dist.seed_offset(rank)) for r in reps]
    stream = torch.cuda.Stream()
    best, timings = autotune(ps, probe_sweeps=20, stream=stream)
    with Batch(ps, stream=stream) as b:
        b.set_tiles(best)
        b.sweep([3] * len(ps))
        b.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.sweep([args.batch_sweeps] * len(ps))
        e1.record(stream)
        e1.synchronize()
        b.sync()
        ms = e0.elapsed_time(e1)
    cells = sum(r["L"] * r["L"] for r in reps)
    batched_rate = len(ps) * args.batch_sweeps / (ms / 1e3)
    solo_steps = 200

    def solo(resident_ok):
        """The replicas one at a time through the single-lattice API: with
        resident_ok, each in its fastest form (small lattices stay in one
        cluster for all the steps); without, one launch per MC step."""
        total_ms = 0.0
        with torch.cuda.stream(stream):
            for p in ps:
                with Lattice(p, stream=stream) as lat:
                    if not resident_ok and lat.tiles()[0] == 3:
                        lat.set_tiles(2)
                    lat.sweep(3)
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    lat.sweep(solo_steps)
                    e1.record(stream)
                    e1.synchronize()
                    total_ms += e0.elapsed_time(e1)
        return len(ps) * solo_steps / (total_ms / 1e3)

    per_launch_rate = solo(False)
    alone_rate = solo(True)
    return {"value": batched_rate, "unit": "replica-sweeps/s", "replicas": len(ps),
            "sweeps_each": args.batch_sweeps, "ms": ms,
            "updates_per_ns": 4.0 * cells * args.batch_sweeps / (ms * 1e6),
            "one_replica_per_launch": {"value": per_launch_rate, "unit": "replica-sweeps/s",
                                       "sweeps_each": solo_steps,
                                       "form": "each replica alone, one sweep launch per MC step"},
            "speedup_vs_one_replica_per_launch": batched_rate / per_launch_rate,
            "one_lattice_at_a_time": {"value": alone_rate, "unit": "replica-sweeps/s",
                                      "sweeps_each": solo_steps,
                                      "form": "each replica alone in its fastest single-lattice "
                                              "form (small lattices resident in one cluster)"},
            "speedup_vs_one_lattice_at_a_time": batched_rate / alone_rate,
            "tile_config": best, "tile": list(tile_configs()[best][:2]),
            "block_threads": tile_configs()[best][2],
            "cells_per_thread": cells_per_thread(best), "autotune_ms_per_step": timings,
            "workload": "256 replicas, L from {32,64,128,256,512} (seed 4), T_i = 270 + 4i K, "
                        "P_j = 0.1 + j 49.9/15 MPa, seeds 1000 + r"}


def measure_serving(args, rank):
    """Configuration 5: Poisson arrivals (200 jobs/s) of EOS jobs, L uniform in
    {64..2048}, steps log-uniform in 10^3..10^5, served by continuous batching
    for a fixed wall-clock budget.  The offered load exceeds one GPU's
    throughput many times over, so the queue grows; latency is reported over
    finished jobs and over all arrived jobs (unfinished ones counted with the
    time they waited: a lower bound, flagged).  Then the same job
    distribution at 3 jobs/s, arrivals over the same budget and served until
    the last job finishes (or three budgets pass), twice: with epochs
    overlapped with the host's admission and read-back (the default), and
    with the host waiting for each epoch, for the GPU-busy comparison."""
    from paper_2505_05919_gb300 import dist, workloads
    from paper_2505_05919_gb300.serve import Job, Server

    def run(trace, budget, **kw):
        jobs = [Job(T=j["T"], P=j["P"], L=j["L"], sweeps=j["sweeps"],
                    seed=j["seed"] + dist.seed_offset(rank), arrival=j["arrival"]) for j in trace]
        srv = Server(**kw)
        try:
            return srv.run_trace(jobs, time_limit=budget)
        finally:
            srv.close()

    # epochs of at most 400 steps (about 4e9 cell-steps when many large
    # lattices are resident): new jobs are admitted every few milliseconds
    common = dict(epoch_steps=400, epoch_cell_steps=4e9, max_resident_cells=64 << 20)
    budget = args.serve_seconds
    over = run(workloads.c5(), budget, **common)
    over["offered_jobs_per_s"] = 200.0
    over["workload"] = ("Poisson 200 jobs/s (seed 5), L uniform {64,...,2048}, steps log-uniform "
                        "1e3..1e5, (T, P) uniform 270-330 K x 0.1-50 MPa, %.0f s budget" % budget)
    rate = 3.0
    light_trace = workloads.c5(n_jobs=max(1, int(rate * budget)), rate_hz=rate)
    light = run(light_trace, 3 * budget, **common)
    light_sync = run(light_trace, 3 * budget, overlap=False, **common)
    desc = ("Poisson %.0f jobs/s (seed 5), %d jobs, the same L, step and (T, P) "
            "distributions, served until done (limit %.0f s)" % (rate, len(light_trace), 3 * budget))
    for d in (light, light_sync):
        d["offered_jobs_per_s"] = rate
        d["workload"] = desc
    return {"overloaded": over, "subsaturated": light, "subsaturated_host_waits": light_sync}


def main():
    args = parse()
    if args.record_counters:
        return record_counters(args.record_counters, args.counter_steps)
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "kernel":
        return run_kernel_mode(args)
    if args.mode == "kernel3":
        return run_kernel3_mode(args)
    if args.mode == "batch":
        return run_batch_mode(args)
    import numpy as np
    import torch
    from paper_2505_05919_gb300 import dist
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist.init()
    from paper_2505_05919_gb300 import Lattice, _capi, build as libbuild
    libbuild.build()
    _capi.load()

    cfgs = workload_configs(args.L)
    L, S = args.L, args.sweeps
    stream = torch.cuda.Stream()
    lats = []
    with torch.cuda.stream(stream):
        for c in cfgs:
            lats.append(Lattice(lib_params(c, seed_offset=dist.seed_offset(rank)), stream=stream))
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        dist.barrier()

    # warm-up (graphs instantiated here)
    for i in range(args.warmup):
        lats[i % len(lats)].sweep(S)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    t_wall0 = time.perf_counter()
    step_ms = []
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        lats[i % len(lats)].sweep(S)
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
    barrier()
    t_wall = time.perf_counter() - t_wall0
    clocks = sampler.stop()
    dev_s = dist.max_over_ranks(sum(step_ms) / 1e3)
    updates = 4.0 * L * L * S * args.steps * world
    value = updates / (dev_s * 1e9)
    obs = [l.observables() for l in lats]

    # dominant kernel: the sweep of the automatic configuration (at 4096^2
    # the wavefront, k_sweep_wave: one launch per call; the tiled sweep:
    # one launch per MC step); its time per MC step from CUDA events around
    # a 200-step call on the lattice's stream
    sw_ms = []
    lat = lats[1]
    wave = lat.tiles()[0] >= 4
    sweep_kernel = ("k_sweep_wave (one launch per call, the MC steps of the call in a wavefront)"
                    if wave else "k_sweep_tiled (one launch per MC step)")
    for _ in range(5):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        lat.sweep(200)
        ev1.record(stream)
        ev1.synchronize()
        sw_ms.append(ev0.elapsed_time(ev1) / 200)
    per_sweep_ms = statistics.median(sw_ms)
    peaks, peak_kind = measured_peaks()
    upd_per_s = 4.0 * L * L / (per_sweep_ms * 1e-3)
    ceiling, philox_ms = philox_ceiling(stream, L * L)
    args.philox_ceiling = ceiling
    counters = sweep_counters()
    achieved = upd_per_s / 1e9
    roofline = {"bound": "alu", "achieved": achieved, "peak": ceiling, "unit": "sigma-updates/ns",
                "frac": achieved / ceiling,
                "traffic": (counters["dram_bytes"] * (L / 4096.0) ** 2 if counters else None),
                "traffic_unit": "bytes per MC step (ncu dram read + write of the current kernel)",
                "kernel": sweep_kernel,
                "peak_kind": "measured: the step's Philox4x32-10 draws alone (cvf_philox_probe "
                             "over the same %d cells, %.1f us per step; four updates per block), "
                             "the random numbers every sweep of this method must make" % (L * L, philox_ms * 1e3)}
    bytes_per_sweep = 4.0 * L * L  # read 2 B + write 2 B per cell (1 B per sigma update)
    achieved_gbs = bytes_per_sweep / (per_sweep_ms * 1e-3) / 1e9
    roofline_hbm = {"bound": "hbm", "achieved": achieved_gbs, "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": achieved_gbs / peaks["hbm_gbs"],
                    "bytes_per_update": 1.0, "peak_kind": peak_kind}
    roofline_issue = None
    if counters:
        ipu = counters["instructions_per_update"]
        issued = ipu * upd_per_s / 1e12
        roofline_issue = {"bound": "issue", "achieved": issued, "peak": ISSUE_PEAK_T,
                          "unit": "T thread-instructions/s", "frac": issued / ISSUE_PEAK_T,
                          "instructions_per_update": ipu,
                          "peak_kind": "derived: 152 SM x 128 thread-instructions per clock x 2070 MHz",
                          "instructions_source": "ncu smsp__inst_executed.sum of one launch of the "
                                                 "current kernel per MC step "
                                                 "(profiles/k_sweep_wave_L4096_counters.json)"}
    # the 32 MB state stays in L2 across steps: the byte roofline that
    # bounds it is the L2 copy bandwidth, measured here with the library's
    # own copy kernel on the same working-set size (and, for reference, on
    # buffers 16x the L2, beside the measured HBM copy peak)
    state_bytes = 2 * L * L
    l2_gbs = copy_bandwidth_gbs(stream, state_bytes, 400)
    dram_gbs = copy_bandwidth_gbs(stream, 1 << 31, 6)
    roofline_l2 = {"bound": "l2", "achieved": achieved_gbs, "peak": l2_gbs, "unit": "GB/s",
                   "frac": achieved_gbs / l2_gbs, "bytes_per_update": 1.0,
                   "peak_kind": "measured: cvf_copy_probe (16-byte copy kernel) between two "
                                "L2-resident %d MiB buffers, 400 copies" % (state_bytes >> 20),
                   "dram_copy_gbs": dram_gbs,
                   "dram_copy_kind": "same kernel between two 2 GiB buffers, 6 copies"}

    # end to end through the C ABI with host buffers
    e2e_ms = []
    # pinned host buffers (the contract's end-to-end copies)
    host_in = torch.empty((L, L), dtype=torch.int16, pin_memory=True).numpy().view(np.uint16)
    host_out = torch.empty((L, L), dtype=torch.int16, pin_memory=True).numpy().view(np.uint16)
    lat = lats[1]
    host_in[:] = lat.state()
    V0 = lat.observables()["V_iso"]
    for i in range(max(2, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.set_state(host_in, V0, 0)
        lat.sweep(S)
        _capi.cvf_get_state(lat.h, host_out.ctypes.data, L * L)
        o = lat.observables()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_s = statistics.median(e2e_ms) / 1e3
    e2e = {"value": 4.0 * L * L * S / (e2e_s * 1e9), "unit": UNIT,
           "h2d_bytes_per_step": 2 * L * L, "d2h_bytes_per_step": 2 * L * L + 96}

    cubic = measure_cubic(args, rank, world) if args.cubic_sweeps > 0 else None
    order = measure_order_parameter(rank) if args.cubic_sweeps > 0 else None
    small = measure_small_configs(rank)
    batched = measure_batched(args, rank) if args.batch_sweeps > 0 else None
    serving = measure_serving(args, rank) if args.serve_seconds > 0 else None

    line = None
    if rank == 0:
        cpu = cpu_all = None
        if not args.no_cpu_baseline and world == 1:
            try:
                cpu = cpu_baseline(cfgs[1], args.cpu_sample_sweeps)
            except Exception as e:  # the baseline never blocks the line
                cpu = {"value": None, "error": str(e)}
            try:
                cpu_all = cpu_baseline_all_cores(cfgs[1])
            except Exception as e:
                cpu_all = {"value": None, "error": str(e)}
            try:
                for k, v in cpu_small_configs().items():
                    small[k]["oracle"] = v
            except Exception as e:
                small["oracle_error"] = str(e)
        # k_set_record per call, then one k_sweep_wave launch per call or one
        # k_sweep_tiled launch per MC step (the volume move runs inside it)
        launches_per_call = 2 if wave else S + 1
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dev_s * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u16+int64+f64", "data": "synthetic",
            "config": arm_config(L, S),
            "roofline": roofline,
            "roofline_hbm": roofline_hbm,
            "roofline_l2": roofline_l2,
            "roofline_issue": roofline_issue,
            "cpu_baseline": cpu,
            "cpu_baseline_all_cores": cpu_all,
            "e2e": e2e,
            "gpu_launches": args.steps * launches_per_call,
            "batched": batched,
            "serving": serving,
            "cubic": cubic,
            "order_parameter_3d": order,
            "small_configs": small,
            "clocks": clocks,
            "wall_s": t_wall,
            "per_sweep_ms": per_sweep_ms,
            "acceptance": [o["acc_sigma"] / max(1, 4 * L * L * o["sweep"]) for o in obs],
        }
        print(json.dumps(line))
    for l in lats:
        l.close()
    dist.finalize()
    return 0


if __name__ == "__main__":
    sys.exit(main())
