"""Benchmark of the GB300 LBGK library: MLUPS and HBM-roofline fraction of the fused step.

python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Workloads (synthetic, shaped like the paper's cases):
  beam1024x1[-f16|-bf16]  the tau*omega = 1 instance of beam1024 alone (profiling).
  beam1024  D2Q37, 4th-order equilibrium, regularized collision, FP32 storage: a 32 x 32 beam
            section centred in a 1024^2 periodic box, body-frame drive, three instances at
            tau*omega = 0.01, 1, 10 (default).  One bench step advances every instance by one
            lattice step (one fused kernel launch each).  The same run adds the rest of the metric
            as extra keys: the 64-instance sweep in FP32 (one persistent launch) and in FP16 (both
            batch modes), the 2048^2 precision study, and the served FP16 request stream (saturated,
            at 70 % load, and its D2Q9 requests alone) with p50/p99 latency.
  plate9    D2Q9 plain BGK, FP64: the 4 x 256 oscillating plate (latency-bound correctness case).
  plate9-2048[-f16|-bf16]  a D2Q9 regularized plate in a 2048^2 box at tau*omega = 0.3 (the largest
            D2Q9 request shape of the served stream; profiling).
  beam2048-<f32|f16|bf16|f64>  D2Q37-H4 beam in a 2048^2 box, tau*omega = 0.1, 1, 10.
  serve[-f16]  the serving loop: the first --requests requests of the seeded request stream (plate
            or beam, AR 0.25..4, tau*omega 1e-3..1e3, sides 128..2048, 10..50 periods, D2Q9 or
            D2Q37), submitted at Poisson arrival times; --load sets the offered load as a fraction of
            the GPU's capacity (estimated from the requests' algorithmic bytes at 0.8 of the measured
            HBM bandwidth), 0 submits at the stream's own rate (50 per second).  Reports aggregate
            MLUPS and p50/p99 latency (submit -> fit available).
  precision2048  precision study: the 2048^2 beam in FP64/FP32/FP16/BF16 storage, force errors
            against the FP64-storage run and MLUPS of each (prints its own JSON line).
  sweep64[-f16|-bf16]  the batched sweep: 64 D2Q37-H4 beam instances (16 tau*omega x 4 AR, sides
            256..1024) in one batch; a bench step is one batch step of all of them; with
            --batch-mode 1, runs of --chunk steps are single launches of the persistent kernel.

Each rank (torchrun, one per GPU) runs its own replicas: the instances are independent, so the
work is sharded with no collective on the data path (weak scaling).  One JSON line is printed by
rank 0.  `--impl reference` times the FP64 CPU oracle on the host cores for the same workload and
metric on a bounded sample (whole lattice, a few steps).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

STORE = {"f64": 0, "f32": 1, "bf16": 2, "f16": 3}

# The metric of the default workload, printed by both arms (this library and the FP64 oracle).
HEADLINE_METRIC = "MLUPS and % HBM roofline, batched mixed-prec vs plain FP32 at <=1e-4 force err; p99 latency"
SUB_METRIC = "MLUPS (fluid lattice updates per second, whole job) and HBM-roofline fraction of the fused step"


def metric_name(workload):
    return HEADLINE_METRIC if workload == "beam1024" else SUB_METRIC


def kernel_source_hash():
    """Digest of the CUDA sources and the C ABI header: the DRAM traffic recorded below is valid
    only for the sources it was captured from."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_0904_4504_gb300", "csrc")
    names = sorted(n for n in os.listdir(csrc) if n.endswith((".cu", ".cuh", ".h")))
    for n in names:
        h.update(n.encode())
        with open(os.path.join(csrc, n), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(ROOT, "include", "lbm.h"), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()[:16]


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the step kernels, from one
# ncu capture each, with the digest of the sources they were captured from: once any source
# changes, the entry no longer applies and the line reports traffic null.
TRAFFIC = {
    ("beam1024", 1): (263564288, "6cb49ca6ec672d3b"),          # 156.4 MB read + 107.2 MB written
    ("beam1024x1-f16", 26): (109641984, "6cb49ca6ec672d3b"),   # 78.8 + 30.8 MB
    ("beam1024x1-f16", 27): (109117184, "6cb49ca6ec672d3b"),   # 78.8 + 30.3 MB
}


def traffic_for(workload, variant):
    e = TRAFFIC.get((workload, variant))
    if e is None or e[1] != kernel_source_hash():
        return None
    return e[0]
# Thread instructions per fluid node (smsp__inst_executed.sum x 32 / fluid nodes) of the 16-bit step
# kernel, from the same kind of capture and with the same digest rule: with 16-bit storage the step
# is bound by instruction issue, so the batched line also reports the issue rate against the SMs'
# issue peak.
INST_PER_NODE = {
    ("beam1024", 1): (739.3, "6cb49ca6ec672d3b"),              # 24,202,187 warp instructions, 1,047,552 fluid nodes
    ("beam1024x1-f16", 26): (770.8, "6cb49ca6ec672d3b"),       # 25,232,720
    ("beam1024x1-f16", 27): (763.4, "6cb49ca6ec672d3b"),       # 24,990,376
}


def inst_per_node(workload, variant):
    e = INST_PER_NODE.get((workload, variant))
    if e is None or e[1] != kernel_source_hash():
        return None
    return e[0]


DTYPE_NAME = {0: "f64", 1: "f32", 2: "bf16", 3: "f16"}


def tune_cache_path():
    """JSON cache of the batch autotuner for this machine's runs (a fresh box tunes once)."""
    import tempfile
    return os.path.join(tempfile.gettempdir(), "lbm_gb300_bench_tune.json")


def workload_list(name):
    from paper_0904_4504_gb300 import inputs as I
    if name == "beam1024":
        return [I.beam_d2q37_h4(to) for to in I.BEAM_TAU_OMEGAS]
    if name.startswith("beam1024x1"):
        st = STORE[name.split("-")[1]] if "-" in name else STORE["f32"]
        return [I.beam_d2q37_h4(1.0, storage=st)]
    if name == "plate9":
        return [I.plate_d2q9_fp64()]
    if name.startswith("plate9-2048"):
        # the largest D2Q9 request shape of the served stream: a 2048^2 plate, regularized, moving wall
        st = STORE[name.split("-")[2]] if name.count("-") == 2 else STORE["f32"]
        return [I.Workload("plate-d2q9-2048", 9, 2048, 2048, 0.3, I.PLATE, drive=I.DRIVE_WALL, u0=1e-3, eq_order=2,
                           collision=I.REG, storage=st, periods=10.0)]
    if name.startswith("beam2048-"):
        st = STORE[name.split("-")[1]]
        return [I.beam_d2q37_h4(to, n=2048, storage=st) for to in I.PRECISION_TAU_OMEGAS]
    raise SystemExit(f"unknown workload {name}")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples (100 ms) while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_setup(n_gpus):
    import torch
    from paper_0904_4504_gb300.replicas import env_rank
    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    from paper_0904_4504_gb300.replicas import barrier as b
    b(world)


def max_over_ranks(x, world):
    from paper_0904_4504_gb300.replicas import max_over_ranks as m
    return m(x, world, device="cuda")


LAYOUT = {"ab": 0, "aa": 1}


def create(L, w, orc_params, layout="ab"):
    tau, omega = orc_params(w)
    geom = L.make_geometry(kind=w.geometry, lx=w.lx, ly=w.ly, drive=w.drive, u0=w.u0, eq_order=w.eq_order,
                           collision=w.collision, storage=w.storage, layout=LAYOUT[layout])
    return L.lbm_create(w.lattice, w.nx, w.ny, tau, omega, geom)


def lattice_params(L):
    def f(w):
        if w.tau is not None:
            return w.tau, w.omega
        tau, omega, _ = L.lbm_params_from_tau_omega(w.lattice, w.tau_omega)
        return tau, omega
    return f


def sweep_descs(L, storage, layout="ab"):
    from paper_0904_4504_gb300 import inputs as I
    out = []
    for w in I.sweep_d2q37():
        tau, omega, P = L.lbm_params_from_tau_omega(37, w.tau_omega)
        out.append((w, L.make_instance(37, w.nx, w.ny, tau, omega, int(w.periods * P), kind=w.geometry, lx=w.lx,
                                       ly=w.ly, drive=w.drive, u0=w.u0, eq_order=w.eq_order, collision=w.collision,
                                       storage=storage, layout=LAYOUT[layout])))
    return out


def issue_roofline(bl):
    """Warp instructions issued per second by the 16-bit step kernel of a batch line against the
    SMs' issue peak (4 schedulers per SM, one warp instruction per scheduler per cycle, at the
    median SM clock sampled during the run); None without a captured instruction count."""
    import torch
    ipn = inst_per_node("beam1024x1-f16", bl["config"].get("kernel_variant"))
    mhz = (bl.get("clocks") or {}).get("sm_mhz")
    if not ipn or not mhz:
        return None
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    achieved = bl["value"] * 1e6 * ipn / 32 / 1e9
    peak = sms * 4 * mhz * 1e6 / 1e9
    return {"bound": "alu", "inst_per_node": ipn, "achieved": round(achieved, 1), "peak": round(peak, 1),
            "unit": "G warp-instructions/s", "frac": round(achieved / peak, 4),
            "peak_source": f"{sms} SMs x 4 schedulers x 1 warp instruction per cycle x {mhz:g} MHz (median SM clock "
                           "of the run)",
            "inst_source": "ncu smsp__inst_executed.sum of the kernel on one 1024^2 beam instance"}


def run_batch(args, sub=False):
    import torch
    from paper_0904_4504_gb300 import lbm as L
    from paper_0904_4504_gb300.builder import build

    from paper_0904_4504_gb300.replicas import env_rank
    rank, world, local = env_rank() if sub else dist_setup(args.gpus)
    build()
    storage = STORE[args.workload.split("-")[1]] if "-" in args.workload else STORE["f32"]
    descs = sweep_descs(L, storage, args.layout)[:args.instances or None]
    stream = torch.cuda.Stream()
    b = L.lbm_batch_create(37, storage, 1)
    L.lbm_batch_set_mode(b, args.batch_mode)
    if args.batch_variant is not None:
        L.lbm_batch_set_variant(b, args.batch_variant)
    if args.batch_segment:
        L.lbm_batch_set_segment(b, args.batch_segment)
    tuned = None
    if args.batch_autotune:
        from paper_0904_4504_gb300 import autotune as A
        t0 = time.perf_counter()
        tuned = A.tune_batch(b, [d for _, d in descs], tune_cache_path(), steps=8)
        tuned = dict(tuned, tune_s=round(time.perf_counter() - t0, 2))
    L.lbm_batch_set_stream(b, stream)
    slots = [L.lbm_batch_add(b, d) for _, d in descs]
    info0 = L.lbm_batch_info(b)
    fluid, bytes_step = info0["fluid_running"], info0["bytes_per_step"]
    # the step kernel the instances run (streams mode: chosen per instance at admission)
    used = sorted({L.lbm_info(L.lbm_batch_instance(b, k))["variant"] for k in slots})

    def run(n):
        left = n
        while left > 0:
            k = min(args.chunk, left)
            L.lbm_batch_run(b, k)
            left -= k

    run(args.warmup)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    l0 = L.lbm_batch_info(b)["launches"]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        ev0.record(stream)
        run(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    L.lbm_batch_synchronize(b)
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ms, world)
    info = L.lbm_batch_info(b)
    launches = info["launches"] - l0
    assert info["running"] == len(descs), "an instance finished inside the timed region"
    L.lbm_batch_destroy(b)
    value = fluid * args.steps * world / (ms_max * 1e-3) / 1e6
    peak, peak_kind = peaks()
    achieved = bytes_step * args.steps / (ms * 1e-3) / 1e9

    e2e = None
    if not args.no_e2e:
        # end to end through the C ABI: batch create + 64 x (geometry, upload) -> K steps -> 64 force
        # histories (D2H) -> 64 fits
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b = L.lbm_batch_create(37, storage, 1)
        L.lbm_batch_set_mode(b, args.batch_mode)
        if args.batch_variant is not None:
            L.lbm_batch_set_variant(b, args.batch_variant)
        if args.batch_segment:
            L.lbm_batch_set_segment(b, args.batch_segment)
        if args.batch_autotune:
            from paper_0904_4504_gb300 import autotune as A
            A.tune_batch(b, [d for _, d in descs], tune_cache_path(), steps=8)   # the cached choice
        slots = [L.lbm_batch_add(b, d) for _, d in descs]
        run(args.steps)
        L.lbm_batch_synchronize(b)
        h2d = d2h = 0
        for sl in slots:
            sim = L.lbm_batch_instance(b, sl)
            d2h += L.lbm_force_history(sim).nbytes
            h2d += L.lbm_info(sim)["h2d_bytes"]
        L.lbm_batch_destroy(b)
        e2e_s = max_over_ranks(time.perf_counter() - t0, world)
        e2e = {"value": fluid * args.steps * world / e2e_s / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": int(h2d / args.steps), "d2h_bytes_per_step": int(d2h / args.steps),
               "scope": "lbm_batch_create + 64 lbm_batch_add (host geometry + upload) -> lbm_batch_run(K) -> "
                        "64 lbm_force_history"}
    if rank == 0:
        line = {
            "metric": metric_name(args.workload),
            "value": round(value, 3), "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms_max / args.steps, 6), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {v: k for k, v in STORE.items()}[storage], "data": "synthetic",
            "config": {"workload": args.workload, "instances": len(descs), "lattice": "D2Q37", "eq_order": 4,
                       "collision": "regularized", "fluid_nodes": fluid, "steps_per_launch": args.chunk,
                       "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{world}",
                       "batch_mode": "persistent" if info["mode"] == 1 else "streams",
                       "graph": bool(info["uses_graph"]), "grid_blocks": info["max_blocks"], "layout": args.layout,
                       "kernel_variant": used[0] if len(used) == 1 else used,
                       "strip_tile_rows": args.batch_segment or "library default",
                       "autotuned": tuned},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": args.traffic,
                         "peak_source": f"{peak_kind} hbm_gbs",
                         "kernel": "pbatch_kernel (persistent; strips of tiles as work items, per-band step "
                                   "counters, no grid barrier; one CUDA graph launch per run)" if info["mode"] == 1 else
                                   "step kernels of every instance on parallel streams",
                         "bytes_per_batch_step": bytes_step},
            "clocks": clocks.summary(), "e2e": e2e, "gpu_launches": launches, "cpu_baseline": None,
        }
        if sub:
            return line
        print(json.dumps(line), flush=True)
    if world > 1 and not sub:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_serve(args, sub=False):
    import torch
    from paper_0904_4504_gb300 import inputs as I
    from paper_0904_4504_gb300 import lbm as L
    from paper_0904_4504_gb300.builder import build

    from paper_0904_4504_gb300.replicas import env_rank
    rank, world, local = env_rank() if sub else dist_setup(args.gpus)
    build()
    storage = STORE["f16"] if args.workload.endswith("-f16") else STORE["f32"]
    from paper_0904_4504_gb300.replicas import rank_slice
    reqs_all = I.serving_requests()
    if args.serve_lattice:
        reqs_all = [r for r in reqs_all if r.workload.lattice == args.serve_lattice]
    stream = rank_slice(reqs_all, rank, args.requests)
    reqs, gpu_s = [], []
    peak, peak_kind = peaks()
    for r in stream:
        w = r.workload
        tau, omega, P = L.lbm_params_from_tau_omega(w.lattice, w.tau_omega)
        nsteps = int(round(w.periods * P))
        d = L.make_instance(w.lattice, w.nx, w.ny, tau, omega, nsteps, kind=w.geometry, lx=w.lx, ly=w.ly,
                            drive=w.drive, u0=w.u0, eq_order=w.eq_order, collision=w.collision, storage=storage,
                            layout=LAYOUT[args.layout])
        perim = 2.0 * (w.lx + w.ly) if w.geometry == 1 else float(w.nx)
        reqs.append((r.arrival_s, L.make_request(d, w.periods / 2.0, perim)))
        bytes_lu = 2 * w.lattice * L.STORAGE_BYTES[storage]
        gpu_s.append(w.nx * w.ny * nsteps * bytes_lu / (0.8 * peak * 1e9))
    if args.load > 0:   # rescale the arrival process to the requested offered load
        rate = args.load / (sum(gpu_s) / len(gpu_s))
        arrivals = np.cumsum(np.random.default_rng(I.SERVE_SEED + 1).exponential(1.0 / rate, len(reqs)))
    else:
        arrivals = np.array([a for a, _ in reqs]) - reqs[0][0]
    srv = L.lbm_server_create(int(args.serve_budget_gb * 1e9), args.chunk)
    L.lbm_server_set_batch_mode(srv, args.batch_mode)
    tuned = None
    if args.batch_autotune:
        # each request class's kernel, chosen by the batch autotuner on a sample of the class's
        # requests before the first submit (outside the timed region)
        from paper_0904_4504_gb300 import autotune as A
        t0 = time.perf_counter()
        ch = A.tune_server(srv, [rq for _, rq in reqs], tune_cache_path(), steps=4, sample=8, mode=args.batch_mode)
        tuned = {f"Q{k[0]}-st{k[1]}-coll{k[2]}": v for k, v in ch.items()}
        tuned["tune_s"] = round(time.perf_counter() - t0, 2)
    ids = []
    torch.cuda.synchronize()
    barrier(world)
    with ClockSampler(local) as clocks:
        t0 = time.perf_counter()
        for (_, rq), at in zip(reqs, arrivals):
            dt = at - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            ids.append(L.lbm_server_submit(srv, rq))
        results = []
        for i in ids:
            done, res = L.lbm_server_wait(srv, i, 3600.0)
            results.append(res)
        makespan = time.perf_counter() - t0
    stats = L.lbm_server_stats(srv)
    L.lbm_server_destroy(srv)
    barrier(world)
    lat = np.array([r["done_s"] - r["submit_s"] for r in results])
    ok = all(r["status"] == 2 for r in results)
    lu = sum(r["steps"] * r["fluid_nodes"] for r in results)
    # algorithmic bytes: one read and one write of every population of every fluid node per step
    nbytes = sum(r["steps"] * r["fluid_nodes"] * 2 * q.workload.lattice * L.STORAGE_BYTES[storage]
                 for r, q in zip(results, stream))
    span = max_over_ranks(makespan, world)
    value = lu * world / span / 1e6
    achieved = nbytes * world / span / 1e9
    if rank == 0:
        line = {
            "metric": "aggregate MLUPS of the served requests (fluid lattice updates per second, submit of the first "
                      "to completion of the last) and p50/p99 latency",
            "value": round(value, 3), "unit": "MLUPS", "n_gpus": world, "steps": stats["rounds"], "warmup": 0,
            "ms_per_step": round(span * 1e3 / max(1, stats["rounds"]), 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {v: k for k, v in STORE.items()}[storage],
            "data": "synthetic",
            "config": {"workload": args.workload, "requests": len(reqs), "offered_load": args.load or "as generated",
                       "lattices": args.serve_lattice or "D2Q9 and D2Q37",
                       "budget_gb": args.serve_budget_gb or "server default",
                       "steps_per_round": args.chunk, "parallelism": f"replicas x{world}", "layout": args.layout,
                       "autotuned": tuned},
            "latency": {"p50_s": round(float(np.percentile(lat, 50)), 4),
                        "p99_s": round(float(np.percentile(lat, 99)), 4), "mean_s": round(float(lat.mean()), 4),
                        "max_s": round(float(lat.max()), 4)},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": None, "peak_source": f"{peak_kind} hbm_gbs",
                         "kernel": "step kernels of the running requests; the makespan (first submit to last "
                                   "completion) includes the ramp and the tail",
                         "bytes": nbytes},
            "server": {"completed": stats["completed"], "all_ok": ok, "busy_frac": round(stats["busy_s"] / span, 4),
                       "peak_running": stats["peak_running"], "peak_used_gb": round(stats["peak_used_bytes"] / 1e9, 3),
                       "total_lattice_updates": lu, "makespan_s": round(span, 3)},
            "clocks": clocks.summary(), "gpu_launches": None, "cpu_baseline": None,
        }
        if sub:
            return line
        print(json.dumps(line), flush=True)
    if world > 1 and not sub:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_precision(args, sub=False):
    """Precision study at full size: the D2Q37-H4 beam in 2048^2 at tau*omega = 0.1, 1, 10 for 30
    periods in every storage type; in-phase/quadrature force error of each against the FP64-storage
    run (the FP64 oracle comparison on the 256^2 downscale is tests/test_gpu_precision.py)."""
    import torch
    from paper_0904_4504_gb300 import inputs as I
    from paper_0904_4504_gb300 import lbm as L
    from paper_0904_4504_gb300.builder import build
    from paper_0904_4504_gb300.replicas import env_rank

    rank, world, local = env_rank() if sub else dist_setup(args.gpus)
    build()
    stream = torch.cuda.Stream()
    out = []
    for to in I.PRECISION_TAU_OMEGAS:
        tau, omega, P = L.lbm_params_from_tau_omega(37, to)
        steps = 30 * P
        fits = {}
        for name in ("f64", "f32", "f16", "bf16"):
            w = I.beam_d2q37_h4(to, n=2048, storage=STORE[name])
            geom = L.make_geometry(kind=w.geometry, lx=w.lx, ly=w.ly, drive=w.drive, u0=w.u0, eq_order=4,
                                   collision=w.collision, storage=STORE[name])
            h = L.lbm_create(37, 2048, 2048, tau, omega, geom)
            L.lbm_set_stream(h, stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            L.lbm_step(h, steps)
            e1.record(stream)
            torch.cuda.synchronize()
            f_in, f_q, _ = L.lbm_fit(h, 15.0)
            info = L.lbm_info(h)
            ms = e0.elapsed_time(e1)
            fits[name] = (f_in, f_q, info["n_fluid"] * steps / (ms * 1e-3) / 1e6)
            L.lbm_destroy(h)
        amp = math.hypot(*fits["f64"][:2])
        row = {"tau_omega": to, "steps": steps, "F_in_f64": fits["f64"][0], "F_q_f64": fits["f64"][1]}
        for name in ("f32", "f16", "bf16"):
            row[f"err_in_{name}"] = abs(fits[name][0] - fits["f64"][0]) / amp
            row[f"err_q_{name}"] = abs(fits[name][1] - fits["f64"][1]) / amp
        for name in fits:
            row[f"mlups_{name}"] = round(fits[name][2], 1)
        out.append(row)
    line = {"study": "precision", "workload": "D2Q37-H4 regularized beam 32x32 in 2048^2, body-frame drive U0=1e-3, "
            "30 periods, fit after 15; force errors (in-phase, quadrature) of FP32/FP16/BF16 storage against the "
            "FP64-storage run, normalized by the FP64 force amplitude; FP32 arithmetic, FP64 force sums",
            "rows": out,
            "max_err": {name: max(max(r[f"err_in_{name}"], r[f"err_q_{name}"]) for r in out)
                        for name in ("f32", "f16", "bf16")}}
    if sub:
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_ours(args):
    if args.workload == "precision2048":
        return run_precision(args)
    if args.workload.startswith("serve"):
        return run_serve(args)
    if args.workload.startswith("sweep64"):
        return run_batch(args)
    import torch
    from paper_0904_4504_gb300 import lbm as L
    from paper_0904_4504_gb300.builder import build

    rank, world, local = dist_setup(args.gpus)
    build()
    wl = workload_list(args.workload)
    params = lattice_params(L)
    stream = torch.cuda.Stream()
    sims = []
    for w in wl:
        h = create(L, w, params, args.layout)
        L.lbm_set_stream(h, stream)
        if args.tile:
            L.lbm_set_tile(h, *args.tile)
        if args.variant is not None:
            L.lbm_set_variant(h, args.variant)
        sims.append(h)
    infos = [L.lbm_info(h) for h in sims]
    fluid = sum(i["n_fluid"] for i in infos)
    bytes_step = sum(i["bytes_per_step"] for i in infos)

    for _ in range(args.warmup):
        for h in sims:
            L.lbm_step(h, 1)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        ev0.record(stream)
        for _ in range(args.steps):
            for h in sims:
                L.lbm_step(h, 1)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ms, world)
    for h in sims:
        L.lbm_synchronize(h)
    launches = args.steps * len(sims)
    value = fluid * args.steps * world / (ms_max * 1e-3) / 1e6

    # dominant kernel: the fused step (one launch per instance per step)
    peak, peak_kind = peaks()
    per_launch_s = ms * 1e-3 / launches
    achieved = bytes_step / len(sims) / per_launch_s / 1e9

    # end to end through the C ABI: create (geometry upload) -> K steps -> force history (D2H) -> fit
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2d = d2h = 0
        for w in wl:
            h = create(L, w, params, args.layout)
            L.lbm_step(h, args.steps)
            F = L.lbm_force_history(h)
            d2h += F.nbytes
            h2d += L.lbm_info(h)["h2d_bytes"]
            L.lbm_destroy(h)
        t1 = time.perf_counter()
        e2e_s = max_over_ranks(t1 - t0, world)
        e2e = {"value": fluid * args.steps * world / e2e_s / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": int(h2d / args.steps), "d2h_bytes_per_step": int(d2h / args.steps),
               "scope": "lbm_create (host geometry + upload) -> lbm_step(K) -> lbm_force_history"}
    for h in sims:
        L.lbm_destroy(h)

    cpu = cpu_baseline(wl, params, args) if (rank == 0 and world == 1 and not args.no_cpu) else None
    extras = {}
    if args.workload == "beam1024" and not args.no_extras:
        # the rest of the metric: the batched forms (FP32 as one persistent launch; mixed precision
        # -- FP16 storage, FP32 arithmetic, FP64 force -- in both batch modes) against this plain
        # FP32 single-instance form, the precision study at 2048^2, and the served mixed-precision
        # stream with its p50/p99 latency
        import copy

        def batch_line(workload, mode, chunk, steps):
            a = copy.copy(args)
            a.workload, a.steps, a.warmup, a.no_e2e, a.batch_mode, a.chunk = workload, steps, 3, True, mode, chunk
            a.batch_variant, a.batch_segment, a.instances = None, 0, 0
            return run_batch(a, sub=True)

        def serve_line(requests, load, lattice):
            a = copy.copy(args)
            a.workload, a.requests, a.load, a.serve_budget_gb, a.serve_lattice = "serve-f16", requests, load, 6.0, lattice
            return run_serve(a, sub=True)

        b32 = batch_line("sweep64", 1, args.sweep_steps, args.sweep_steps)
        b16 = batch_line("sweep64-f16", 0, 64, args.sweep_steps)
        p16 = batch_line("sweep64-f16", 1, 64, args.sweep_steps)
        prec = run_precision(args, sub=True) if not args.no_precision else None
        sm = serve_line(args.requests, 0.0, 0)
        s70 = serve_line(max(1, args.requests // 2), 0.7, 0)
        s9 = serve_line(max(1, args.requests // 2), 0.0, 9)
        if rank == 0:
            def keep(line, *keys):
                return {k: line[k] for k in keys if k in line}
            extras["batched_fp32_persistent"] = dict(
                keep(b32, "value", "unit", "steps", "ms_per_step", "roofline", "clocks", "gpu_launches", "config"),
                workload="sweep64: 64 D2Q37-H4 beam instances (16 tau*omega x 4 AR, sides 256..1024), FP32, all "
                         "timed steps in one launch of the persistent kernel through a CUDA graph",
                speedup_vs_plain_fp32=round(b32["value"] / value, 4))
            extras["batched_mixed_precision"] = dict(
                keep(b16, "value", "unit", "steps", "ms_per_step", "roofline", "clocks", "gpu_launches", "config"),
                workload="sweep64-f16: the same 64 instances, streams mode (one launch of the staged step kernel "
                         "per instance per step, on 16 parallel streams), FP16 storage scaled by U0, FP32 "
                         "arithmetic, FP64 force",
                speedup_vs_plain_fp32=round(b16["value"] / value, 4), issue=issue_roofline(b16),
                force_error_vs_oracle="FP16 storage <= 1.6e-5 of the force amplitude (in-phase and quadrature, body "
                                      "and lab frame, tests/test_gpu_precision.py); target 1e-4")
            extras["batched_mixed_precision_persistent"] = dict(
                keep(p16, "value", "unit", "steps", "ms_per_step", "roofline", "clocks", "gpu_launches", "config"),
                workload="sweep64-f16 in the persistent mode: one launch per 64 steps of the persistent kernel "
                         "(staged 64 x 3 tiles, work items of one tile column x 8 tile rows) through a CUDA graph",
                speedup_vs_plain_fp32=round(p16["value"] / value, 4))
            if prec is not None:
                extras["precision_study"] = prec
            extras["serving_mixed_precision_saturated"] = keep(sm, "value", "unit", "config", "roofline", "latency",
                                                               "server", "clocks")
            extras["serving_mixed_precision_70pct"] = keep(s70, "value", "unit", "config", "roofline", "latency",
                                                           "server", "clocks")
            extras["serving_d2q9_saturated"] = keep(s9, "value", "unit", "config", "roofline", "latency", "server",
                                                    "clocks")
    if rank == 0:
        w0 = wl[0]
        line = {
            "metric": metric_name(args.workload),
            "value": round(value, 3), "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms_max / args.steps, 6), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE_NAME[w0.storage], "data": "synthetic",
            "config": {"workload": args.workload, "instances": [w.name for w in wl], "lattice": f"D2Q{w0.lattice}",
                       "eq_order": w0.eq_order, "collision": "regularized" if w0.collision == 1 else "bgk",
                       "nodes_per_instance": [w.nx * w.ny for w in wl], "fluid_nodes": fluid,
                       "l2": "inputs larger than L2 (no flush)" if bytes_step / len(wl) > 2 * 129e6 else
                             "inputs smaller than L2", "parallelism": f"replicas x{world}",
                       "tile": [infos[0]["block_x"], infos[0]["block_y"]], "variant": infos[0]["variant"],
                       "layout": args.layout},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4),
                         "traffic": args.traffic if args.traffic is not None else
                         traffic_for(args.workload, infos[0]["variant"]) if args.layout == "ab" else None,
                         "peak_source": f"{peak_kind} hbm_gbs", "kernel": "fused stream+collide+force step (kernel variant in config)",
                         "bytes_per_launch": bytes_step // len(wl)},
            "clocks": clocks.summary(), "e2e": e2e, "gpu_launches": launches, "cpu_baseline": cpu,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def cpu_baseline(wl, params, args, budget_s=15.0):
    """The FP64 oracle on the host cores: whole-lattice steps of the first instance until about
    budget_s of CPU work."""
    import oracle as orc
    w = wl[0]
    tau, omega = params(w)
    lab = {0: lambda: orc.geometry_plate(w.lattice, w.nx, w.ny), 1: lambda: orc.geometry_beam(w.nx, w.ny, w.lx, w.ly)}[
        w.geometry]()
    nt = orc.max_threads()
    f = orc.rest_state(w.lattice, w.nx, w.ny)
    steps, t_used = 0, 0.0
    while t_used < budget_s and steps < 10000:
        n = 1 if w.nx * w.ny > 1e5 else 200
        t0 = time.perf_counter()
        f, _ = orc.run(w.lattice, lab, tau, omega, w.u0, n, eq_order=w.eq_order, collision=w.collision, drive=w.drive,
                       f=f, n0=steps, nthreads=nt)
        t_used += time.perf_counter() - t0
        steps += n
    fluid = int((lab == 0).sum())
    return {"value": round(fluid * steps / t_used / 1e6, 4), "unit": "MLUPS", "cores": nt, "kind": "oracle",
            "sample": f"{steps} whole-lattice steps of {w.name} ({fluid} fluid nodes), FP64, {nt} OpenMP threads"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = workload_list(args.workload)
    import oracle as orc

    def params(w):
        if w.tau is not None:
            return w.tau, w.omega
        t, o, _ = orc.params_from_tau_omega(w.lattice, w.tau_omega)
        return t, o

    orc.build()
    nt = orc.max_threads()
    labs = [{0: lambda w=w: orc.geometry_plate(w.lattice, w.nx, w.ny),
             1: lambda w=w: orc.geometry_beam(w.nx, w.ny, w.lx, w.ly)}[w.geometry]() for w in wl]
    states = [orc.rest_state(w.lattice, w.nx, w.ny) for w in wl]
    fluid = [int((lab == 0).sum()) for lab in labs]

    def one(step_idx):
        k = step_idx % len(wl)
        w = wl[k]
        tau, omega = params(w)
        states[k], _ = orc.run(w.lattice, labs[k], tau, omega, w.u0, 1, eq_order=w.eq_order, collision=w.collision,
                               drive=w.drive, f=states[k], n0=step_idx // len(wl), nthreads=nt)
        return fluid[k]

    for s in range(args.warmup):
        one(s)
    t0 = time.perf_counter()
    done = 0
    for s in range(args.steps):
        done += one(args.warmup + s)
    dt = time.perf_counter() - t0
    v = done / dt / 1e6
    w0 = wl[0]
    print(json.dumps({
        "impl": "reference", "metric": metric_name(args.workload),
        "value": round(v, 4), "unit": "MLUPS", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "instances": [w.name for w in wl], "lattice": f"D2Q{w0.lattice}"},
        "cpu_baseline": {"value": round(v, 4), "unit": "MLUPS", "cores": nt, "kind": "oracle",
                         "sample": f"one whole-lattice step of one instance per bench step (instances in turn), "
                                   f"FP64 oracle, {nt} OpenMP threads"},
        "e2e": {"value": round(v, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="beam1024")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tile", type=int, nargs=2, default=None)
    ap.add_argument("--variant", type=int, default=None, help="step kernel variant (lbm_set_variant)")
    ap.add_argument("--layout", default="ab", choices=["ab", "aa"],
                    help="population layout: two buffers (ab) or one buffer updated in place (aa)")
    ap.add_argument("--chunk", type=int, default=64, help="batch steps per persistent launch (sweep64, serve)")
    ap.add_argument("--requests", type=int, default=400,
                    help="requests per rank (serve; the default workload's saturated serving line; its 70%%-load and "
                         "D2Q9 lines take half as many)")
    ap.add_argument("--serve-lattice", type=int, default=0, choices=[0, 9, 37],
                    help="serve: only the requests of this lattice (0: all)")
    ap.add_argument("--serve-budget-gb", type=float, default=0.0,
                    help="serve: device memory the server may give to resident lattices (0: its default)")
    ap.add_argument("--load", type=float, default=0.7, help="offered load, fraction of capacity (serve; 0: as generated)")
    ap.add_argument("--sweep-steps", type=int, default=640, help="timed batch steps of the batched part of beam1024")
    ap.add_argument("--no-extras", action="store_true", help="beam1024: skip the batched and serving parts")
    ap.add_argument("--no-precision", action="store_true", help="beam1024: skip the 2048^2 precision study")
    ap.add_argument("--instances", type=int, default=0, help="sweep64: use only the first N instances (profiling)")
    ap.add_argument("--batch-mode", type=int, default=0,
                    help="sweep64 and serve: 0 parallel streams, 1 the persistent kernel")
    ap.add_argument("--batch-variant", type=int, default=None, help="sweep64: step kernel of the streams mode")
    ap.add_argument("--batch-autotune", type=int, default=1,
                    help="sweep64/serve: choose the batch kernels with the batch autotuner (JSON cache in the temp "
                         "dir) before the timed region (1) or use the library's defaults (0)")
    ap.add_argument("--batch-segment", type=int, default=0,
                    help="sweep64, persistent mode: tile rows per work item (strip; 0: the library's default)")
    ap.add_argument("--traffic", type=float, default=None, help="ncu DRAM bytes per launch of the step kernel")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end C-ABI run (profiling runs)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
