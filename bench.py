#!/usr/bin/env python
"""Throughput benchmark of the CCPR time-domain adjoint gradient on GB300.

One benchmark step = one gradient evaluation of the whole hot path: forward Yee/CPML/CCPR run
with the running DFT, adjoint run, and dF/drho over the design box.  Metric: Gcell-updates/s =
2 * n_cells * n_time_steps / wall time per gradient.

Default workload (config 2 of the paper-shaped workloads): 256^3 grid, 12-cell CPML, 4000 time
steps, 128^3 design box with smooth seeded density blending air and a 3-pair CCPR metal,
3 objective frequencies (500/600/700 nm), TF/SF plane wave along x, FP32 fields with FP64 DFT.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent replica (the problem does not need a
collective); value = all ranks' cell-updates / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcell-updates/s Yee+CCPR fwd+adj FP32, % HBM roofline; p50/p99 grad latency"
UNIT = "Gcell-updates/s"
L2_BYTES = 129 * 2 ** 20


def parse(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c4", "f3_Au", "f3_Al", "f3_Si", "f3_TiO2"])
    ap.add_argument("--time-steps", type=int, default=0, help="override the workload's time steps")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-sample-steps", type=int, default=16,
                    help="time steps of the bounded oracle sample (CPU baseline / reference arm)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=200,
                    help="requests of the seeded serving stream (Poisson, 20 req/s) replayed after the throughput "
                         "run through the server and one after another (0: skip the serving leg)")
    ap.add_argument("--serving-load-requests", type=int, default=100,
                    help="requests of the same stream replayed again with arrivals slowed to about 0.7 of the "
                         "server's measured capacity (latency below saturation; 0: skip)")
    ap.add_argument("--serving-slots", type=int, default=16)
    ap.add_argument("--serving-batch-max-cells", type=int, default=0,
                    help="grids of at most this many cells take the batch lane (persistent kernel); -1: all; "
                         "0 (default): none")
    ap.add_argument("--serving-exclusive-cells", type=int, default=128 ** 3,
                    help="grids of at least this many cells run one at a time (0: strict FIFO, no limit)")
    ap.add_argument("--precision-study", action="store_true",
                    help="config 3: FP32 fields + FP64 DFT vs all-FP64 build; prints one JSON line")
    ap.add_argument("--filter", action="store_true",
                    help="time the density filter + projection and its chain rule on the workload's design box "
                         "(R = 12 cells, beta = 52, eta = 0.5); prints one JSON line")
    ap.add_argument("--paper-mode", action="store_true",
                    help="time the paper's time-domain gradient (checkpoint-recompute) on the workload; "
                         "prints one JSON line")
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ---------------------------------------------------------------------------------------------
def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init_dist(world, backend):
    if world <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def barrier(dist, device=None):
    if dist is None:
        return
    if device is not None:
        dist.barrier(device_ids=[device])
    else:
        dist.barrier()


def max_over_ranks(dist, value, device=None):
    """Max of a float over ranks (the job's wall time is its slowest rank's)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=f"cuda:{device}" if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value, device=None):
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=f"cuda:{device}" if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.idx)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------------------------
def cell_update_model(w, gcells, peak):
    """HBM fraction of the whole run under the per-cell-update byte count of the method (FP32 state
    words read once and written once per step, separate H and E passes): every cell 72 B (E, H r/w and
    the other field read once per half-step); per design voxel 4 (rho) + 48 P_tot (pole currents r/w)
    + 96 F (FP64 DFT accumulators r/w); per CPML slab cell and attenuated axis 32 B (two psi_E and two
    psi_H r/w).  fraction = Gcell-updates/s x bytes per cell-update / peak."""
    import synth
    d = w["desc"]
    ts = 4.0 if d["precision"] == 32 else 8.0
    n = (d["nx"], d["ny"], d["nz"])
    ncell = float(n[0] * n[1] * n[2])
    bs = synth.box_shape(d["design_box"])
    nd = float(bs[0] * bs[1] * bs[2]) if d["design_box"][1] > d["design_box"][0] else 0.0
    p_tot = sum(len(w["m1"]["poles"][k]) + len(w["m2"]["poles"][k]) for k in range(3)) / 3.0
    slab = sum((d["cpml"][2 * a] + d["cpml"][2 * a + 1]) / n[a] for a in range(3))
    b = 18.0 * ts + nd / ncell * (ts + 12.0 * p_tot * ts + 96.0 * len(d["freqs_hz"])) + slab * 8.0 * ts
    return {"bytes_per_cell_update": b, "achieved_gbs": gcells * b, "frac": gcells * b / peak,
            "note": "per-cell-update byte model of the method (separate H and E passes); step_bytes_frac "
                    "counts the bytes of this build's kernels (fused interior: 48 B per cell)"}


def set_steps(d, M):
    """Set a description's time steps; a sampled source waveform is cut to the new window (its
    first 2 M + 1 half-step samples are the same function of time)."""
    if d.get("src_wave") is not None:
        if 2 * M + 1 > len(d["src_wave"]):
            raise ValueError("more time steps than the source waveform covers")
        d["src_wave"] = d["src_wave"][:2 * M + 1]
    d["n_steps"] = M


def workload_and_config(args):
    import synth
    if args.workload.startswith("f3_"):
        w = synth.paper_workload(args.workload[3:])
    else:
        w = synth.workload(args.workload)
    d = w["desc"]
    if args.time_steps:
        set_steps(d, args.time_steps)
    ncell = d["nx"] * d["ny"] * d["nz"]
    dshape = synth.box_shape(d["design_box"])
    poles = [len(w["m1"]["poles"][0]) + len(w["m2"]["poles"][0])]
    cfg = {
        "workload": {
            "c1": "config 1: 32^3 Yee grid dx=5nm, 8-cell CPML, 1000 steps, z-dipole, 16^3 design, "
                  "vacuum | 2-pair Drude-Lorentz metal, 600 nm, FP64",
            "c2": "config 2: 256^3 Yee grid dx=5nm, 12-cell CPML, 4000 steps, 128^3 design with smooth "
                  "seeded density, air | 3-pair CCPR metal, objective at 500/600/700 nm, TF/SF plane wave "
                  "along x, FP32 fields + FP64 DFT",
            "c3": "config 3: 512x512x384 grid, 16-cell CPML, 6000 steps, 256x256x192 design, 2-pair "
                  "Lorentz dielectric | 4-pair metal, FP32",
            "c4": "config 4: 64^3 grid, 2000 steps, 32^3 design, 2-pair metal, rho in [0.2,0.8]",
        }.get(args.workload) or (
            f"the paper's setup with {args.workload[3:]}: design 25x100x100 / gap 25x6x6 cells (the paper's "
            "100x25x100 / 6x25x6 with x and y exchanged), z-polarised plane wave along x carrying the "
            "truncated sinc x Hanning pulse at 576.5 THz, 20-cell CPML, 15 air cells of padding, "
            f"dx={'2' if args.workload[3:] in ('Al', 'Au') else '5'} nm, dt=dx/(2c0), air | Table-1 "
            f"{args.workload[3:]} with gamma=5e4, one density per E sample, 8 objective frequencies over "
            "350-1000 nm, FP32 fields + FP64 DFT"),
        "grid": [d["nx"], d["ny"], d["nz"]], "time_steps": d["n_steps"], "design": list(dshape[::-1]),
        "pole_pairs_total": poles[0], "n_freq": len(d["freqs_hz"]), "precision": d["precision"],
        "dft_accumulators": "f64", "parallelism": f"replicas x{args.gpus}",
    }
    return w, cfg, ncell


def footprint_bytes(w):
    from paper_2305_00234_gb300 import fdtd_footprint_bytes
    pt = [len(w["m1"]["poles"][k]) + len(w["m2"]["poles"][k]) for k in range(3)]
    return fdtd_footprint_bytes(w["desc"], pt)


def kernel_hash():
    """Hash of the device-kernel sources with comments and whitespace removed (a comment edit does not
    change the kernels the DRAM counters were taken on)."""
    h = hashlib.sha256()
    for f in ("fdtd_kernels.cuh", "fdtd_step.cuh", "fdtd_shell2.cuh", "fdtd_design2.cuh", "fdtd_params.h"):
        with open(os.path.join(ROOT, "paper_2305_00234_gb300", "csrc", f), "rb") as fh:
            t = fh.read().decode()
        t = re.sub(r"/\*.*?\*/", "", t, flags=re.S)
        t = re.sub(r"//[^\n]*", "", t)
        h.update(re.sub(r"\s+", " ", t).encode())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    return 6800.0, "fallback (6.8 TB/s)"


def profiled_traffic(workload, kernel):
    """DRAM bytes (read + write) per launch of `kernel` from the committed ncu summary, if it was
    taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        j = json.load(f)
    if j.get("kernel_hash") != kernel_hash():
        return None
    return j.get("per_launch_bytes", {}).get(workload, {}).get(kernel)


def cpu_baseline(args, w_full):
    """The FP64 oracle as it stands, on a bounded sample of the same workload (its first
    cpu-sample-steps time steps, forward + adjoint + gradient), on the host cores."""
    import copy

    import oracle
    w = copy.deepcopy(w_full)
    set_steps(w["desc"], args.cpu_sample_steps)
    d = w["desc"]
    ncell = d["nx"] * d["ny"] * d["nz"]
    t0 = time.perf_counter()
    o = oracle.problem(w)
    t1 = time.perf_counter()
    o.forward()
    o.adjoint()
    o.gradient()
    t2 = time.perf_counter()
    o.close()
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    cu = 2.0 * ncell * d["n_steps"]
    return {"value": cu / (t2 - t1) / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{args.workload} grid and materials, first {d['n_steps']} time steps of the forward "
                      f"and adjoint runs + gradient ({cu:.3g} cell-updates, {t2 - t1:.1f} s; setup "
                      f"{t1 - t0:.1f} s excluded)",
            "seconds": t2 - t1}


def serving_run(args, device):
    """The seeded serving stream (Poisson, mean 20 req/s; cubic grids 48..192, 1500-4000 steps, 1-4 pole
    pairs): N requests through the continuous-batching server (batch lane: persistent kernel for grids up to
    --serving-batch-max-cells cells, none by default; plain lane: per-request CUDA-graph streams for the
    others, grids of --serving-exclusive-cells cells and more one at a time) and, as the
    baseline, the same requests one after another on the same GPU (plain path, FIFO).  The offered load
    (about 2.3e11 cell-updates/s) is above one GPU's capacity, so that replay measures throughput and
    queueing latency; a second replay of the first M requests with arrivals slowed to about 0.7 of the
    capacity just measured gives the latency below saturation.  Accuracy: the largest relative differences
    of F and dF/drho between the server's and the sequential results."""
    import numpy as np

    import synth
    from paper_2305_00234_gb300 import serve
    items = synth.serving_stream(n_requests=args.serving_requests)
    bmc = None if args.serving_batch_max_cells < 0 else args.serving_batch_max_cells
    exc = args.serving_exclusive_cells or None
    cu = sum(2.0 * it["desc"]["nx"] * it["desc"]["ny"] * it["desc"]["nz"] * it["desc"]["n_steps"] for it in items)
    serve.evaluate(serve.from_stream(items[:1])[0])            # warm-up (library, pools)
    server = serve.GradientServer(max_slots=args.serving_slots, device=device, batch_max_cells=bmc,
                                      exclusive_cells=exc)
    res_s, wall_s = serve.replay_stream(serve.from_stream(items), server)
    server.close()
    res_q, wall_q = serve.replay_stream(serve.from_stream(items), None)
    dF = max(abs(a.F - b.F) / abs(b.F) for a, b in zip(res_s, res_q))
    dG = max(float(np.linalg.norm(a.grad - b.grad) / np.linalg.norm(b.grad)) for a, b in zip(res_s, res_q))
    lanes = {ln: sum(1 for r in res_s if r.lane == ln) for ln in ("batch", "plain")}
    out = {"requests": len(items), "rate_hz": 20.0, "slots": args.serving_slots, "batch_max_cells": bmc,
           "exclusive_cells": exc,
           "server": {"grad_evals_per_s": len(items) / wall_s, "Gcell_updates_per_s": cu / wall_s / 1e9,
                      "wall_s": wall_s, "peak_active": server.peak_active, "peak_batched": server.peak_batched,
                      "batch_launches": server.launches, "lanes": lanes, **serve.latency_stats(res_s)},
           "sequential": {"grad_evals_per_s": len(items) / wall_q, "Gcell_updates_per_s": cu / wall_q / 1e9,
                          "wall_s": wall_q, **serve.latency_stats(res_q)},
           "max_rel_diff_vs_sequential": {"F": dF, "dF_drho": dG}}
    out["speedup_grad_evals_per_s"] = out["server"]["grad_evals_per_s"] / out["sequential"]["grad_evals_per_s"]
    m = min(args.serving_load_requests, len(items))
    if m > 0:
        cap = len(items) / wall_s                                  # the server's measured evaluations/s
        rate = 0.7 * cap
        scale = 20.0 / rate                                        # stretch the 20 req/s arrivals
        sub = items[:m]
        server = serve.GradientServer(max_slots=args.serving_slots, device=device, batch_max_cells=bmc,
                                      exclusive_cells=exc)
        res_l, wall_l = serve.replay_stream(serve.from_stream(sub), server, time_scale=scale)
        server.close()
        out["load_0p7"] = {"requests": m, "offered_rate_hz": rate, "wall_s": wall_l,
                           "grad_evals_per_s": m / wall_l, **serve.latency_stats(res_l)}
    return out


def precision_study(args):
    """Config 3 in the FP32 build (FP64 DFT and gradient accumulators) and the all-FP64 build:
    relative L2 of the final fields, the DFTs and dF/drho against the FP64 run."""
    import numpy as np
    import torch

    import paper_2305_00234_gb300 as lib
    import synth
    w = synth.workload("c3")
    if args.time_steps:
        set_steps(w["desc"], args.time_steps)
    out = {}
    res = {}
    for prec in (64, 32):
        d = dict(w["desc"], precision=prec)
        p = lib.Problem(d, w["bg"], w["m1"], w["m2"], w["gamma"], stream=torch.cuda.current_stream().cuda_stream)
        p.set_density(w["rho"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        F, gap = p.forward()
        fields = [p.field(c) for c in range(3)]
        dft = p.dft()
        p.adjoint()
        g = p.gradient()
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        res[prec] = (F, fields, dft, g)
        ncell = d["nx"] * d["ny"] * d["nz"]
        out[f"fp{prec}"] = {"seconds_per_gradient_incl_field_readback": t, "F": F,
                            "Gcell_updates_per_s": 2.0 * ncell * d["n_steps"] / t / 1e9,
                            "device_bytes": p.info()["device_bytes"]}
        p.close()

    def rel(a, b):
        return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))
    F64, f64, d64, g64 = res[64]
    F32, f32, d32, g32 = res[32]
    out["rel_l2_fp32_vs_fp64"] = {"E_final": rel(np.stack(f32), np.stack(f64)), "forward_dft": rel(d32, d64),
                                  "objective": abs(F32 - F64) / abs(F64), "dF_drho": rel(g32, g64)}
    line = {"metric": "precision study (config 3)", "config": {"workload": "config 3: 512x512x384 grid, "
            "16-cell CPML, 256x256x192 design, 2-pair Lorentz dielectric (eps_inf 11.7/11.7/12.1) | 4-pair "
            "metal", "time_steps": w["desc"]["n_steps"]}, **out}
    print(json.dumps(line), flush=True)
    return 0


def filter_bench(args):
    """fdtd_filter_project + fdtd_filter_project_grad on the design box (the paper's R = 12 cells, its
    final beta = 52, eta = 0.5): CUDA-event time per forward + chain-rule pair.  Each call runs one cone
    correlation (the filter, or its transpose) and the normalising sums, which come in closed form from a
    summed-volume table of the weights; the algorithmic work is one FMA per sphere tap (|d| < R) per voxel
    per correlation, against the FP32 FMA rate of the SMs (152 SMs x 128 lanes x 2 flop x the sampled SM
    clock)."""
    import numpy as np
    import torch

    import paper_2305_00234_gb300 as lib
    import synth
    w, cfg, ncell = workload_and_config(args)
    shape = synth.box_shape(w["desc"]["design_box"])
    R, beta, eta = 12.0, 52.0, 0.5
    rho = torch.tensor(synth.smooth_rho(shape, 7, 3.0), dtype=torch.float32, device="cuda")
    rt, rb, gin, gout = (torch.empty_like(rho) for _ in range(4))
    gin.copy_(torch.tensor(synth.uniform_rho(shape, 8, -1.0, 1.0), dtype=torch.float32))
    stream = torch.cuda.current_stream()
    times = []
    clocks = ClockSampler(torch.cuda.current_device())
    for s_ in range(args.warmup + args.steps):
        if s_ == args.warmup:
            clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        lib.fdtd_filter_project(rho, rt, rb, R, beta, eta, stream.cuda_stream)
        lib.fdtd_filter_project_grad(rt, gin, gout, R, beta, eta, stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if s_ >= args.warmup:
            times.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    ms = statistics.median(times)
    n = int(np.ceil(R)) - 1
    d = np.arange(-n, n + 1)
    taps = int(np.count_nonzero(np.sqrt(d[:, None, None] ** 2 + d[None, :, None] ** 2 + d[None, None, :] ** 2) < R))
    nv = int(np.prod(shape))
    flops = 2.0 * taps * nv * 2
    mhz = clk.get("sm_mhz") or 2070.0
    peak = 152 * 128 * 2 * mhz * 1e6 / 1e12
    line = {"metric": "density filter + projection and chain rule (cone R = 12)", "value": ms, "unit": "ms",
            "higher_is_better": False, "steps": args.steps, "warmup": args.warmup, "design": list(shape[::-1]),
            "taps_per_voxel": taps,
            "roofline": {"bound": "alu", "achieved": flops / (ms * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flops / (ms * 1e-3) / 1e12 / peak,
                         "peak_source": "152 SMs x 128 FP32 lanes x 2 flop (FMA) x sampled SM clock"},
            "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def paper_mode(args):
    """The paper's time-domain objective and history gradient (fdtd_paper_forward + fdtd_paper_gradient,
    checkpoint-recompute) on the workload: wall time per gradient with CUDA events on the handle's
    stream, and the same cell-update count as the main metric (forward + adjoint; the recomputed
    forward segments are the mode's overhead)."""
    import torch

    import paper_2305_00234_gb300 as lib
    w, cfg, ncell = workload_and_config(args)
    if w["desc"].get("density_layout", 0) != 0:   # paper mode takes one density per voxel
        import synth
        w["desc"] = dict(w["desc"], density_layout=0)
        w["rho"] = synth.smooth_rho(synth.box_shape(w["desc"]["design_box"]), w["seed"] + 1000, 3.0)
    stream = torch.cuda.current_stream()
    p = lib.Problem(w["desc"], w["bg"], w["m1"], w["m2"], w["gamma"], stream=stream.cuda_stream)
    p.set_density(w["rho"])
    grad = torch.zeros(p.dshape, dtype=torch.float32, device="cuda")
    times = []
    for s in range(args.warmup + args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        F = p.paper_forward()
        p.paper_gradient(grad)
        e1.record(stream)
        torch.cuda.synchronize()
        if s >= args.warmup:
            times.append(e0.elapsed_time(e1))
    M = w["desc"]["n_steps"]
    ms = statistics.median(times)
    info = p.info()
    p.close()
    line = {"metric": "paper-mode gradient (time-domain objective, Eq. (Gradient_FDTD), checkpoint-recompute)",
            "value": 2.0 * ncell * M / (ms * 1e-3) / 1e9, "unit": "Gcell-updates/s", "ms_per_gradient": ms,
            "steps": args.steps, "warmup": args.warmup, "objective": F, "device_bytes": info["device_bytes"],
            "config": cfg}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    w, cfg, ncell = workload_and_config(args)
    import copy

    import oracle
    ws = copy.deepcopy(w)
    set_steps(ws["desc"], args.cpu_sample_steps)
    o = oracle.problem(ws)
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        o.forward()
        o.adjoint()
        o.gradient()
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    o.close()
    cu = 2.0 * ncell * args.cpu_sample_steps
    value = cu * len(times) / sum(times) / 1e9
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"each step: the {args.workload} workload's grid and materials for its first "
              f"{args.cpu_sample_steps} time steps (forward + adjoint + gradient), FP64 oracle")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    import paper_2305_00234_gb300 as lib
    lib.load_library()
    w, cfg, ncell = workload_and_config(args)
    d = w["desc"]
    M = d["n_steps"]
    fp = footprint_bytes(w)
    cfg["working_set_bytes"] = fp
    cfg["l2"] = ("inputs larger than L2: working set %.2f GB vs 129 MB L2, no flush" % (fp / 1e9)
                 if fp > L2_BYTES else "working set below L2: L2 flushed between steps")
    stream = torch.cuda.current_stream()
    p = lib.Problem(d, w["bg"], w["m1"], w["m2"], w["gamma"], stream=stream.cuda_stream)
    rho_dev = torch.tensor(w["rho"], dtype=torch.float32, device=f"cuda:{local}")
    grad_dev = torch.zeros(p.dshape, dtype=torch.float32, device=f"cuda:{local}")
    p.set_density(rho_dev)
    flush = None
    if fp <= L2_BYTES:
        flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=f"cuda:{local}")

    def one_step():
        p.forward()
        p.adjoint()
        p.gradient(grad_dev)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    # ---- timed region (device-resident inputs; the product path: CUDA graphs, profiling off) ----
    p.reset_timings()
    sampler = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier(dist, local)
    torch.cuda.synchronize()
    sampler.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for s in range(args.steps):
        if flush is not None:
            flush.zero_()
        ev[s][0].record(stream)
        one_step()
        ev[s][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(dist, local)
    clocks = sampler.stop()
    launches = int(p.timings()["launches"])            # kernels this library launched in the timed region
    elapsed_ms = t_start.elapsed_time(t_end)
    # ---- per-kernel times: one more gradient evaluation after the timed region, with profiling on
    # (every fourth 16-step block launched kernel by kernel between CUDA events on the library's stream)
    p.reset_timings()
    p.set_profiling(True)
    one_step()
    torch.cuda.synchronize()
    p.set_profiling(False)
    tim = p.timings()
    per_step = [a.elapsed_time(b) for a, b in ev]
    t_max = max_over_ranks(dist, elapsed_ms / 1e3, local)
    cu_step = 2.0 * ncell * M
    total_cu = sum_over_ranks(dist, cu_step * args.steps, local)
    value = total_cu / t_max / 1e9
    # per-kernel achieved bandwidth: algorithmic bytes per launch / average launch time (CUDA events
    # on the library's stream over the timed region); the dominant kernel is the one with most time
    peak, peak_src = measured_peaks()
    prec_t = "float" if d["precision"] == 32 else "double"
    names = {"shell_h": "shell_h2_kernel" if tim["paired_shell"] else f"shell_h_kernel<{prec_t}>",
             "step": f"step_kernel<{prec_t}>",
             "shell_e": "shell_e2_kernel" if tim["paired_shell"] else f"shell_e_kernel<{prec_t}>",
             "ed": "e_design2_kernel<*>" if tim["paired_design"] else f"e_design_kernel<{prec_t},*>",
             "dft": f"dft_kernel<{prec_t}>", "grad": f"grad_kernel<{prec_t}>"}
    kern = {}
    runs = 2 * args.steps                                   # forward + adjoint per gradient in the timed region
    blocks = -(-M // int(max(tim["dft_steps_per_launch"], 1)))
    total = {"shell_h": M * runs, "step": M * runs if tim["step_launches"] else 0, "shell_e": M * runs,
             "ed": M * runs if tim["ed_launches"] else 0,
             "dft": blocks * runs if tim["dft_launches"] else 0, "grad": args.steps}
    # Two byte counts per launch.  method: the per-cell-update count of the method (state words read
    # once and written once per half-step, separate H and E passes: 9 words per cell per half-step, psi
    # and design terms as in cell_update_model) over the cells the launch updates; the fused interior
    # kernel does both half-steps of its cells in one pass and so moves fewer bytes than this count.
    # kernel: the bytes the kernel itself must move (fdtd_get_timings: each word it touches read once,
    # written once).  They differ only for the interior kernel (48 B per cell against 72 B) and the
    # design-E kernel (its E snapshot for the blocked DFT is not a term of the method).
    ts = 4.0 if d["precision"] == 32 else 8.0
    ni, ndi = tim["interior_cells"], tim["interior_design_cells"]
    psi_in = tim["bytes_step_per_launch"] - ts * (12.0 * ni - 3.0 * ndi)   # psi of the slab cells it updates
    method = {"step": 9.0 * ts * (2.0 * ni - ndi) + psi_in,
              "ed": tim["bytes_ed_per_launch"] - 3.0 * ts * p.nd}
    for k in ("shell_h", "step", "shell_e", "ed", "dft", "grad"):
        nl = tim[f"{k}_launches"]
        if nl == 0:
            continue
        avg_s = tim[f"{k}_ms"] / nl / 1e3
        kb = tim[f"bytes_{k}_per_launch"]
        mb = method.get(k, kb)
        ach = mb / avg_s / 1e9 if avg_s > 0 else 0.0
        kach = kb / avg_s / 1e9 if avg_s > 0 else 0.0
        # time_share: launches x (sampled, serialised) launch time / timed region; in the captured
        # graphs the shell H kernel runs next to the interior kernel and the shell E kernel next to the
        # design E kernel, so the shares may sum above 1
        kern[k] = {"kernel": names[k], "timed_launches": nl, "launches": total[k], "avg_launch_ms": avg_s * 1e3,
                   "algorithmic_bytes_per_launch": mb, "achieved": ach, "frac": ach / peak,
                   "kernel_bytes_per_launch": kb, "kernel_bytes_achieved": kach, "kernel_bytes_frac": kach / peak,
                   "time_share": avg_s * total[k] / (elapsed_ms / 1e3)}
    dom = max(kern, key=lambda k: kern[k]["time_share"])
    kd = kern[dom]
    roof = {"bound": "hbm", "kernel": kd["kernel"], "achieved": kd["achieved"], "peak": peak, "unit": "GB/s",
            "frac": kd["frac"], "traffic": profiled_traffic(args.workload, dom), "peak_source": peak_src,
            "algorithmic_bytes_per_launch": kd["algorithmic_bytes_per_launch"],
            "kernel_bytes_frac": kd["kernel_bytes_frac"],
            "avg_launch_ms": kd["avg_launch_ms"], "kernels": kern,
            "step_bytes_frac": sum(v["kernel_bytes_per_launch"] * v["launches"] for v in kern.values())
            / (elapsed_ms / 1e3) / 1e9 / peak,
            "dft_steps_per_launch": tim["dft_steps_per_launch"],
            "per_kernel_times": "CUDA events on the library's stream in one profiled gradient evaluation after "
                                "the timed region (kernels launched one by one); value is timed without them",
            "cell_update_model": cell_update_model(w, value, peak)}
    # ---- end to end through the public API with host buffers ----
    e2e = None
    if args.e2e_steps > 0:
        rho_host = torch.tensor(w["rho"], dtype=torch.float32).pin_memory()
        grad_host = torch.zeros(p.dshape, dtype=torch.float32).pin_memory()
        torch.cuda.synchronize()
        barrier(dist, local)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            p.set_density(rho_host)
            p.forward()
            p.adjoint()
            p.gradient(grad_host)
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(dist, time.perf_counter() - t0, local)
        e2e_value = sum_over_ranks(dist, cu_step * args.e2e_steps, local) / e2e_s / 1e9
        nd = int(np.prod(p.dshape))
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * nd, "d2h_bytes_per_step": 4 * nd,
               "note": "per step: float32 density H2D from pinned memory, float32 gradient D2H to pinned "
                       "memory (plus < 2 KB of gap DFT and adjoint coefficients)"}
    p.close()
    serving = None
    if rank == 0 and args.serving_requests > 0:
        serving = serving_run(args, local)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, w)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if d["precision"] == 32 else "f64",
                "data": "synthetic", "config": cfg, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks,
                "latency_ms": {"p50": statistics.median(per_step),
                               "p99": float(np.percentile(per_step, 99)), "n": len(per_step),
                               "note": "single-request gradient latency in the timed loop"},
                "serving": serving}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    args = parse(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.precision_study:
        return precision_study(args)
    if args.paper_mode:
        return paper_mode(args)
    if args.filter:
        return filter_bench(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
