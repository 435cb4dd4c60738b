"""Benchmark: one full USPG/USCG reconstruction per step on GB300.

A step is the whole hot path on one batch of synthetic input: coefficient
generation for the representative views (FP64), per-view simultaneous MART
(FP32, 5 iterations), and the Cartesian resample -- on the 3D cone-beam
workload (128 rings x 128 slabs, 90 views over 360 deg, 256x256 detector,
12 ellipsoids + blob, Poisson noise at 1e5 photons, lambda 0.1).

Metric: MART ray-cell updates per second (nonzeros of the full system matrix
over all views x iterations, per second of step time).  Also reported:
ms per MART iteration, the per-phase split, the roofline of the dominant
kernel (per-launch CUDA-event times), the end-to-end number through the C ABI
with host buffers, and the FP64 oracle on the host cores (bounded sample).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU: one independent reconstruction per rank (replicas; the method has
no exchange step), value = all ranks' updates / max rank time.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "3d-cone-128r-128s-90v-256"
METRIC = "MART ray-cell updates/s"
UNIT = "ray-cell updates/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
REASON_BITS = {
    0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
    0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
    0x100: "display_clock_setting",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--coeff-dtype", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--serve-rate", type=float, default=200.0, help="serve-mixed: mean requests per second")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="serve-mixed: arrival window")
    ap.add_argument("--serve-sustained-seconds", type=float, default=60.0,
                    help="serve-mixed: arrival window of the run at 70%% of capacity")
    ap.add_argument("--serve-active", type=int, default=64, help="serve-mixed: jobs running at once")
    return ap.parse_args()


def max_over_ranks(values, device=None):
    """Element-wise max of per-rank timings over the process group (the
    slowest rank sets a replica run's time); identity without a group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def replica_seed(base_seed: int, rank: int) -> int:
    """Each rank reconstructs its own object (independent replicas)."""
    return base_seed + 1000 * rank


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active"
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms",
                                          "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 4:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, 0
        for s in self.samples:
            try:
                sm.append(float(s[0]))
                mx = float(s[1])
                reasons |= int(s[3], 16) if s[3].startswith("0x") else int(s[3])
            except ValueError:
                continue
        names = [n for b, n in REASON_BITS.items() if reasons & b and n != "gpu_idle"]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": names,
                "samples": len(sm)}


def load_peaks():
    try:
        d = json.load(open(PEAKS_FILE))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ------------------------------------------------------------ our path ---

def run_ours(args, rank, world, local):
    import torch

    from paper_2208_12964_gb300 import synth, uspg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    spec = synth.workload(args.workload)
    spec["seed"] = replica_seed(spec["seed"], rank)
    proj_host = synth.projections(spec)
    n_views, n_rays = proj_host.shape
    iters, lam = spec["iterations"], spec["lam"]
    dt = {"f32": uspg.F32, "f16": uspg.F16, "bf16": uspg.BF16}[args.coeff_dtype]
    g, s, o, _ = uspg.descs_from_spec(spec, dtype=dt)
    ctx = uspg.uspg_create(g, s, o)
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream
    proj_dev = torch.from_numpy(proj_host).to(dev)
    proj_pin = torch.from_numpy(proj_host).pin_memory()
    R = spec["n_rings"]
    nx = ny = 2 * R
    ns = spec["n_slabs"]
    img_dev = torch.empty((ns, ny, nx), dtype=torch.float32, device=dev)
    img_pin = torch.empty((ns, ny, nx), dtype=torch.float32).pin_memory()
    seq = spec.get("schedule") == "sequential"  # the paper's ray order (one persistent warp)
    rule = spec.get("rule", uspg.POWER)  # Table 1's fan scan uses the update of Eq. 18
    opts, _keep = uspg.mart_opts(iters, lam, uspg.SEQUENTIAL if seq else uspg.PER_VIEW, rule)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    def step_device():
        uspg.uspg_set_projections(ctx, proj_dev, True, sp)
        uspg.uspg_build_coeffs(ctx, sp)
        uspg.uspg_fill_image(ctx, 1.0, sp)
        uspg.uspg_mart(ctx, opts, sp)
        uspg.uspg_resample_cartesian(ctx, uspg.RESAMPLE_POINT, nx, ny, img_dev, True, sp)

    def step_e2e():
        # host projections in, host image out, both through the C ABI
        uspg.uspg_set_projections(ctx, proj_pin, False, sp)
        uspg.uspg_build_coeffs(ctx, sp)
        uspg.uspg_fill_image(ctx, 1.0, sp)
        uspg.uspg_mart(ctx, opts, sp)
        uspg.uspg_resample_cartesian(ctx, uspg.RESAMPLE_POINT, nx, ny, img_pin, False, sp)

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed(fn, k):
        """per-step device time (CUDA events on the launching stream), L2
        flushed between steps; returns total ms"""
        tot = 0.0
        for _ in range(k):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        return tot

    step_device()
    tuned = (0, 0) if seq else uspg.uspg_autotune(ctx, sp)  # launch shape of the per-view kernels
    for _ in range(args.warmup):
        step_device()
    torch.cuda.synchronize(dev)
    st = uspg.uspg_coeff_stats(ctx)
    updates_per_step = st["nnz_all_views"] * iters

    launches0 = uspg.uspg_kernel_launches()
    barrier()
    with ClockSampler(local) as clk:
        t_dev = timed(step_device, args.steps)
    barrier()
    launches = uspg.uspg_kernel_launches() - launches0
    uspg.uspg_sync(ctx, sp)

    # phase split (separate, after the timed region)
    def phase_ms(fn, k=2):
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / k

    ms_build = phase_ms(lambda: uspg.uspg_build_coeffs(ctx, sp))

    def mart_only():
        uspg.uspg_fill_image(ctx, 1.0, sp)
        uspg.uspg_mart(ctx, opts, sp)

    ms_mart = phase_ms(mart_only)
    ms_resample = phase_ms(lambda: uspg.uspg_resample_cartesian(ctx, uspg.RESAMPLE_POINT, nx, ny, img_dev, True, sp))

    # per-launch kernel times of the dominant phase
    fw = bw = None
    if not seq:
        uspg.uspg_fill_image(ctx, 1.0, sp)
        fw, bw = uspg.uspg_mart_kernel_times(ctx, opts, iters * n_views, sp)

    e2e = None
    if not args.no_e2e:
        for _ in range(2):
            step_e2e()
        torch.cuda.synchronize(dev)
        barrier()
        t_e2e = timed(step_e2e, args.steps)
        barrier()
        e2e = (t_e2e, int(proj_pin.numel() * 4), int(img_pin.numel() * 4))

    t_max = t_dev
    if world > 1:
        t_max, t_e2e = max_over_ranks([t_dev, e2e[0] if e2e else 0.0], dev)
        if e2e:
            e2e = (t_e2e, e2e[1], e2e[2])
    # image quality of the final reconstruction against its phantom (Table 2's measures)
    torch.cuda.synchronize(dev)
    quality_rep = None
    if rank == 0:
        from paper_2208_12964_gb300 import quality

        quality_rep = quality.report(spec, img_dev.cpu().numpy())
    info = dict(quality=quality_rep, weight_bytes=4 if args.coeff_dtype == "f32" else 2, coeff_dtype=args.coeff_dtype, tuned=tuned, stats=st, t_ms=t_max, updates_per_step=updates_per_step, launches=launches, clk=clk.summary(),
                ms_build=ms_build, ms_mart=ms_mart, ms_resample=ms_resample, fw=fw, bw=bw, e2e=e2e, spec=spec,
                proj=proj_host)
    uspg.uspg_destroy(ctx)
    return info


def latency_line(info):
    """The ray-sequential schedule is a chain of dependent ray steps (each
    ray's update must land before the next ray's sum): its bound is latency,
    reported as time per ray step, not as a bandwidth fraction."""
    st = info["stats"]
    steps = info["spec"]["iterations"] * st["n_views"] * st["n_rays"]
    return {"bound": "latency", "kernel": "k_sequential", "achieved": round(info["ms_mart"] * 1e3 / steps, 4),
            "unit": "us per ray step", "peak": None, "frac": None, "traffic": None,
            "ray_steps": steps}


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic_cone128_mart.json")


def sources_sha256(files) -> str:
    """SHA-256 over the given repository files, in order."""
    import hashlib

    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def sources_hash_matches(rec: dict) -> bool:
    return sources_sha256(rec["sources"]) == rec["sources_sha256"]


def measured_traffic(kernel: str, dtype: str, mirrored: bool, spec: dict):
    """DRAM bytes per launch of `kernel` from the committed ncu capture, or
    None when there is no capture for this form or the kernel sources have
    changed since it was taken (checked by hash)."""
    try:
        rec = json.load(open(TRAFFIC_FILE))
    except (OSError, ValueError):
        return None
    if not sources_hash_matches(rec):
        return None
    geo = f"{spec['n_rings']}r-{spec['n_slabs'] if spec['geometry'] == 1 else 1}s-{spec['n_u']}x{spec['n_v']}"
    k = rec["kernels"].get(f"{geo}/{kernel}/{dtype}/{'mirrored' if mirrored else 'full'}")
    return k["dram_bytes_per_launch"] if k else None


def roofline(info):
    """Dominant per-view kernel: algorithmic HBM bytes per launch / mean launch time.

    Per view, with S = entries the representative stores (half of the view's
    nonzeros under the z-mirror), b = index + weight bytes per entry:
      forward:    S*b (rows) + S/8*4 (group rays) + rays*12 (projection in,
                  ray sum accumulate, ray term out); the image gathers hit L2
      correction: S*b (columns) + slices*72 (offset and meta, lane table)
                  + cells*8 (image read and write) + rays*16 (ray terms: 8 B a ray,
                  twice with the z-mirror)
    """
    st = info["stats"]
    fw, bw = np.asarray(info["fw"], np.float64), np.asarray(info["bw"], np.float64)
    n_rays = st["n_rays"]
    S = st["nnz_store"] / st["n_reps"]
    b_e = 4 + info.get("weight_bytes", 4)
    cells = st["n_cells"]
    fwd_bytes = S * b_e + S / 8 * 4 + n_rays * 12
    bwd_bytes = S * b_e + st["slices"] * 72 + cells * 8 + n_rays * (16 if st["mirrored"] else 8)
    t_f, t_b = fw.mean(), bw.mean()
    if t_b >= t_f:
        name, b, t = "k_backward", bwd_bytes, t_b
    else:
        name, b, t = "k_forward", fwd_bytes, t_f
    peak, src = load_peaks()
    achieved = b / (t * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": name, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_source": src,
            "traffic": measured_traffic(name, info.get("coeff_dtype", "f32"), bool(st["mirrored"]), info["spec"]),
            "bytes_per_launch": int(b), "ms_per_launch": round(t, 5),
            "other": {"k_forward_ms": round(t_f, 5), "k_backward_ms": round(t_b, 5),
                      "k_forward_GBs": round(fwd_bytes / (t_f * 1e-3) / 1e9, 1),
                      "k_backward_GBs": round(bwd_bytes / (t_b * 1e-3) / 1e9, 1),
                      "mirrored_store": bool(st["mirrored"])}}


# ------------------------------------------------------------- oracle ---

def oracle_sample(spec, proj, threads=None, n_views=1):
    """The FP64 oracle, as it stands, on a bounded sample: per-view MART steps
    for the first n_views views of the same workload (all rays)."""
    import oracle

    threads = threads or os.cpu_count() or 1
    keys = dict(oracle.Problem._fields_)
    if spec.get("schedule") == "sequential":  # the whole ray-sequential run, single-threaded
        o = oracle.Oracle({k: v for k, v in spec.items() if k in keys}, threads=1)
        f = np.ones(o.n_cells)
        nnz = spec["iterations"] * sum(o.view_nnz(k) for k in range(spec["n_views"]))
        t0 = time.perf_counter()
        o.mart_sequential(proj, f, spec["iterations"], spec["lam"], rule=spec.get("rule", oracle.POWER))
        dt = time.perf_counter() - t0
        return nnz / dt, 1, dt, nnz
    o = oracle.Oracle({k: v for k, v in spec.items() if k in keys}, threads=threads)
    f = np.ones(o.n_cells)
    t0 = time.perf_counter()
    nnz = o.mart_views_sample(proj, f, list(range(n_views)), spec["lam"])
    dt = time.perf_counter() - t0
    return nnz / dt, threads, dt, nnz


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from paper_2208_12964_gb300 import synth

    spec = synth.workload(args.workload)
    proj = synth.projections(spec)
    import oracle

    oracle.build()
    for _ in range(args.warmup):
        oracle_sample(spec, proj)
    vals, tot = [], 0.0
    for _ in range(args.steps):
        v, thr, dt, nnz = oracle_sample(spec, proj)
        vals.append(v)
        tot += dt
    val = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload,
                       "sample": ("the whole ray-sequential run" if spec.get("schedule") == "sequential"
                                  else "one per-view MART step (view 0, all rays)")},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": thr, "kind": "oracle",
                             "sample": f"{nnz} ray-cell updates per step"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def batch_specs(n=64, seed=4):
    """64 independent 2D parallel-beam reconstructions of uneven size: rings
    from {64, 128, 256, 512}, views from {18, 36, 90, 180} over a half turn,
    2R+1 detector bins, seeded ellipse phantoms, 10 per-view iterations."""
    from paper_2208_12964_gb300 import synth

    g = synth.Stream(seed)
    out = []
    for i in range(n):
        a, b = g.u(2)
        R = (64, 128, 256, 512)[int(a * 4)]
        V = (18, 36, 90, 180)[int(b * 4)]
        out.append(synth.parallel_workload(R, V, 2 * R + 1, seed=100 + i, iterations=10, lam=0.2))
    return out


def run_batched(args, rank, world, local):
    import torch

    from paper_2208_12964_gb300 import synth, uspg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream
    specs = batch_specs()
    ctxs = []
    for spc in specs:
        g, s, o, _ = uspg.descs_from_spec(spc)
        c = uspg.uspg_create(g, s, o)
        uspg.uspg_build_coeffs(c, sp)
        uspg.uspg_set_projections(c, synth.projections(spc), False, sp)
        uspg.uspg_fill_image(c, 1.0, sp)
        ctxs.append(c)
    torch.cuda.synchronize(dev)
    opts, _k = uspg.mart_opts(10, 0.2, uspg.PER_VIEW)
    b = uspg.uspg_batch_create(ctxs, opts, sp)
    info = uspg.uspg_batch_info(b)
    tuning = uspg.uspg_batch_tuning(b)

    def timed(fn, k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    for _ in range(args.warmup):
        uspg.uspg_batch_run(b, sp)
    torch.cuda.synchronize(dev)
    launches0 = uspg.uspg_kernel_launches()
    with ClockSampler(local) as clk:
        t = timed(lambda: uspg.uspg_batch_run(b, sp), args.steps)
    launches = uspg.uspg_kernel_launches() - launches0

    def sequential():
        for c in ctxs:
            uspg.uspg_mart(c, opts, sp)

    sequential()
    t_seq = timed(sequential, 1)
    uspg.uspg_batch_destroy(b)
    for c in ctxs:
        uspg.uspg_destroy(c)
    upd = info["updates_per_run"]
    line = {"metric": METRIC, "value": upd * args.steps / (t * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch-2d-64", "instances": len(specs),
                       "rings": sorted({s_["n_rings"] for s_ in specs}), "views": sorted({s_["n_views"] for s_ in specs}),
                       "iterations": 10, "graph_kernel_nodes": info["kernel_nodes"], "global_steps": info["steps"],
                       "step": "one batched run (10 per-view sweeps of every instance)"},
            "launch_shape": {"buckets": tuning["buckets"],
                             "probe_ms_default": round(tuning["ms_default"], 4),
                             "probe_ms_tuned": round(tuning["ms_tuned"], 4),
                             "gain": round(tuning["ms_default"] / tuning["ms_tuned"], 3) if tuning["ms_tuned"] else None,
                             "how": "blocks per unit of work per ring-count bucket, tuned on the first 4 global steps"},
            "sequential": {"value": upd / (t_seq * 1e-3), "ms": t_seq,
                           "how": "the same instances, uspg_mart one after another (one graph each)"},
            "gpu_launches": int(launches), "clocks": clk.summary()}
    print(json.dumps(line))
    return 0


SERVE_2D = [(R, V) for R in (64, 128, 256, 512) for V in (18, 36, 90, 180)]
SERVE_3D = [(64, 45, 128), (128, 90, 256), (256, 180, 512)]


def serve_trace(rate: float, seconds: float, seed: int = 5):
    """Seeded Poisson request stream of the mixed serving workload: exponential
    gaps of mean 1/rate; 80% 2D parallel-beam jobs (rings from {64, 128, 256,
    512}, views from {18, 36, 90, 180} over a half turn, 2R+1 bins, 10 per-view
    iterations, lambda 0.2) and 20% 3D cone-beam jobs (rings = slabs, views,
    detector) in {(64, 45, 128^2), (128, 90, 256^2), (256, 180, 512^2)}, 5
    iterations, lambda 0.1.  Returns [(arrival seconds, geometry key)]."""
    import math

    from paper_2208_12964_gb300 import synth

    g = synth.Stream(seed)
    t, out = 0.0, []
    while True:
        u, k, a = g.u(3)
        t += -math.log(1.0 - u) / rate
        if t >= seconds:
            return out
        if k < 0.8:
            R, V = SERVE_2D[min(int(a * len(SERVE_2D)), len(SERVE_2D) - 1)]
            out.append((t, ("2d", R, V)))
        else:
            out.append((t, ("3d",) + SERVE_3D[min(int(a * len(SERVE_3D)), len(SERVE_3D) - 1)]))


def serve_spec(key):
    from paper_2208_12964_gb300 import synth

    if key[0] == "2d":
        R, V = key[1:]
        return synth.parallel_workload(R, V, 2 * R + 1, seed=200 + R + V, iterations=10, lam=0.2)
    R, V, D = key[1:]
    return synth.cone_workload(R, R, V, D, iterations=5, lam=0.1, seed=300 + R, noise=False)


def _serve_trace_once(uspg, srv, trace, specs, proj, opts, dt, local):
    """Submits every request of `trace` at its arrival time and collects the
    results; returns the per-request results and the timing of the run."""
    results, pending = [], []
    launches0 = uspg.uspg_kernel_launches()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for t_arr, k in trace:
            while True:
                now = time.perf_counter() - t0
                if now >= t_arr:
                    break
                if pending:
                    pending = _serve_poll(uspg, srv, pending, results)
                time.sleep(min(2e-4, max(t_arr - now, 0.0)))
            pending.append(uspg.uspg_server_submit(srv, specs[k], proj[k], opts[k], dt, borrow=True))
        t_sub = time.perf_counter() - t0
        uspg.uspg_server_drain(srv, 1800.0)
        wall = time.perf_counter() - t0
        pending = _serve_poll(uspg, srv, pending, results)
    bad = [r for r in results if r["status"] != uspg.OK]
    if bad or pending:
        raise RuntimeError(f"{len(bad)} served jobs failed, {len(pending)} not collected: "
                           f"{bad[0]['message'] if bad else ''}")
    lat = np.array([r["latency_s"] for r in results]) * 1e3
    upd = sum(r["updates"] for r in results)
    return {"value": upd / wall, "jobs_per_s": len(results) / wall, "wall_s": wall, "submit_window_s": t_sub,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
            "queue_p50_ms": float(np.percentile([r["queue_s"] * 1e3 for r in results], 50)),
            "gpu_launches": int(uspg.uspg_kernel_launches() - launches0), "clocks": clk.summary()}


def run_serving(args, rank, world, local):
    """The request loop of the library (uspg_server_*) under a Poisson stream:
    each request is submitted at its arrival time with its projections read in
    place from page-locked host memory; the result image comes back to host
    memory.  Two streams are served, each with FP16 and with FP32
    coefficients: the offered rate (--serve-rate, far above one GPU's capacity
    for this mix, so it measures saturated throughput) and a rate at 70% of
    the FP16 capacity just measured (so latency reflects service, not a
    growing queue).  Before them one request per geometry runs untimed, so
    every store is resident (the steady state of a server that has seen its
    protocols); the images of those requests give the FP16-vs-FP32 error."""
    # more hardware work queues than the default 8, so that the streams of
    # concurrent jobs do not serialise behind one another (read at context creation)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import torch

    from paper_2208_12964_gb300 import synth, uspg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    trace = serve_trace(args.serve_rate, args.serve_seconds)
    keys = sorted({k for _, k in trace} | {("2d",) + g for g in SERVE_2D} | {("3d",) + g for g in SERVE_3D})
    specs = {k: serve_spec(k) for k in keys}
    proj = {k: torch.from_numpy(synth.projections(specs[k])).pin_memory() for k in keys}
    opts = {k: uspg.mart_opts(specs[k]["iterations"], specs[k]["lam"], uspg.PER_VIEW)[0] for k in keys}
    free, _total = torch.cuda.mem_get_info(dev)
    budget = int(free * 0.85)
    runs, images = {"offered": {}, "sustained": {}}, {}
    trace_s = None
    for name, dt in (("f16", uspg.F16), ("f32", uspg.F32)):
        srv = uspg.uspg_server_create(budget, args.serve_active, 1)
        try:
            warm = {k: uspg.uspg_server_submit(srv, specs[k], proj[k], opts[k], dt, borrow=True) for k in keys}
            uspg.uspg_server_drain(srv, 1800.0)
            for k, jid in warm.items():
                img = np.zeros(_n_cells(specs[k]), np.float32)
                r = uspg.uspg_server_poll(srv, jid, img)
                if r["status"] != uspg.OK:
                    raise RuntimeError(f"warm-up job {k} failed: {r['message']}")
                images.setdefault(k, {})[name] = img
            torch.cuda.synchronize(dev)
            runs["offered"][name] = _serve_trace_once(uspg, srv, trace, specs, proj, opts, dt, local)
            if trace_s is None:
                rate_s = 0.7 * runs["offered"]["f16"]["jobs_per_s"]
                trace_s = serve_trace(rate_s, args.serve_sustained_seconds, seed=6)
            runs["sustained"][name] = _serve_trace_once(uspg, srv, trace_s, specs, proj, opts, dt, local)
            st = uspg.uspg_server_stats(srv)
            runs["offered"][name]["store_reuses"] = st["store_reuses"]
            runs["offered"][name]["peak_device_bytes"] = st["peak_device_bytes"]
        finally:
            uspg.uspg_server_destroy(srv)
    errs = []
    for k in keys:
        a, b = images[k]["f16"].astype(np.float64), images[k]["f32"].astype(np.float64)
        errs.append(float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)))
    f16, f32 = runs["offered"]["f16"], runs["offered"]["f32"]
    s16, s32 = runs["sustained"]["f16"], runs["sustained"]["f32"]
    n2 = sum(1 for _, k in trace if k[0] == "2d")
    pick = ("value", "jobs_per_s", "p50_ms", "p99_ms", "mean_ms", "max_ms", "queue_p50_ms", "wall_s")
    line = {"metric": METRIC + " (served)", "value": f16["value"], "unit": UNIT, "n_gpus": 1,
            "steps": len(trace), "warmup": len(keys), "ms_per_step": f16["wall_s"] * 1e3 / len(trace),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f16 coefficients, f32 image and accumulation", "data": "synthetic",
            "config": {"workload": "serve-mixed", "offered_rate_per_s": args.serve_rate,
                       "arrival_window_s": args.serve_seconds, "requests": len(trace), "requests_2d": n2,
                       "requests_3d": len(trace) - n2, "geometries": len(keys), "max_active": args.serve_active,
                       "chunk": "1 sweep", "device_budget_bytes": budget,
                       "step": "one request (value = updates of all requests / wall time from first "
                               "arrival to last result)",
                       "l2": "inputs of the 3D jobs exceed L2; no flush between requests"},
            "latency_ms": {"p50": f16["p50_ms"], "p99": f16["p99_ms"], "mean": f16["mean_ms"], "max": f16["max_ms"],
                           "queue_p50": f16["queue_p50_ms"]},
            "jobs_per_s": f16["jobs_per_s"], "wall_s": f16["wall_s"], "store_reuses": f16["store_reuses"],
            "peak_device_bytes": f16["peak_device_bytes"],
            "fp32_coefficients": {k_: f32[k_] for k_ in pick},
            "sustained": {"offered_rate_per_s": len(trace_s) / args.serve_sustained_seconds,
                          "arrival_window_s": args.serve_sustained_seconds, "requests": len(trace_s),
                          "f16": {k_: s16[k_] for k_ in pick}, "f32": {k_: s32[k_] for k_ in pick}},
            "image_rel_l2_f16_vs_f32": {"median": float(np.median(errs)), "max": float(max(errs))},
            "e2e": {"value": f16["value"], "unit": UNIT, "how": "host projections in, host image out, per request",
                    "h2d_bytes_per_step": int(np.mean([proj[k].numel() * 4 for _, k in trace])),
                    "d2h_bytes_per_step": int(np.mean([_n_cells(specs[k]) * 4 for _, k in trace]))},
            "gpu_launches": f16["gpu_launches"], "clocks": f16["clocks"]}
    print(json.dumps(line))
    return 0


def _n_cells(spec):
    R = spec["n_rings"]
    per_slab = 3 * R * (R + 1)  # 6n sectors per ring
    return per_slab * (spec["n_slabs"] if spec["geometry"] == 1 else 1)


def _serve_poll(uspg, srv, pending, results):
    left = []
    for jid in pending:
        r = uspg.uspg_server_poll(srv, jid)
        if r is None:
            left.append(jid)
        else:
            results.append(r)
    return left


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batch-2d-64":
        return run_batched(args, rank, world, local)
    if args.workload == "serve-mixed":
        return run_serving(args, rank, world, local)
    info = run_ours(args, rank, world, local)
    if rank != 0:
        return 0
    st = info["stats"]
    K = args.steps
    ms_step = info["t_ms"] / K
    value = info["updates_per_step"] * K * world / (info["t_ms"] * 1e-3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ("f32" if args.coeff_dtype == "f32" else
                      f"{args.coeff_dtype} coefficients, f32 accumulation and image"),
            "data": "synthetic",
            "config": {"workload": args.workload, "rings": info["spec"]["n_rings"],
                       "slabs": info["spec"]["n_slabs"] if info["spec"]["geometry"] == 1 else 1,
                       "views": st["n_views"],
                       "detector": [info["spec"]["n_u"], info["spec"]["n_v"] if info["spec"]["geometry"] == 1 else 1],
                       "geometry": ("parallel-2d", "cone-3d", "fan-2d")[info["spec"]["geometry"]],
                       "iterations": info["spec"]["iterations"], "schedule": info["spec"].get("schedule", "per_view"),
                       "update_rule": "eq18-linear" if info["spec"].get("rule", 0) == 1 else "power",
                       "lambda": info["spec"]["lam"],
                       "coeff_dtype": args.coeff_dtype,
                       "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas{world}",
                       "step": "coefficient build + MART + resample",
                       "launch_shape": dict(zip(["fwd_blocks_per_sm", "bwd_blocks_per_sm"], info["tuned"]))},
            "ms_per_iteration": info["ms_mart"] / info["spec"]["iterations"],
            "phases_ms": {"coefficients": round(info["ms_build"], 3), "mart": round(info["ms_mart"], 3),
                          "resample": round(info["ms_resample"], 3)},
            "store": {"reps": st["n_reps"], "nnz_store": st["nnz_store"], "nnz_all_views": st["nnz_all_views"],
                      "store_bytes": st["store_bytes"], "full_matrix_bytes": st["full_matrix_bytes"]},
            "gpu_launches": int(info["launches"]),
            "clocks": info["clk"], "roofline": roofline(info) if info["fw"] is not None else latency_line(info)}
    if info["e2e"]:
        t_e2e, hb, db = info["e2e"]
        line["e2e"] = {"value": info["updates_per_step"] * K * world / (t_e2e * 1e-3), "unit": UNIT,
                       "h2d_bytes_per_step": hb, "d2h_bytes_per_step": db, "ms_per_step": t_e2e / K}
    if info.get("quality"):
        q = info["quality"]
        line["quality"] = {"mae": round(q["mae"], 5), "rmse": round(q["rmse"], 5), "ssim": round(q["ssim"], 4),
                           "vs": "seeded phantom at the resampled image's pixel centres (MAE/RMSE inside the disk)",
                           "pixels": q["pixels"], "phantom_range": round(q["phantom_range"], 4)}
    if not args.no_cpu_baseline and world == 1:
        v, thr, dt, nnz = oracle_sample(info["spec"], info["proj"])
        what = (f"the whole {info['spec']['iterations']}-iteration ray-sequential run ({nnz} ray-cell updates, "
                f"{dt:.1f} s)" if info["fw"] is None else f"one per-view MART step of view 0 ({nnz} nonzeros, {dt:.1f} s)")
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": what}
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
