"""Host arithmetic of bench.py's JSON line (no GPU): the roofline object of the
dominant per-view kernel, the DRAM-traffic record keyed by the kernel
sources' hash, and the latency line of the ray-sequential schedule."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2208_12964_gb300 import synth  # noqa: E402


def _info(fw_ms, bw_ms, weight_bytes=4):
    spec = synth.workload("3d-cone-128r-128s-90v-256")
    stats = dict(n_rays=65536, nnz_store=77217546, n_reps=15, n_cells=6340608, slices=102912, mirrored=1,
                 n_views=90)
    return dict(stats=stats, fw=[fw_ms] * 4, bw=[bw_ms] * 4, weight_bytes=weight_bytes, coeff_dtype="f32",
                spec=spec, ms_mart=23.0)


def test_roofline_is_algorithmic_bytes_over_mean_launch_time():
    info = _info(0.027, 0.033)
    r = bench.roofline(info)
    S = 77217546 / 15
    bwd = S * 8 + 102912 * 72 + 6340608 * 8 + 65536 * 16
    assert r["kernel"] == "k_backward" and r["bytes_per_launch"] == int(bwd)
    assert abs(r["achieved"] - bwd / 0.033e-3 / 1e9) < 0.1
    peak, src = bench.load_peaks()
    assert r["peak"] == peak and abs(r["frac"] - r["achieved"] / peak) < 1e-4
    assert r["unit"] == "GB/s" and r["bound"] == "hbm"
    # the forward becomes the dominant kernel when it is the slower one
    r2 = bench.roofline(_info(0.05, 0.033))
    fwd = S * 8 + S / 8 * 4 + 65536 * 12
    assert r2["kernel"] == "k_forward" and r2["bytes_per_launch"] == int(fwd)


def test_traffic_record_matches_its_sources_and_geometry():
    rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic_cone128_mart.json")))
    spec = synth.workload("3d-cone-128r-128s-90v-256")
    t = bench.measured_traffic("k_backward", "f32", True, spec)
    # a capture belongs to the kernel sources it was taken from: while they are
    # unchanged the line reports its bytes, after a change null (until a new capture)
    if bench.sources_hash_matches(rec):
        assert t == rec["kernels"]["128r-128s-256x256/k_backward/f32/mirrored"]["dram_bytes_per_launch"]
    else:
        assert t is None
    # no record for another geometry or store form: the line says null, not a guess
    assert bench.measured_traffic("k_backward", "f32", True, synth.workload("3d-cone-256r-256s-180v-512")) is None
    assert bench.measured_traffic("k_backward", "f16", True, spec) is None


def test_latency_line_of_the_sequential_schedule():
    info = dict(stats=dict(n_views=50, n_rays=101), spec=dict(iterations=10), ms_mart=99.9)
    r = bench.latency_line(info)
    assert r["ray_steps"] == 50500 and r["unit"] == "us per ray step"
    assert abs(r["achieved"] - 99.9e3 / 50500) < 1e-3 and r["frac"] is None
