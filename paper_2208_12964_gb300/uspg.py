"""ctypes binding of libuspg (include/uspg.h) -- argument marshalling only.

Every function has the name of the C entry point it calls and raises
``UspgError`` on a non-OK status.  All computation happens in the CUDA
library; importing this module without the built library raises at once
(there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libuspg.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED, EBUSY, ENOTREADY, EDEVICE = range(9)
SECT_6N, SECT_4_2N1, SECT_CUSTOM = 0, 1, 2
PARALLEL_2D, CONE_3D, FAN_2D = 0, 1, 2
LENGTH, BINARY = 0, 1
STORE_REPRESENTATIVES, STORE_SEGMENTS = 0, 1
SYMMETRY_AUTO, SYMMETRY_ALWAYS, SYMMETRY_NEVER = 0, 1, 2
F32, F16, BF16 = 0, 1, 2
SEQUENTIAL, PER_VIEW = 0, 1
POWER, LINEAR_EQ18 = 0, 1
RESAMPLE_POINT, RESAMPLE_BIJECTION = 0, 1
JOB_BORROW_PROJECTIONS = 1


class UspgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libuspg status {status}: {msg}")
        self.status = status


class GridDesc(C.Structure):
    _fields_ = [("n_rings", C.c_int32), ("sector_rule", C.c_int32), ("sectors", C.c_void_p),
                ("ring_width", C.c_double), ("n_slabs", C.c_int32), ("reserved", C.c_int32),
                ("slab_height", C.c_double), ("z_min", C.c_double)]


class ScanDesc(C.Structure):
    _fields_ = [("geometry", C.c_int32), ("n_views", C.c_int32), ("arc_num", C.c_int64), ("arc_den", C.c_int64),
                ("n_u", C.c_int32), ("n_v", C.c_int32), ("du", C.c_double), ("dv", C.c_double),
                ("src_to_axis", C.c_double), ("src_to_det", C.c_double)]


class CoeffOpts(C.Structure):
    _fields_ = [("weight_mode", C.c_int32), ("coeff_dtype", C.c_int32), ("store_form", C.c_int32),
                ("symmetry", C.c_int32)]


class MartOpts(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("schedule", C.c_int32), ("update_rule", C.c_int32),
                ("view_steps", C.c_int32), ("lambda_", C.c_double), ("stop_tol", C.c_double),
                ("view_order", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("n_cells", "cells_per_slab", "n_rays", "n_views", "n_reps", "nnz_store",
                                         "nnz_all_views", "store_bytes", "full_matrix_bytes", "max_row", "gcd",
                                         "mirrored", "slices", "walked_rows", "derived_reps")]


class Job(C.Structure):
    _fields_ = [("grid", GridDesc), ("scan", ScanDesc), ("coeff", CoeffOpts), ("mart", MartOpts),
                ("projections", C.c_void_p), ("f0", C.c_float), ("flags", C.c_int32)]


class JobResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("reused_store", C.c_int32), ("n_cells", C.c_int64), ("updates", C.c_int64),
                ("queue_s", C.c_double), ("run_s", C.c_double), ("latency_s", C.c_double),
                ("message", C.c_char * 200)]


class ServerReport(C.Structure):
    _fields_ = ([(n, C.c_int64) for n in ("submitted", "completed", "failed", "queued", "active", "store_reuses",
                                          "device_bytes", "peak_device_bytes")]
                + [(n, C.c_double) for n in ("p50_s", "p99_s", "mean_s", "jobs_per_s", "updates_per_s")])


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libuspg is not built ({LIB_PATH} missing): run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        P, V, I32, I64 = C.POINTER, C.c_void_p, C.c_int32, C.c_int64
        sig = {
            "uspg_create": ([P(GridDesc), P(ScanDesc), P(CoeffOpts), P(V)], I32),
            "uspg_destroy": ([V], None),
            "uspg_last_error": ([V], C.c_char_p),
            "uspg_sync": ([V, V], I32),
            "uspg_build_coeffs": ([V, V], I32),
            "uspg_coeff_stats": ([V, P(Stats)], I32),
            "uspg_get_row": ([V, I32, I32, I32, V, V, P(I32)], I32),
            "uspg_set_projections": ([V, V, I32, V], I32),
            "uspg_set_image": ([V, V, I32, V], I32),
            "uspg_fill_image": ([V, C.c_float, V], I32),
            "uspg_get_image": ([V, V, I32, V], I32),
            "uspg_mart": ([V, P(MartOpts), V], I32),
            "uspg_forward_project": ([V, I32, V, V], I32),
            "uspg_mart_sweeps": ([V, P(I32)], I32),
            "uspg_resample_cartesian": ([V, I32, I32, I32, V, I32, V], I32),
            "uspg_kernel_launches": ([], I64),
            "uspg_mart_kernel_times": ([V, P(MartOpts), V, V, I32, P(I32), V], I32),
            "uspg_autotune": ([V, V, V], I32),
            "uspg_forward_project_noalloc": ([V, I32, V, V, V], I32),
            "uspg_batch_create": ([V, I32, P(MartOpts), V, P(V)], I32),
            "uspg_batch_run": ([V, V], I32),
            "uspg_batch_info": ([V, P(I64), P(I64), P(I64)], I32),
            "uspg_batch_tuning": ([V, I32, V, V, V, P(I32), P(C.c_float), P(C.c_float)], I32),
            "uspg_batch_destroy": ([V], None),
            "uspg_server_create": ([C.c_size_t, I32, I32, P(V)], I32),
            "uspg_server_submit": ([V, P(Job), P(C.c_uint64)], I32),
            "uspg_server_poll": ([V, C.c_uint64, V, P(JobResult)], I32),
            "uspg_server_drain": ([V, C.c_double], I32),
            "uspg_server_stats": ([V, P(ServerReport)], I32),
            "uspg_server_destroy": ([V], None),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def exported_symbols():
    """Names of the C entry points this binding expects."""
    lib()
    return [n for n in dir(_lib) if n.startswith("uspg_")]


def _check(st, ctx=None):
    if st != OK:
        msg = lib().uspg_last_error(ctx)
        raise UspgError(st, msg.decode() if msg else "")


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream", stream))


def _ptr(x):
    """Address of a numpy array (host) or a torch tensor (device or host)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return int(x.data_ptr())


def descs_from_spec(spec: dict, dtype: int = F32, weight_mode: int | None = None, store_form: int | None = None):
    """C descriptors for a workload description (see synth.workload)."""
    g = GridDesc(n_rings=spec["n_rings"], sector_rule=spec["sector_rule"], sectors=None, ring_width=spec["r"],
                 n_slabs=spec["n_slabs"] if spec["geometry"] == CONE_3D else 1, reserved=0,
                 slab_height=spec["h"], z_min=spec["z_min"])
    keep = None
    if spec.get("custom_sectors") is not None:
        keep = np.ascontiguousarray(spec["custom_sectors"], np.int32)
        g.sectors = keep.ctypes.data
    s = ScanDesc(geometry=spec["geometry"], n_views=spec["n_views"], arc_num=spec["arc_num"],
                 arc_den=spec["arc_den"], n_u=spec["n_u"], n_v=spec["n_v"] if spec["geometry"] == CONE_3D else 1,
                 du=spec["du"], dv=spec["dv"], src_to_axis=spec["d_so"], src_to_det=spec["d_sd"])
    if weight_mode is None:
        weight_mode = spec.get("weight_mode", LENGTH)
    if store_form is None:
        store_form = spec.get("store_form", STORE_REPRESENTATIVES)
    o = CoeffOpts(weight_mode=weight_mode, coeff_dtype=dtype, store_form=store_form,
                  symmetry=spec.get("symmetry", SYMMETRY_AUTO))
    return g, s, o, keep


def uspg_create(grid: GridDesc, scan: ScanDesc, opts: CoeffOpts | None = None):
    h = C.c_void_p()
    st = lib().uspg_create(C.byref(grid), C.byref(scan), C.byref(opts) if opts is not None else None, C.byref(h))
    _check(st, None)
    return h.value


def uspg_destroy(ctx):
    lib().uspg_destroy(ctx)


def uspg_last_error(ctx):
    m = lib().uspg_last_error(ctx)
    return m.decode() if m else ""


def uspg_sync(ctx, stream=None):
    _check(lib().uspg_sync(ctx, _stream(stream)), ctx)


def uspg_build_coeffs(ctx, stream=None):
    _check(lib().uspg_build_coeffs(ctx, _stream(stream)), ctx)


def uspg_coeff_stats(ctx) -> dict:
    s = Stats()
    _check(lib().uspg_coeff_stats(ctx, C.byref(s)), ctx)
    return {n: getattr(s, n) for n, _ in Stats._fields_}


def uspg_get_row(ctx, view: int, ray: int):
    n = C.c_int32(0)
    st = lib().uspg_get_row(ctx, view, ray, 0, None, None, C.byref(n))
    if st not in (OK, EINVAL) or (st == EINVAL and n.value == 0):
        _check(st, ctx)
    cap = max(n.value, 1)
    cells = np.zeros(cap, np.int64)
    w = np.zeros(cap, np.float64)
    _check(lib().uspg_get_row(ctx, view, ray, cap, cells.ctypes.data, w.ctypes.data, C.byref(n)), ctx)
    return cells[:n.value], w[:n.value]


def uspg_set_projections(ctx, p, on_device: bool, stream=None):
    _check(lib().uspg_set_projections(ctx, _ptr(p), int(on_device), _stream(stream)), ctx)


def uspg_set_image(ctx, f, on_device: bool, stream=None):
    _check(lib().uspg_set_image(ctx, _ptr(f), int(on_device), _stream(stream)), ctx)


def uspg_fill_image(ctx, value: float, stream=None):
    _check(lib().uspg_fill_image(ctx, float(value), _stream(stream)), ctx)


def uspg_get_image(ctx, f, to_device: bool, stream=None):
    _check(lib().uspg_get_image(ctx, _ptr(f), int(to_device), _stream(stream)), ctx)


def mart_opts(iterations: int, lam: float, schedule: int, rule: int = POWER, stop_tol: float = 0.0,
              view_order=None, view_steps: int = 0):
    keep = None
    o = MartOpts(iterations=iterations, schedule=schedule, update_rule=rule, view_steps=view_steps, lambda_=lam,
                 stop_tol=stop_tol, view_order=None)
    if view_order is not None:
        keep = np.ascontiguousarray(view_order, np.int32)
        o.view_order = keep.ctypes.data
    return o, keep


def uspg_mart(ctx, opts: MartOpts, stream=None):
    _check(lib().uspg_mart(ctx, C.byref(opts), _stream(stream)), ctx)


def uspg_forward_project(ctx, view: int, out, stream=None):
    _check(lib().uspg_forward_project(ctx, view, _ptr(out), _stream(stream)), ctx)


def uspg_mart_sweeps(ctx) -> int:
    n = C.c_int32(0)
    _check(lib().uspg_mart_sweeps(ctx, C.byref(n)), ctx)
    return n.value


def uspg_resample_cartesian(ctx, mode: int, nx: int, ny: int, out, on_device: bool, stream=None):
    _check(lib().uspg_resample_cartesian(ctx, mode, nx, ny, _ptr(out), int(on_device), _stream(stream)), ctx)


def uspg_kernel_launches() -> int:
    return int(lib().uspg_kernel_launches())


def uspg_mart_kernel_times(ctx, opts: MartOpts, steps: int, stream=None):
    """Per-launch device milliseconds (forward, backward) of a per-view MART."""
    fw = np.zeros(max(steps, 1), np.float32)
    bw = np.zeros(max(steps, 1), np.float32)
    n = C.c_int32(0)
    _check(lib().uspg_mart_kernel_times(ctx, C.byref(opts), fw.ctypes.data, bw.ctypes.data, len(fw), C.byref(n),
                                        _stream(stream)), ctx)
    return fw[:n.value], bw[:n.value]


def uspg_autotune(ctx, stream=None):
    """Times the per-view kernels' launch shapes; returns the choice
    (forward blocks per SM, correction blocks per SM)."""
    ch = np.zeros(2, np.int32)
    _check(lib().uspg_autotune(ctx, ch.ctypes.data, _stream(stream)), ctx)
    return tuple(int(x) for x in ch)


NOALLOC_MAX_RAYS = 1 << 20


def uspg_forward_project_noalloc(ctx, view: int, f, out, stream=None):
    """Forward projection of one view into ``out`` with no device allocation
    (accumulator in the library's static device array); ``f`` and ``out`` are
    device tensors."""
    _check(lib().uspg_forward_project_noalloc(ctx, view, _ptr(f), _ptr(out), _stream(stream)), ctx)


def uspg_batch_create(ctxs, opts: MartOpts, stream=None):
    """Batched per-view MART over several contexts (one CUDA graph)."""
    arr = (C.c_void_p * len(ctxs))(*ctxs)
    h = C.c_void_p()
    _check(lib().uspg_batch_create(arr, len(ctxs), C.byref(opts), _stream(stream), C.byref(h)), None)
    return h.value


def uspg_batch_run(batch, stream=None):
    _check(lib().uspg_batch_run(batch, _stream(stream)), None)


def uspg_batch_info(batch) -> dict:
    u, k, s = C.c_int64(0), C.c_int64(0), C.c_int64(0)
    _check(lib().uspg_batch_info(batch, C.byref(u), C.byref(k), C.byref(s)), None)
    return {"updates_per_run": u.value, "kernel_nodes": k.value, "steps": s.value}


def uspg_batch_tuning(batch) -> dict:
    cap = 64
    rings = np.zeros(cap, np.int32)
    fr = np.zeros(cap, np.float64)
    br = np.zeros(cap, np.float64)
    n = C.c_int32(0)
    t0, t1 = C.c_float(0), C.c_float(0)
    _check(lib().uspg_batch_tuning(batch, cap, rings.ctypes.data, fr.ctypes.data, br.ctypes.data, C.byref(n),
                                   C.byref(t0), C.byref(t1)), None)
    k = n.value
    return {"buckets": [{"rings": int(rings[q]), "fwd_blocks_per_group": float(fr[q]),
                         "bwd_blocks_per_slice": float(br[q])} for q in range(k)],
            "ms_default": t0.value, "ms_tuned": t1.value}


def uspg_batch_destroy(batch):
    lib().uspg_batch_destroy(batch)


def uspg_server_create(device_budget: int, max_active: int, chunk_sweeps: int):
    """Reconstruction server on the current device (scheduler and preparer
    threads in the library)."""
    h = C.c_void_p()
    _check(lib().uspg_server_create(device_budget, max_active, chunk_sweeps, C.byref(h)), None)
    return h.value


def uspg_server_submit(server, spec: dict, projections, opts: MartOpts, dtype: int = F32,
                       weight_mode: int = LENGTH, f0: float = 1.0, borrow: bool = False) -> int:
    """Queues one reconstruction of workload ``spec`` (see synth.workload) with
    host float32 ``projections`` [views][rays] (a numpy array, or a host torch
    tensor); returns the job id.  borrow: the server reads ``projections`` in
    place, so the caller keeps it unchanged until the job has been polled."""
    g, s, o, keep = descs_from_spec(spec, dtype, weight_mode)
    if isinstance(projections, np.ndarray):
        projections = np.ascontiguousarray(projections, np.float32)
        addr = projections.ctypes.data
    else:
        if not projections.is_contiguous() or projections.is_cuda or str(projections.dtype) != "torch.float32":
            raise ValueError("projections: contiguous host float32")
        addr = int(projections.data_ptr())
    job = Job(grid=g, scan=s, coeff=o, mart=opts, projections=addr, f0=f0,
              flags=JOB_BORROW_PROJECTIONS if borrow else 0)
    jid = C.c_uint64(0)
    _check(lib().uspg_server_submit(server, C.byref(job), C.byref(jid)), None)
    del keep
    return jid.value


def uspg_server_poll(server, job_id: int, image: np.ndarray | None = None):
    """None while the job runs; else its result as a dict (``status`` is the
    job's own outcome) with the image written into ``image`` (host float32)."""
    r = JobResult()
    st = lib().uspg_server_poll(server, job_id, _ptr(image), C.byref(r))
    if st == ENOTREADY:
        return None
    _check(st, None)
    out = {n: getattr(r, n) for n, _ in JobResult._fields_}
    out["message"] = r.message.decode(errors="replace")
    return out


def uspg_server_drain(server, timeout_s: float):
    _check(lib().uspg_server_drain(server, timeout_s), None)


def uspg_server_stats(server) -> dict:
    r = ServerReport()
    _check(lib().uspg_server_stats(server, C.byref(r)), None)
    return {n: getattr(r, n) for n, _ in ServerReport._fields_}


def uspg_server_destroy(server):
    lib().uspg_server_destroy(server)
