"""FP64 CPU oracle for USPG/USCG MART (arXiv 2208.12964) -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never loads it and shares no code with it: the oracle is a
plain C program (``uspg_oracle.c``) compiled with gcc, reached here through
ctypes.

Functions mirror the paper's steps; see the C file for the passages each one
follows and the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "uspg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

SECT_6N, SECT_4_2N1, SECT_CUSTOM = 0, 1, 2
PARALLEL_2D, CONE_3D, FAN_2D = 0, 1, 2
LENGTH, BINARY = 0, 1
POWER, LINEAR_EQ18 = 0, 1
STORE_ROWS, STORE_SEGMENTS = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, so results do not
    depend on whether the host has fused multiply-add)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared"]
        cmd = base + ["-fopenmp", "-o", _LIB, _SRC, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:  # no OpenMP runtime: build single-threaded
            r = subprocess.run(base + ["-o", _LIB, _SRC, "-lm"], capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError("oracle build failed:\n" + r.stderr)
    return _LIB


class Problem(C.Structure):
    _fields_ = [
        ("n_rings", C.c_int32), ("n_slabs", C.c_int32), ("sector_rule", C.c_int32), ("geometry", C.c_int32),
        ("r", C.c_double), ("h", C.c_double), ("z_min", C.c_double),
        ("n_views", C.c_int32), ("n_u", C.c_int32), ("n_v", C.c_int32), ("weight_mode", C.c_int32),
        ("arc_num", C.c_int64), ("arc_den", C.c_int64),
        ("du", C.c_double), ("dv", C.c_double), ("d_so", C.c_double), ("d_sd", C.c_double),
        ("custom_sectors", C.c_void_p),
        ("store_form", C.c_int32),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            P, V = C.POINTER, C.c_void_p
            L.orc_create.restype = V
            L.orc_create.argtypes = [P(Problem)]
            L.orc_destroy.argtypes = [V]
            L.orc_set_threads.argtypes = [V, C.c_int32]
            for n in ("orc_cells", "orc_cells_per_slab"):
                getattr(L, n).restype = C.c_int64
                getattr(L, n).argtypes = [V]
            for n in ("orc_rays", "orc_gcd"):
                getattr(L, n).restype = C.c_int32
                getattr(L, n).argtypes = [V]
            L.orc_grid_tables.restype = C.c_int32
            L.orc_grid_tables.argtypes = [V, V, V]
            for n in ("orc_trace", "orc_trace_rotated", "orc_rebin_row"):
                getattr(L, n).restype = C.c_int32
                getattr(L, n).argtypes = [V, C.c_int32, C.c_int32, C.c_int32, V, V]
            L.orc_segments.restype = C.c_int32
            L.orc_segments.argtypes = [V, C.c_int32, C.c_int32, V, V, V, V, V, V]
            L.orc_view_turns.restype = C.c_uint64
            L.orc_view_turns.argtypes = [V, C.c_int32]
            L.orc_view_classes.restype = C.c_int32
            L.orc_view_classes.argtypes = [V, V, V]
            L.orc_view_nnz.restype = C.c_int64
            L.orc_view_nnz.argtypes = [V, C.c_int32]
            L.orc_forward.argtypes = [V, C.c_int32, V, V]
            L.orc_mart_sequential.restype = C.c_int32
            L.orc_mart_sequential.argtypes = [V, V, V, C.c_int32, C.c_double, C.c_int32, C.c_double]
            L.orc_mart_per_view.restype = C.c_int32
            L.orc_mart_per_view.argtypes = [V, V, V, C.c_int32, C.c_double, V, C.c_int32, C.c_double]
            L.orc_mart_views_sample.restype = C.c_int64
            L.orc_mart_views_sample.argtypes = [V, V, V, V, C.c_int32, C.c_double]
            L.orc_resample_point.argtypes = [V, V, C.c_int32, C.c_int32, V]
            L.orc_resample_bijection.restype = C.c_int32
            L.orc_resample_bijection.argtypes = [V, V, V]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class Oracle:
    """One problem (grid + scan) in the FP64 oracle.

    ``spec`` is a dict with the keys of :class:`Problem` (missing keys take
    2D defaults); ``custom_sectors`` may be a sequence of per-ring counts.
    """

    def __init__(self, spec: dict, threads: int = 1):
        L = _load()
        self._keep = None
        d = dict(n_rings=1, n_slabs=1, sector_rule=SECT_6N, geometry=PARALLEL_2D, r=1.0, h=1.0, z_min=0.0,
                 n_views=1, n_u=1, n_v=1, weight_mode=LENGTH, arc_num=1, arc_den=2, du=1.0, dv=1.0,
                 d_so=1.0, d_sd=2.0, store_form=STORE_ROWS)
        d.update({k: v for k, v in spec.items() if k != "custom_sectors"})
        p = Problem(**{k: d[k] for k, _ in Problem._fields_ if k != "custom_sectors"})
        if spec.get("custom_sectors") is not None:
            self._keep = np.ascontiguousarray(spec["custom_sectors"], dtype=np.int32)
            p.custom_sectors = self._keep.ctypes.data
        self.spec = d
        self._h = L.orc_create(C.byref(p))
        if not self._h:
            raise ValueError("oracle rejected the problem description")
        L.orc_set_threads(self._h, int(threads))
        self.L = L
        self.n_cells = L.orc_cells(self._h)
        self.cells_per_slab = L.orc_cells_per_slab(self._h)
        self.n_rays = L.orc_rays(self._h)
        self.G = L.orc_gcd(self._h)
        self.n_views = d["n_views"]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self.L.orc_destroy(h)
            self._h = None

    def set_threads(self, n: int):
        self.L.orc_set_threads(self._h, int(n))

    def grid_tables(self):
        N = self.spec["n_rings"]
        ng = np.zeros(N, np.int32)
        head = np.zeros(N, np.int64)
        self.L.orc_grid_tables(self._h, _ptr(ng), _ptr(head))
        return ng, head

    def _row(self, fn, view, ray):
        cap = 512
        while True:
            cells = np.zeros(cap, np.int64)
            w = np.zeros(cap, np.float64)
            n = fn(self._h, int(view), int(ray), cap, _ptr(cells), _ptr(w))
            if n >= 0:
                return cells[:n].copy(), w[:n].copy()
            cap = -n

    def row(self, view: int, ray: int):
        """Directly traced row: (cells ascending, weights)."""
        return self._row(self.L.orc_trace, view, ray)

    def row_rotated(self, view: int, ray: int):
        """Row rebuilt from the view's representative by sector rotation."""
        return self._row(self.L.orc_trace_rotated, view, ray)

    def rebin_row(self, view: int, ray: int):
        """Binary row of a view from the first view's segments (Algorithm 1)."""
        return self._row(self.L.orc_rebin_row, view, ray)

    def segments(self, ray: int):
        """Segments of a first-view ray: (ring, slab, azimuth in, azimuth out
        (uint64 fixed turns), length, direction of turn)."""
        cap = 2 * self.spec["n_rings"] + self.spec["n_slabs"] + 8
        rg = np.zeros(cap, np.int32)
        sb = np.zeros(cap, np.int32)
        fa = np.zeros(cap, np.uint64)
        fb = np.zeros(cap, np.uint64)
        ln = np.zeros(cap, np.float64)
        dr = np.zeros(1, np.int32)
        n = self.L.orc_segments(self._h, int(ray), cap, _ptr(rg), _ptr(sb), _ptr(fa), _ptr(fb), _ptr(ln), _ptr(dr))
        assert n >= 0
        return rg[:n], sb[:n], fa[:n], fb[:n], ln[:n], int(dr[0])

    def view_turns(self, view: int) -> int:
        return int(self.L.orc_view_turns(self._h, int(view)))

    def view_classes(self):
        rep = np.zeros(self.n_views, np.int32)
        sh = np.zeros(self.n_views, np.int32)
        n = self.L.orc_view_classes(self._h, _ptr(rep), _ptr(sh))
        return n, rep, sh

    def view_nnz(self, view: int) -> int:
        return int(self.L.orc_view_nnz(self._h, int(view)))

    def forward(self, view: int, f: np.ndarray) -> np.ndarray:
        f = np.ascontiguousarray(f, np.float64)
        s = np.zeros(self.n_rays, np.float64)
        self.L.orc_forward(self._h, int(view), _ptr(f), _ptr(s))
        return s

    def mart_sequential(self, proj, f0, iters, lam, rule=POWER, tol=0.0):
        proj = np.ascontiguousarray(proj, np.float32).reshape(-1)
        f = np.array(f0, np.float64, copy=True).reshape(-1)
        n = self.L.orc_mart_sequential(self._h, _ptr(proj), _ptr(f), int(iters), float(lam), int(rule), float(tol))
        return f, int(n)

    def mart_per_view(self, proj, f0, iters, lam, order=None, rule=POWER, tol=0.0, return_sweeps=False):
        """Per-view simultaneous MART (geometric-mean POWER or arithmetic-mean
        LINEAR_EQ18 combination of the view's rays, Eq. 18), up to ``iters``
        sweeps, stopping early by Eq. 19 when ``tol`` > 0.  Returns the image,
        or (image, sweeps run) with ``return_sweeps``."""
        proj = np.ascontiguousarray(proj, np.float32).reshape(-1)
        f = np.array(f0, np.float64, copy=True).reshape(-1)
        o = None
        if order is not None:
            o = np.ascontiguousarray(order, np.int32)
        n = self.L.orc_mart_per_view(self._h, _ptr(proj), _ptr(f), int(iters), float(lam),
                                     _ptr(o) if o is not None else None, int(rule), float(tol))
        return (f, int(n)) if return_sweeps else f

    def mart_views_sample(self, proj, f, views, lam):
        """One per-view step for each view in ``views`` (f updated in place);
        returns the nonzeros processed."""
        proj = np.ascontiguousarray(proj, np.float32).reshape(-1)
        v = np.ascontiguousarray(views, np.int32)
        return int(self.L.orc_mart_views_sample(self._h, _ptr(proj), _ptr(f), _ptr(v), len(v), float(lam)))

    def resample_point(self, f, nx, ny):
        f = np.ascontiguousarray(f, np.float64)
        ns = self.spec["n_slabs"] if self.spec["geometry"] == CONE_3D else 1
        out = np.zeros((ns, ny, nx), np.float64)
        self.L.orc_resample_point(self._h, _ptr(f), int(nx), int(ny), _ptr(out))
        return out

    def resample_bijection(self, f):
        f = np.ascontiguousarray(f, np.float64)
        ns = self.spec["n_slabs"] if self.spec["geometry"] == CONE_3D else 1
        W = 2 * self.spec["n_rings"]
        out = np.zeros((ns, W, W), np.float64)
        if self.L.orc_resample_bijection(self._h, _ptr(f), _ptr(out)) != 0:
            raise ValueError("bijective resample needs the 4(2n-1) sector rule")
        return out
