"""Seeded synthetic inputs: workload descriptions, phantoms and projections.

This module is shared by the CUDA path's tests and benchmark and by the FP64
oracle's tests.  It holds none of the reconstruction method's arithmetic: it
does not trace the polar/cylindrical grid, form coefficients or run MART.  It
only describes scans, draws random phantoms (ellipses / ellipsoids, standing in
for the paper's soil/softwood/foam and Shepp-Logan phantoms, Table 1, which the
paper does not define), integrates them analytically along the scan rays and
adds Poisson counting noise.  Randomness comes from SplitMix64 (Steele, Lea,
Flood 2014) so that both sides receive identical arrays.

Scan conventions (the same ones the library and the oracle state):
  * parallel 2D: view k at angle 2*pi*k*arc/p; detector axis (cos, sin), rays
    along (-sin, cos); bin b at u = (2b - (B-1)) * du/2.
  * cone 3D: source (-d_so, 0, 0), detector centre (d_sd - d_so, 0, 0), axes
    e_u = (0,1,0), e_v = (0,0,1), pixel (a, c) at ((2a-(Nu-1)) du/2,
    (2c-(Nv-1)) dv/2), ray index c*Nu + a; the whole set rotates about z.
  * fan 2D: source (-d_so, 0), line detector centred at (d_sd - d_so, 0)
    along e_u = (0,1), bin a at u = (2a-(Nu-1)) du/2; rotates about the axis.
"""
from __future__ import annotations

import math
import re

import numpy as np

SECT_6N, SECT_4_2N1, SECT_CUSTOM = 0, 1, 2
PARALLEL_2D, CONE_3D, FAN_2D = 0, 1, 2
POWER, LINEAR_EQ18 = 0, 1
LENGTH, BINARY = 0, 1
STORE_REPRESENTATIVES, STORE_SEGMENTS = 0, 1

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied to states ``x`` (uint64)."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniforms(seed: int, counters: np.ndarray) -> np.ndarray:
    """53-bit uniforms in [0, 1) from counter-based SplitMix64."""
    with np.errstate(over="ignore"):
        base = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _GAMMA
        x = splitmix64(np.asarray(counters, dtype=np.uint64) * _GAMMA + base)
    return (x >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


class Stream:
    """Sequential SplitMix64 stream (for phantom parameters)."""

    def __init__(self, seed: int):
        self.seed = seed
        self.n = 0

    def u(self, n: int = 1) -> np.ndarray:
        c = np.arange(self.n, self.n + n, dtype=np.uint64)
        self.n += n
        return uniforms(self.seed, c)


# --------------------------------------------------------------- workloads --

def workload(name: str) -> dict:
    """Problem description of a named workload (grid + scan + MART options)."""
    if name == "2d-parallel-64r-36v":
        return dict(name=name, n_rings=64, r=1.0 / 64, n_slabs=1, h=1.0, z_min=0.0, sector_rule=SECT_6N,
                    geometry=PARALLEL_2D, n_views=36, arc_num=1, arc_den=2, n_u=65, n_v=1, du=2.0 / 65, dv=1.0,
                    d_so=1.0, d_sd=2.0, iterations=10, lam=0.2, schedule="sequential", seed=1, noise=False)
    if name == "2d-fan-128r-50v-101":
        return fan_workload(128, 50, name=name)
    if name == "2d-fan-128r-50v-101-segments":  # the paper's binary coefficients from the first view's segments
        return dict(fan_workload(128, 50, name=name), weight_mode=BINARY, store_form=STORE_SEGMENTS)
    if name == "3d-cone-128r-128s-90v-256":
        return cone_workload(128, 128, 90, 256, iterations=5, lam=0.1, seed=2, name=name)
    if name == "3d-cone-256r-256s-180v-512":
        return cone_workload(256, 256, 180, 512, iterations=5, lam=0.1, seed=3, name=name)
    m = re.fullmatch(r"3d-cone-(\d+)r-(\d+)s-(\d+)v-(\d+)", name)
    if m:  # same cone geometry at other sizes (profiling and test cases)
        R, S, V, D = map(int, m.groups())
        return cone_workload(R, S, V, D, iterations=5, lam=0.1, seed=2, name=name)
    raise KeyError(name)


def cone_workload(rings: int, slabs: int, views: int, det: int, iterations=5, lam=0.1, seed=2, name=None,
                  noise=True) -> dict:
    """Cone-beam cylinder of radius 1 and height 2 (h = 2/slabs, centred on
    z = 0), source at 4R, detector at 8R, pitch 2*(8/3)R/det so the detector
    covers the magnified cylinder (near-edge magnification 8/3)."""
    return dict(name=name or f"3d-cone-{rings}r-{slabs}s-{views}v-{det}", n_rings=rings, r=1.0 / rings,
                n_slabs=slabs, h=2.0 / slabs, z_min=-1.0, sector_rule=SECT_6N, geometry=CONE_3D, n_views=views,
                arc_num=1, arc_den=1, n_u=det, n_v=det, du=2.0 * (8.0 / 3.0) / det, dv=2.0 * (8.0 / 3.0) / det,
                d_so=4.0, d_sd=8.0, iterations=iterations, lam=lam, schedule="per_view", seed=seed, noise=noise)


def fan_workload(rings: int, views: int, bins: int = 101, du: float = 0.05, d_so: float = 8.0, d_sd: float = 16.0,
                 iterations=10, lam=0.4, seed=5, schedule="sequential", rule=LINEAR_EQ18, name=None) -> dict:
    """Fan-beam 2D scan of the paper's 2-D phantoms (Table 1): source at
    (-8, 0), line detector of 101 bins of 0.05 centred at (8, 0), 50 views
    over a full turn, relaxation 0.4 in the update of Eq. 18, a polar grid
    with the 4(2n-1) sector rule (rings = half the Cartesian side, so the
    256 x 256 case is 128 rings).  The object is the unit disk; at the axis
    the fan spans +-1.26, so every view sees all of it (the outermost bins
    pass beside the disk).  Table 1 gives no iteration count: 10, as for the
    parallel workload."""
    return dict(name=name or f"2d-fan-{rings}r-{views}v-{bins}", n_rings=rings, r=1.0 / rings, n_slabs=1, h=1.0,
                z_min=0.0, sector_rule=SECT_4_2N1, geometry=FAN_2D, n_views=views, arc_num=1, arc_den=1, n_u=bins,
                n_v=1, du=du, dv=du, d_so=d_so, d_sd=d_sd, iterations=iterations, lam=lam, schedule=schedule,
                rule=rule, seed=seed, noise=False)


def parallel_workload(rings: int, views: int, bins: int | None = None, arc=(1, 2), seed=1, iterations=10,
                      lam=0.2, sector_rule=SECT_6N, name=None) -> dict:
    bins = bins if bins is not None else 2 * rings + 1
    return dict(name=name or f"2d-parallel-{rings}r-{views}v", n_rings=rings, r=1.0 / rings, n_slabs=1, h=1.0,
                z_min=0.0, sector_rule=sector_rule, geometry=PARALLEL_2D, n_views=views, arc_num=arc[0],
                arc_den=arc[1], n_u=bins, n_v=1, du=2.0 / bins, dv=1.0, d_so=1.0, d_sd=2.0, iterations=iterations,
                lam=lam, schedule="per_view", seed=seed, noise=False)


def n_rays(spec: dict) -> int:
    return spec["n_u"] * (spec["n_v"] if spec["geometry"] == CONE_3D else 1)


# ------------------------------------------------------------------ geometry --

def ray_endpoints(spec: dict, view: int):
    """(S, D) arrays of shape [rays, 3] for one view."""
    frac = (view * spec["arc_num"]) / float(spec["arc_den"] * spec["n_views"])
    th = 2.0 * math.pi * frac
    ct, st = math.cos(th), math.sin(th)
    R = spec["n_rings"] * spec["r"]
    if spec["geometry"] == PARALLEL_2D:
        b = np.arange(spec["n_u"], dtype=np.float64)
        u = (2.0 * b - (spec["n_u"] - 1)) * (0.5 * spec["du"])
        L = 2.0 * R
        S = np.stack([u * ct + L * st, u * st - L * ct, np.zeros_like(u)], axis=1)
        D = np.stack([u * ct - L * st, u * st + L * ct, np.zeros_like(u)], axis=1)
        return S, D
    if spec["geometry"] == FAN_2D:
        a = np.arange(spec["n_u"], dtype=np.float64)
        u = (2.0 * a - (spec["n_u"] - 1)) * (0.5 * spec["du"])
        off = spec["d_sd"] - spec["d_so"]
        S = np.tile(np.array([-spec["d_so"] * ct, -spec["d_so"] * st, 0.0]), (spec["n_u"], 1))
        D = np.stack([off * ct - u * st, off * st + u * ct, np.zeros_like(u)], axis=1)
        return S, D
    nu, nv = spec["n_u"], spec["n_v"]
    a = np.tile(np.arange(nu, dtype=np.float64), nv)
    c = np.repeat(np.arange(nv, dtype=np.float64), nu)
    u = (2.0 * a - (nu - 1)) * (0.5 * spec["du"])
    v = (2.0 * c - (nv - 1)) * (0.5 * spec["dv"])
    off = spec["d_sd"] - spec["d_so"]
    S = np.tile(np.array([-spec["d_so"] * ct, -spec["d_so"] * st, 0.0]), (nu * nv, 1))
    D = np.stack([off * ct - u * st, off * st + u * ct, v], axis=1)
    return S, D


# ------------------------------------------------------------------ phantoms --

def ellipse_phantom(seed: int, n: int = 6, R: float = 1.0):
    """n random ellipses inside the disk of radius R: densities U[0.1, 1],
    semi-axes U[0.05, 0.4]*R, orientation U[0, pi), centres drawn so that the
    whole ellipse lies inside the disk; densities add where they overlap."""
    g = Stream(seed)
    out = []
    for _ in range(n):
        rho, a, b, ang, cr, cphi = g.u(6)
        dens = 0.1 + 0.9 * rho
        a = (0.05 + 0.35 * a) * R
        b = (0.05 + 0.35 * b) * R
        ang = math.pi * ang
        rmax = R - max(a, b)
        cr = rmax * math.sqrt(cr)
        cphi = 2.0 * math.pi * cphi
        out.append(dict(kind="ellipse", dens=dens, c=(cr * math.cos(cphi), cr * math.sin(cphi), 0.0), axes=(a, b, 1.0),
                        rot=np.array([[math.cos(ang), -math.sin(ang), 0.0], [math.sin(ang), math.cos(ang), 0.0],
                                      [0.0, 0.0, 1.0]])))
    return out


def _normals(g: Stream, n: int) -> np.ndarray:
    u1, u2 = g.u(n), g.u(n)
    return np.sqrt(-2.0 * np.log(1.0 - u1)) * np.cos(2.0 * math.pi * u2)


def ellipsoid_phantom(seed: int, n: int = 12, R: float = 1.0, zhalf: float = 1.0, blob: bool = True):
    """n random ellipsoids (values U[0.1, 1], semi-axes U[0.05, 0.4]*R, uniform
    random orientation) plus, if ``blob``, a dense sphere of radius 0.08R and
    value 5; every body lies inside the cylinder r <= R, |z| <= zhalf."""
    g = Stream(seed)
    out = []
    for _ in range(n):
        dens = 0.1 + 0.9 * float(g.u(1)[0])
        ax = (0.05 + 0.35 * g.u(3)) * R
        q = _normals(g, 4)
        q = q / np.linalg.norm(q)
        w, x, y, z = q
        rot = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
        m = float(ax.max())
        cr, cphi, cz = g.u(3)
        cr = (R - m) * math.sqrt(cr)
        cphi = 2.0 * math.pi * cphi
        cz = (2.0 * cz - 1.0) * (zhalf - m)
        out.append(dict(kind="ellipsoid", dens=dens, c=(cr * math.cos(cphi), cr * math.sin(cphi), cz),
                        axes=tuple(float(v) for v in ax), rot=rot))
    if blob:
        rb = 0.08 * R
        cr, cphi, cz = g.u(3)
        cr = (R - rb) * math.sqrt(cr)
        cphi = 2.0 * math.pi * cphi
        cz = (2.0 * cz - 1.0) * (zhalf - rb)
        out.append(dict(kind="ellipsoid", dens=5.0, c=(cr * math.cos(cphi), cr * math.sin(cphi), cz),
                        axes=(rb, rb, rb), rot=np.eye(3)))
    return out


def line_integrals(bodies, S: np.ndarray, D: np.ndarray, planar: bool) -> np.ndarray:
    """Exact integral of the phantom along each segment S->D (segments are
    long enough to cross every body).  Each body maps to the unit ball by
    x -> diag(1/axes) rot^T (x - c); the chord length of the mapped line in
    the unit ball, divided by the mapped direction's length, is the chord in
    parameter units."""
    dvec = D - S
    L = np.linalg.norm(dvec, axis=1)
    total = np.zeros(S.shape[0], np.float64)
    for b in bodies:
        c = np.asarray(b["c"], np.float64)
        M = (b["rot"].T / np.asarray(b["axes"], np.float64)[:, None])
        if planar:
            M = M[:2, :2]
            q0 = (S[:, :2] - c[:2]) @ M.T
            qd = dvec[:, :2] @ M.T
        else:
            q0 = (S - c) @ M.T
            qd = dvec @ M.T
        aa = np.einsum("ij,ij->i", qd, qd)
        bb = np.einsum("ij,ij->i", q0, qd)
        cc = np.einsum("ij,ij->i", q0, q0) - 1.0
        disc = bb * bb - aa * cc
        chord = np.where(disc > 0.0, 2.0 * np.sqrt(np.maximum(disc, 0.0)) / aa, 0.0)
        total += b["dens"] * chord * L
    return total


# ------------------------------------------------------------------- noise --

def poisson(seed: int, mean: np.ndarray) -> np.ndarray:
    """Poisson(mean) per element, counter-based so that element i draws from
    its own stream.  Means >= 10: transformed rejection with squeeze (PTRS,
    Hoermann 1993); smaller means: inversion by sequential search."""
    from scipy.special import gammaln

    mean = np.asarray(mean, np.float64)
    out = np.zeros(mean.shape, np.int64)
    idx = np.arange(mean.size, dtype=np.uint64)
    flat = mean.reshape(-1)
    res = out.reshape(-1)
    small = flat < 10.0
    # inversion for small means
    si = np.nonzero(small)[0]
    if si.size:
        mu = flat[si]
        u = uniforms(seed, idx[si] * np.uint64(1024))
        k = np.zeros(si.size, np.int64)
        p = np.exp(-mu)
        cdf = p.copy()
        active = u > cdf
        while active.any():
            k[active] += 1
            p[active] *= mu[active] / k[active]
            cdf[active] += p[active]
            active &= (u > cdf) & (k < 200)
        res[si] = k
    li = np.nonzero(~small)[0]
    mu = flat[li]
    smu = np.sqrt(mu)
    b = 0.931 + 2.53 * smu
    a = -0.059 + 0.02483 * b
    inv_alpha = 1.1239 + 1.1328 / (b - 3.4)
    vr = 0.9277 - 3.6224 / (b - 2.0)
    pending = np.ones(li.size, bool)
    attempt = 0
    while pending.any() and attempt < 500:
        pi_ = np.nonzero(pending)[0]
        base = idx[li[pi_]] * np.uint64(1024) + np.uint64(2 * attempt)
        U = uniforms(seed, base) - 0.5
        V = uniforms(seed, base + np.uint64(1))
        us = 0.5 - np.abs(U)
        k = np.floor((2.0 * a[pi_] / us + b[pi_]) * U + mu[pi_] + 0.43)
        acc = (us >= 0.07) & (V <= vr[pi_])
        ok = ~acc & (k >= 0) & ~((us < 0.013) & (V > us))
        kk = np.maximum(k, 0.0)
        lhs = np.log(V * inv_alpha[pi_] / (a[pi_] / (us * us) + b[pi_]))
        rhs = -mu[pi_] + kk * np.log(mu[pi_]) - gammaln(kk + 1.0)
        acc |= ok & (lhs <= rhs)
        done = pi_[acc]
        res[li[done]] = k[acc].astype(np.int64)
        pending[done] = False
        attempt += 1
    return out


# -------------------------------------------------------------- projections --

def phantom_for(spec: dict):
    R = spec["n_rings"] * spec["r"]
    if spec["geometry"] != CONE_3D:
        return ellipse_phantom(spec["seed"], 6, R)
    zhalf = 0.5 * spec["n_slabs"] * spec["h"]
    return ellipsoid_phantom(spec["seed"], 12, R, zhalf, blob=True)


def projections(spec: dict, noise: bool | None = None, photons: float = 1e5) -> np.ndarray:
    """Float32 projections [views][rays] of the workload's seeded phantom.
    With noise: counts ~ Poisson(photons * exp(-P)), P~ = ln(photons /
    max(counts, 1)) clamped to >= 0."""
    bodies = phantom_for(spec)
    planar = spec["geometry"] != CONE_3D
    P = np.zeros((spec["n_views"], n_rays(spec)), np.float64)
    for k in range(spec["n_views"]):
        S, D = ray_endpoints(spec, k)
        P[k] = line_integrals(bodies, S, D, planar)
    if noise is None:
        noise = bool(spec.get("noise", False))
    if noise:
        counts = poisson(spec["seed"] * 7919 + 17, photons * np.exp(-P))
        P = np.maximum(np.log(photons / np.maximum(counts, 1).astype(np.float64)), 0.0)
    return P.astype(np.float32)


def sample_phantom_on_points(bodies, x, y, z=None) -> np.ndarray:
    """Phantom value at points (for image-quality checks)."""
    pts = np.stack([x, y, np.zeros_like(x) if z is None else z], axis=-1)
    val = np.zeros(x.shape, np.float64)
    for b in bodies:
        M = (b["rot"].T / np.asarray(b["axes"], np.float64)[:, None])
        q = (pts - np.asarray(b["c"])) @ M.T
        if b["kind"] == "ellipse":
            inside = (q[..., 0] ** 2 + q[..., 1] ** 2) <= 1.0
        else:
            inside = np.einsum("...i,...i->...", q, q) <= 1.0
        val += np.where(inside, b["dens"], 0.0)
    return val
