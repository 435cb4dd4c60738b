"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: numbers the
paper prints, closed-form chord lengths, brute-force point sampling along the
ray, cell areas, closed-form MART updates, and invariants (rotation, fixed
points).  A plausible slip anywhere in the oracle (a dropped crossing family,
a wrong sector index, an inverted ratio, a transposed head table) fails one of
them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2208_12964_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def par2d(rings, views=1, bins=3, rule=oracle.SECT_6N, arc=(1, 2), custom=None, weight=oracle.LENGTH):
    d = dict(n_rings=rings, r=1.0 / rings, n_slabs=1, h=1.0, z_min=0.0, sector_rule=rule,
             geometry=oracle.PARALLEL_2D, n_views=views, arc_num=arc[0], arc_den=arc[1], n_u=bins, n_v=1,
             du=2.0 / bins, dv=1.0, weight_mode=weight)
    if custom is not None:
        d["custom_sectors"] = custom
    return d


def fan2d(rings, views, bins, du, rule=oracle.SECT_4_2N1, d_so=8.0, d_sd=16.0):
    s = synth.fan_workload(rings, views, bins, du, d_so, d_sd)
    s["sector_rule"] = rule
    return {k: v for k, v in s.items() if k in dict(oracle.Problem._fields_)}


def _fan_axis_distance(u, d_so=8.0, d_sd=16.0):
    """Distance from the rotation axis of the fan ray through detector
    offset u: the ray joins (-d_so, 0) to (d_sd - d_so, u), so by similar
    triangles its distance from the origin is d_so |u| / sqrt(d_sd^2 + u^2)."""
    return d_so * abs(u) / math.sqrt(d_sd * d_sd + u * u)


def cone3d(rings, slabs, views, det, rule=oracle.SECT_6N):
    s = synth.cone_workload(rings, slabs, views, det)
    s["sector_rule"] = rule
    return {k: v for k, v in s.items() if k in dict(oracle.Problem._fields_)}


# ------------------------------------------------------------------ grid ---

def test_grid_matches_paper_printed_counts_and_heads():
    g = json.load(open(os.path.join(GOLD, "paper_grid.json")))
    o = oracle.Oracle(par2d(g["rings"], rule=oracle.SECT_4_2N1))
    ng, head = o.grid_tables()
    assert ng.tolist() == g["sectors"]
    assert head.tolist() == g["heads"]
    N = g["total_cells_for_half_N_rings"]["N"]
    o2 = oracle.Oracle(par2d(N // 2, rule=oracle.SECT_4_2N1))
    assert o2.n_cells == g["total_cells_for_half_N_rings"]["cells"] == N * N


@pytest.mark.parametrize("N", [1, 5, 64, 128, 256])
def test_grid_6n_closed_form(N):
    o = oracle.Oracle(par2d(N))
    ng, head = o.grid_tables()
    i = np.arange(N)
    assert np.array_equal(ng, 6 * (i + 1))
    assert np.array_equal(head, 3 * i * (i + 1))
    assert o.n_cells == 3 * N * (N + 1)
    assert o.G == 6


def test_grid_custom_and_gcd():
    o = oracle.Oracle(par2d(3, rule=oracle.SECT_CUSTOM, custom=[4, 10, 14]))
    ng, head = o.grid_tables()
    assert ng.tolist() == [4, 10, 14] and head.tolist() == [0, 4, 14] and o.G == 2


# ---------------------------------------------------------- coefficients ---

def test_row_sum_is_chord_length_2d():
    """Every parallel ray's weights add up to its chord 2*sqrt(R^2 - u^2)."""
    spec = synth.workload("2d-parallel-64r-36v")
    o = oracle.Oracle({k: v for k, v in spec.items() if k in dict(oracle.Problem._fields_)})
    for k in (0, 5, 17, 35):
        for b in range(65):
            c, w = o.row(k, b)
            u = (2 * b - 64) / 65.0
            assert abs(w.sum() - 2.0 * math.sqrt(1.0 - u * u)) < 1e-12
            assert np.all(np.diff(c) > 0) and np.all(w > 0)


def test_row_sum_is_chord_length_2d_fan_table1():
    """The paper's 2-D fan scan (Table 1: source (-8,0), detector centre
    (8,0), 101 bins of 0.05, 256 x 256 grid = 128 rings of 4(2n-1) sectors):
    every ray's weights add up to its chord 2 sqrt(R^2 - d^2) through the unit
    disk, in every view; the centre bin passes through the axis and the
    outermost bins pass beside the disk."""
    spec = fan2d(128, 50, 101, 0.05)
    o = oracle.Oracle(spec)
    assert o.n_cells == 256 * 256 and o.G == 4
    for k in (0, 7, 13, 25, 49):
        for a in range(101):
            c, w = o.row(k, a)
            d = _fan_axis_distance((2 * a - 100) * 0.025)
            assert abs(w.sum() - 2.0 * math.sqrt(max(1.0 - d * d, 0.0))) < 1e-12, (k, a)
            assert np.all(np.diff(c) > 0) and np.all(w > 0)
            assert (len(c) == 0) == (d >= 1.0)  # the outer bins of the fan miss the disk


def _cylinder_chord_3d(S, D, R, z0, z1):
    """Length of segment S->D inside {x^2+y^2 <= R^2, z0 <= z <= z1}, from the
    quadratic in the segment parameter (written independently of the oracle)."""
    d = D - S
    A = d[0] ** 2 + d[1] ** 2
    B = 2 * (S[0] * d[0] + S[1] * d[1])
    Cq = S[0] ** 2 + S[1] ** 2 - R * R
    disc = B * B - 4 * A * Cq
    if disc <= 0:
        return 0.0
    lo, hi = (-B - math.sqrt(disc)) / (2 * A), (-B + math.sqrt(disc)) / (2 * A)
    za, zb = sorted(((z0 - S[2]) / d[2], (z1 - S[2]) / d[2]))
    lo, hi = max(lo, za, 0.0), min(hi, zb, 1.0)
    return max(hi - lo, 0.0) * float(np.linalg.norm(d))


def test_row_sum_is_chord_length_3d_cone():
    spec = cone3d(8, 6, 5, 16)
    o = oracle.Oracle(spec)
    rng = np.random.default_rng(0)
    for k in range(5):
        S, D = synth.ray_endpoints(spec, k)
        for ray in rng.choice(o.n_rays, 40, replace=False):
            c, w = o.row(k, ray)
            ref = _cylinder_chord_3d(S[ray], D[ray], 1.0, -1.0, 1.0)
            assert abs(w.sum() - ref) < 1e-12, (k, ray)


def _brute_force_row(spec, S, D, M=400000):
    """Per-cell length by dense midpoint sampling of the whole segment; cells
    are found from each sample's radius, height and azimuth with the grid rule
    written out here (not taken from the oracle)."""
    N, r = spec["n_rings"], spec["r"]
    rule = spec["sector_rule"]
    if rule == oracle.SECT_6N:
        ng = 6 * np.arange(1, N + 1)
    elif rule == oracle.SECT_4_2N1:
        ng = 4 * (2 * np.arange(1, N + 1) - 1)
    else:
        ng = np.asarray(spec["custom_sectors"])
    head = np.concatenate([[0], np.cumsum(ng)[:-1]])
    C = int(ng.sum())
    lam = (np.arange(M) + 0.5) / M
    P = S[None, :] + lam[:, None] * (D - S)[None, :]
    step = float(np.linalg.norm(D - S)) / M
    rho = np.hypot(P[:, 0], P[:, 1])
    inside = rho < N * r
    is3d = spec["geometry"] == oracle.CONE_3D
    if is3d:
        zz = (P[:, 2] - spec["z_min"]) / spec["h"]
        inside &= (zz >= 0) & (zz < spec["n_slabs"])
    P, rho = P[inside], rho[inside]
    ring = np.floor(rho / r).astype(np.int64)
    phi = np.mod(np.arctan2(P[:, 1], P[:, 0]), 2 * np.pi)
    sec = np.floor(phi * ng[ring] / (2 * np.pi)).astype(np.int64) % ng[ring]
    slab = np.floor((P[:, 2] - spec["z_min"]) / spec["h"]).astype(np.int64) if is3d else 0 * ring
    cell = slab * C + head[ring] + sec
    u, cnt = np.unique(cell, return_counts=True)
    return u, cnt * step, step


@pytest.mark.parametrize("case", ["6n", "4_2n1", "custom", "3d", "fan"])
def test_row_matches_brute_force_sampling(case):
    # Bin counts are chosen so that no ray passes through the axis (where
    # the sampled azimuth of points exactly on a sector boundary would depend
    # on rounding) and no ray is exactly tangent to a ring circle.  Those two
    # degenerate cases are pinned by the rotation and chord-sum tests.
    if case == "6n":
        spec = par2d(3, views=7, bins=8, arc=(1, 2))
    elif case == "4_2n1":
        spec = par2d(4, views=5, bins=8, rule=oracle.SECT_4_2N1, arc=(1, 1))
    elif case == "custom":
        spec = par2d(3, views=4, bins=6, rule=oracle.SECT_CUSTOM, custom=[3, 7, 5], arc=(1, 1))
    elif case == "fan":
        spec = fan2d(3, 5, 8, 0.5)
    else:
        spec = cone3d(3, 3, 3, 8)
    o = oracle.Oracle(spec)
    rng = np.random.default_rng(1)
    checked = 0
    for k in range(spec["n_views"]):
        S, D = synth.ray_endpoints(spec, k)
        rays = range(o.n_rays) if o.n_rays <= 16 else rng.choice(o.n_rays, 16, replace=False)
        for ray in rays:
            c, w = o.row(k, ray)
            bc, bw, step = _brute_force_row(spec, S[ray], D[ray])
            ref = dict(zip(bc.tolist(), bw.tolist()))
            got = dict(zip(c.tolist(), w.tolist()))
            for cell in set(ref) | set(got):
                a, b = got.get(cell, 0.0), ref.get(cell, 0.0)
                assert abs(a - b) <= 6 * step, (case, k, ray, cell, a, b)
                if b > 8 * step:
                    assert cell in got
                if a > 8 * step:
                    assert cell in ref
            checked += len(c)
    assert checked > 0


def test_parallel_weights_integrate_to_cell_area():
    """With many thin parallel bins, sum_b w_bj * du tends to the area of
    cell j, pi((i+1)^2 - i^2) r^2 / n_g(i); with n_g = 4(2n-1) every cell
    has the same area pi r^2 / 4 (Eq. 1 divided among the ring's cells)."""
    B = 4001
    spec = par2d(4, views=1, bins=B, rule=oracle.SECT_4_2N1)
    o = oracle.Oracle(spec)
    acc = np.zeros(o.n_cells)
    du = 2.0 / B
    for b in range(B):
        c, w = o.row(0, b)
        acc[c] += w * du
    r = 0.25
    assert np.allclose(acc, math.pi * r * r / 4.0, rtol=2e-3)


def test_rotated_rows_equal_direct_rows_2d_workload():
    spec = synth.workload("2d-parallel-64r-36v")
    o = oracle.Oracle({k: v for k, v in spec.items() if k in dict(oracle.Problem._fields_)})
    for k in range(36):
        for b in range(65):
            c, w = o.row(k, b)
            c2, w2 = o.row_rotated(k, b)
            assert np.array_equal(c, c2), (k, b)
            assert np.allclose(w2, w, rtol=1e-6, atol=0)


def test_rotated_rows_equal_direct_rows_3d_cone():
    spec = cone3d(12, 8, 18, 24)
    o = oracle.Oracle(spec)
    n, rep, sh = o.view_classes()
    assert n == 3  # 20-degree steps against 60-degree grid symmetry
    rng = np.random.default_rng(2)
    for k in range(18):
        for ray in rng.choice(o.n_rays, 30, replace=False):
            c, w = o.row(k, ray)
            c2, w2 = o.row_rotated(k, ray)
            assert np.array_equal(c, c2), (k, ray)
            assert np.allclose(w2, w, rtol=1e-6, atol=0)


def test_rotated_rows_equal_direct_rows_2d_fan():
    """Table 1 fan, 50 views over a full turn on a 4(2n-1) grid (symmetry
    order 4): 25 representatives, and every view's rows equal the rotated
    rows of its representative."""
    spec = fan2d(32, 50, 101, 0.05 * 4)
    o = oracle.Oracle(spec)
    n, rep, sh = o.view_classes()
    assert n == 25
    for k in range(50):
        for a in range(101):
            c, w = o.row(k, a)
            c2, w2 = o.row_rotated(k, a)
            assert np.array_equal(c, c2), (k, a)
            assert np.allclose(w2, w, rtol=1e-6, atol=0)


@pytest.mark.parametrize("views,arc,expect", [(36, (1, 2), 12), (90, (1, 1), 15), (180, (1, 1), 30),
                                              (6, (1, 1), 1), (12, (1, 1), 2)])
def test_view_classes_counts(views, arc, expect):
    o = oracle.Oracle(par2d(4, views=views, arc=arc))
    n, rep, sh = o.view_classes()
    assert n == expect
    # every view is its representative turned by a whole number of 1/6 turns
    for k in range(views):
        dturn = (k - rep[k]) * arc[0] / (arc[1] * views)
        assert abs(dturn * 6 - sh[k]) < 1e-12


def test_binary_weights():
    spec = par2d(5, views=3, bins=7, weight=oracle.BINARY)
    o = oracle.Oracle(spec)
    ol = oracle.Oracle(dict(spec, weight_mode=oracle.LENGTH))
    for k in range(3):
        for b in range(7):
            c, w = o.row(k, b)
            cl, wl = ol.row(k, b)
            assert np.array_equal(c, cl) and np.all(w == 1.0)


# ------------------------------------------------------------------ MART ---

def _one_cell(views=1, bins=1):
    return par2d(1, views=views, bins=bins, rule=oracle.SECT_CUSTOM, custom=[1])


def test_sequential_one_cell_closed_form():
    o = oracle.Oracle(_one_cell())
    c, w = o.row(0, 0)
    assert c.tolist() == [0] and abs(w[0] - 2.0) < 1e-15  # full diameter
    p = np.array([[0.7]], np.float32)
    f0, lam = 1.3, 0.4
    f, _ = o.mart_sequential(p, [f0], 1, lam)
    assert abs(f[0] - f0 * (float(p[0, 0]) / (2.0 * f0)) ** lam) < 1e-14
    f, _ = o.mart_sequential(p, [f0], 1, lam, rule=oracle.LINEAR_EQ18)
    assert abs(f[0] - f0 * (1.0 - lam * (1.0 - float(p[0, 0]) / (2.0 * f0)))) < 1e-14


def test_sequential_two_ring_closed_form():
    """Two off-centre rays (u = -1/4, +1/4) through two one-sector rings:
    each ray's weights are the inner chord and the outer chord minus the inner
    one; the power update uses w/max w and the rays act one after another."""
    spec = dict(par2d(2, views=1, bins=2, rule=oracle.SECT_CUSTOM, custom=[1, 1]), du=0.5)
    o = oracle.Oracle(spec)
    u, r = 0.25, 0.5
    w0 = 2 * math.sqrt(r * r - u * u)
    w1 = 2 * math.sqrt(1.0 - u * u) - w0
    for b in (0, 1):
        c, w = o.row(0, b)
        assert c.tolist() == [0, 1] and np.allclose(w, [w0, w1], rtol=1e-14)
    f = np.array([0.8, 1.7])
    p = np.array([[1.1, 0.6]], np.float32)
    wv = np.array([w0, w1])
    for b in (0, 1):
        s = float(wv @ f)
        f = f * (float(p[0, b]) / s) ** (0.3 * wv / wv.max())
    got, _ = o.mart_sequential(p, [0.8, 1.7], 1, 0.3)
    assert np.allclose(got, f, rtol=1e-14)


def test_per_view_one_cell_two_rays_closed_form():
    o = oracle.Oracle(_one_cell(views=1, bins=2))
    (c0, w0), (c1, w1) = o.row(0, 0), o.row(0, 1)
    w0, w1 = w0[0], w1[0]
    p = np.array([[0.9, 0.4]], np.float32)
    f0, lam = 1.2, 0.25
    lr = (w0 * math.log(float(p[0, 0]) / (w0 * f0)) + w1 * math.log(float(p[0, 1]) / (w1 * f0))) / (w0 + w1)
    f = o.mart_per_view(p, [f0], 1, lam)
    assert abs(f[0] - f0 * math.exp(lam * lr)) < 1e-14


def test_per_view_zero_projection_zeroes_cells_and_skips_empty():
    spec = par2d(3, views=2, bins=5)
    o = oracle.Oracle(spec)
    p = np.ones((2, 5), np.float32)
    p[0, 2] = 0.0
    f = o.mart_per_view(p, np.ones(o.n_cells), 1, 0.5, order=[0, 1])
    c, _ = o.row(0, 2)
    assert np.all(f[c] == 0.0)
    assert np.all(np.isfinite(f)) and np.all(f >= 0)


def test_per_view_linear_eq18_one_cell_closed_form():
    """Per-view form of Eq. 18 on one cell met by three rays of one view
    (u = -2/3, 0, 2/3: chords 2 sqrt(5)/3, 2, 2 sqrt(5)/3): the cell's factor
    is the weighted arithmetic mean of the rays' factors 1 - beta (1 - P/Pbar),
    weights the rays' chords.  A ray with P = 0 contributes 1 - beta (it does
    not zero the cell, unlike the power form); the power form's geometric mean
    is checked on the same rays."""
    o = oracle.Oracle(_one_cell(views=1, bins=3))
    w = np.array([2 * math.sqrt(5) / 3, 2.0, 2 * math.sqrt(5) / 3])
    for b in range(3):
        assert abs(o.row(0, b)[1][0] - w[b]) < 1e-14
    f0, beta = 1.2, 0.35
    for pv in ((0.9, 0.4, 1.3), (0.0, 0.7, 1.1)):
        p = np.array([pv], np.float32)
        q = p[0].astype(np.float64)
        fac = 1.0 - beta * (1.0 - q / (w * f0))
        want = f0 * float(np.sum(w * fac) / np.sum(w))
        got = o.mart_per_view(p, [f0], 1, beta, rule=oracle.LINEAR_EQ18)
        assert abs(got[0] - want) < 1e-14
    p = np.array([[0.9, 0.4, 1.3]], np.float32)
    q = p[0].astype(np.float64)
    want = f0 * math.exp(beta * float(np.sum(w * np.log(q / (w * f0))) / np.sum(w)))
    assert abs(o.mart_per_view(p, [f0], 1, beta)[0] - want) < 1e-14


def test_per_view_two_ring_closed_form_both_rules():
    """Two one-sector rings, two off-centre rays (u = -1/4, +1/4) of one view:
    both rays cross both cells with weights (inner chord, outer chord minus
    inner); each cell is corrected once from both rays' ratios, by the
    geometric (POWER) or arithmetic (Eq. 18) weighted mean."""
    spec = dict(par2d(2, views=1, bins=2, rule=oracle.SECT_CUSTOM, custom=[1, 1]), du=0.5)
    o = oracle.Oracle(spec)
    u, r = 0.25, 0.5
    w_in = 2 * math.sqrt(r * r - u * u)
    w_out = 2 * math.sqrt(1.0 - u * u) - w_in
    wv = np.array([w_in, w_out])
    f0 = np.array([0.8, 1.7])
    p = np.array([[1.1, 0.6]], np.float32)
    s = np.array([wv @ f0, wv @ f0])  # both rays have the same weights
    ratio = np.array([float(p[0, 0]), float(p[0, 1])]) / s
    lam = 0.3
    # every cell sees both rays with its own weight, so its weights cancel in the mean
    geo = f0 * np.exp(lam * np.mean(np.log(ratio)))
    lin = f0 * np.mean(1.0 - lam * (1.0 - ratio))
    assert np.allclose(o.mart_per_view(p, f0, 1, lam), geo, rtol=1e-14)
    assert np.allclose(o.mart_per_view(p, f0, 1, lam, rule=oracle.LINEAR_EQ18), lin, rtol=1e-14)


def test_per_view_eq19_stopping_and_linear_fixed_point():
    """Eq. 19 in the per-view schedule: consistent data p = A f* leaves f*
    in place (ratio 1: both rules give factor 1), so the first sweep meets a
    tolerance of 1e-3 and the run stops after it; from f = 1 a tolerance of
    1e-9 is never met and every sweep runs."""
    spec = par2d(3, views=4, bins=7)
    o = oracle.Oracle(spec)
    rng = np.random.default_rng(5)
    fstar = 0.5 + rng.random(o.n_cells)
    p = np.stack([o.forward(k, fstar) for k in range(4)]).astype(np.float32)
    for rule in (oracle.POWER, oracle.LINEAR_EQ18):
        f, n = o.mart_per_view(p, fstar, 50, 0.5, rule=rule, tol=1e-3, return_sweeps=True)
        assert n == 1 and np.max(np.abs(f / fstar - 1)) < 1e-6
        _, n = o.mart_per_view(p, np.ones(o.n_cells), 7, 0.5, rule=rule, tol=1e-9, return_sweeps=True)
        assert n == 7
        _, n = o.mart_per_view(p, np.ones(o.n_cells), 7, 0.5, rule=rule, return_sweeps=True)
        assert n == 7


def test_per_view_linear_reduces_misfit():
    spec = par2d(6, views=12, bins=13, arc=(1, 2))
    o = oracle.Oracle(spec)
    fstar = 0.2 + np.random.default_rng(4).random(o.n_cells)
    p = np.stack([o.forward(k, fstar) for k in range(12)]).astype(np.float32)

    def misfit(f):
        return sum(np.sum((o.forward(k, f) - p[k]) ** 2) for k in range(12))

    f0 = np.ones(o.n_cells)
    f1 = o.mart_per_view(p, f0, 2, 0.5, rule=oracle.LINEAR_EQ18)
    f2 = o.mart_per_view(p, f0, 10, 0.5, rule=oracle.LINEAR_EQ18)
    assert misfit(f2) < misfit(f1) < misfit(f0)
    assert np.all(f2 > 0)


def test_fixed_point_of_consistent_data():
    """p = A f* (rounded to float32) leaves f* unchanged up to that rounding."""
    spec = par2d(6, views=8, bins=13, arc=(1, 2))
    o = oracle.Oracle(spec)
    rng = np.random.default_rng(3)
    fstar = 0.5 + rng.random(o.n_cells)
    p = np.stack([o.forward(k, fstar) for k in range(8)]).astype(np.float32)
    f, _ = o.mart_sequential(p, fstar, 1, 0.5)
    assert np.max(np.abs(f / fstar - 1)) < 1e-6
    f2 = o.mart_per_view(p, fstar, 1, 0.5)
    assert np.max(np.abs(f2 / fstar - 1)) < 1e-6


def test_mart_reduces_data_misfit_on_consistent_data():
    spec = par2d(6, views=12, bins=13, arc=(1, 2))
    o = oracle.Oracle(spec)
    rng = np.random.default_rng(4)
    fstar = 0.2 + rng.random(o.n_cells)
    p = np.stack([o.forward(k, fstar) for k in range(12)]).astype(np.float32)

    def misfit(f):
        return sum(np.sum((o.forward(k, f) - p[k]) ** 2) for k in range(12))

    f0 = np.ones(o.n_cells)
    m0 = misfit(f0)
    f1 = o.mart_per_view(p, f0, 2, 0.5)
    f2 = o.mart_per_view(p, f0, 10, 0.5)
    assert misfit(f2) < misfit(f1) < m0
    g1, _ = o.mart_sequential(p, f0, 2, 0.5)
    g2, _ = o.mart_sequential(p, f0, 10, 0.5)
    assert misfit(g2) < misfit(g1) < m0
    assert np.all(f2 > 0) and np.all(g2 > 0)


def test_eq19_stopping():
    spec = par2d(3, views=4, bins=7)
    o = oracle.Oracle(spec)
    rng = np.random.default_rng(5)
    fstar = 0.5 + rng.random(o.n_cells)
    p = np.stack([o.forward(k, fstar) for k in range(4)]).astype(np.float32)
    _, n = o.mart_sequential(p, fstar, 50, 0.5, tol=1e-3)
    assert n == 1
    _, n = o.mart_sequential(p, np.ones(o.n_cells), 50, 0.5, tol=1e-9)
    assert n > 1


# -------------------------------------------------------------- resample ---

def test_resample_constant_and_cell_containment():
    spec = par2d(5)
    o = oracle.Oracle(spec)
    out = o.resample_point(np.full(o.n_cells, 3.0), 40, 40)[0]
    x = -1 + (np.arange(40) + 0.5) / 20
    X, Y = np.meshgrid(x, x)
    inside = np.hypot(X, Y) < 1
    assert np.all(out[inside] == 3.0) and np.all(out[~inside] == 0.0)
    ids = o.resample_point(np.arange(o.n_cells, dtype=np.float64), 40, 40)[0]
    ng, head = o.grid_tables()
    for yy, xx, cid in zip(Y[inside], X[inside], ids[inside]):
        ring = int(np.searchsorted(head, cid, side="right") - 1)
        sec = int(cid - head[ring])
        assert ring == int(math.floor(math.hypot(xx, yy) / 0.2))
        a = math.atan2(yy, xx) % (2 * math.pi)
        lo, hi = 2 * math.pi * sec / ng[ring], 2 * math.pi * (sec + 1) / ng[ring]
        assert lo - 1e-9 <= a < hi + 1e-9


def test_resample_bijection_is_ring_preserving_permutation():
    N = 6
    spec = par2d(N, rule=oracle.SECT_4_2N1)
    o = oracle.Oracle(spec)
    ids = o.resample_bijection(np.arange(o.n_cells, dtype=np.float64))[0]
    assert sorted(ids.reshape(-1).astype(int).tolist()) == list(range(o.n_cells))
    ng, head = o.grid_tables()
    c = np.arange(2 * N) - N + 0.5
    X, Y = np.meshgrid(c, c)
    sq = np.maximum(np.abs(X), np.abs(Y)) + 0.5
    ring = np.searchsorted(head, ids, side="right") - 1
    assert np.array_equal(ring + 1, sq.astype(int))
    with pytest.raises(ValueError):
        oracle.Oracle(par2d(3)).resample_bijection(np.zeros(36))


def test_resample_bijection_order_hand_listed():
    """The pixel order of the one-to-one map for N = 1, 2, 3 against lists
    written by hand from the reading of Sec. II.A-B (both rings numbered
    counter-clockwise from +x; tests/golden/bijection_order.json): a
    clockwise walk, or one starting a pixel off, fails here."""
    gold = json.load(open(os.path.join(GOLD, "bijection_order.json")))["lists"]
    for N_s, rings in gold.items():
        N = int(N_s)
        o = oracle.Oracle(par2d(N, rule=oracle.SECT_4_2N1))
        ng, head = o.grid_tables()
        ids = o.resample_bijection(np.arange(o.n_cells, dtype=np.float64))[0]
        assert len(rings) == N
        for n, pix in enumerate(rings, start=1):
            assert len(pix) == ng[n - 1] == 8 * n - 4
            for j, (a, b) in enumerate(pix):
                assert ids[b, a] == head[n - 1] + j, (N, n, j)


@pytest.mark.parametrize("N", [4, 7, 16])
def test_resample_bijection_azimuth_order(N):
    """Within every square ring the cell index H_n + j grows with the
    pixel-centre azimuth measured counter-clockwise from +x in [0, 2 pi), and
    j = 0 is the pixel with the smallest azimuth (the first at or above +x)."""
    o = oracle.Oracle(par2d(N, rule=oracle.SECT_4_2N1))
    ng, head = o.grid_tables()
    ids = o.resample_bijection(np.arange(o.n_cells, dtype=np.float64))[0].astype(np.int64)
    c = np.arange(2 * N) - N + 0.5
    X, Y = np.meshgrid(c, c)  # X[b, a] = a - N + 1/2, Y[b, a] = b - N + 1/2
    az = np.mod(np.arctan2(Y, X), 2 * math.pi)
    for n in range(1, N + 1):
        sel = (ids >= head[n - 1]) & (ids < head[n - 1] + ng[n - 1])
        j = ids[sel] - head[n - 1]
        order = np.argsort(j)
        a_sorted = az[sel][order]
        assert np.all(np.diff(a_sorted) > 0), n
        assert j[np.argmin(az[sel])] == 0


# ----------------------------------------------------------------- inputs ---

def test_synth_disk_projection_closed_form():
    disk = [dict(kind="ellipse", dens=1.0, c=(0.0, 0.0, 0.0), axes=(0.6, 0.6, 1.0), rot=np.eye(3))]
    spec = par2d(8, views=3, bins=31, arc=(1, 2))
    for k in range(3):
        S, D = synth.ray_endpoints(spec, k)
        P = synth.line_integrals(disk, S, D, planar=True)
        u = (2 * np.arange(31) - 30) / 31.0
        ref = 2 * np.sqrt(np.maximum(0.36 - u * u, 0))
        assert np.allclose(P, ref, atol=1e-12)


def test_synth_fan_disk_projection_closed_form():
    disk = [dict(kind="ellipse", dens=1.0, c=(0.0, 0.0, 0.0), axes=(0.6, 0.6, 1.0), rot=np.eye(3))]
    spec = synth.fan_workload(8, 5)
    for k in range(5):
        S, D = synth.ray_endpoints(spec, k)
        P = synth.line_integrals(disk, S, D, planar=True)
        d = np.array([_fan_axis_distance((2 * a - 100) * 0.025) for a in range(101)])
        ref = 2 * np.sqrt(np.maximum(0.36 - d * d, 0))
        assert np.allclose(P, ref, atol=1e-12)


def test_synth_poisson_moments_and_determinism():
    mean = np.concatenate([np.full(20000, 3.0), np.full(20000, 2500.0)])
    a = synth.poisson(11, mean)
    b = synth.poisson(11, mean)
    assert np.array_equal(a, b)
    lo, hi = a[:20000], a[20000:]
    assert abs(lo.mean() - 3.0) < 0.05 and abs(lo.var() - 3.0) < 0.15
    assert abs(hi.mean() - 2500.0) < 1.5 and abs(hi.var() / 2500.0 - 1) < 0.05


# ------------------------------------------- view-0 segment store (binary) ---

def _binary(spec, store_form=oracle.STORE_ROWS):
    d = {k: v for k, v in spec.items() if k in dict(oracle.Problem._fields_)}
    d["weight_mode"] = oracle.BINARY
    d["store_form"] = store_form
    return oracle.Oracle(d)


@pytest.mark.parametrize("case", ["parallel64", "fan128", "cone12_6n", "cone12_4n"])
def test_segment_store_rows_equal_direct_binary_rows(case):
    """Algorithm 1: the first view's segments (cylinder and axial-plane
    crossings, ring, slice, end azimuths), turned by each view's source angle
    and re-binned to sectors, give every view's binary row exactly as the
    direct trace of that view does -- including the centre rays through the
    axis and the crossings that lie on a sector boundary."""
    if case == "parallel64":
        spec = synth.workload("2d-parallel-64r-36v")
    elif case == "fan128":
        spec = synth.workload("2d-fan-128r-50v-101")
    else:
        spec = synth.cone_workload(12, 8, 18, 24, noise=False)
        spec["sector_rule"] = oracle.SECT_6N if case == "cone12_6n" else oracle.SECT_4_2N1
    o = _binary(spec)
    for k in range(spec["n_views"]):
        for ray in range(o.n_rays):
            c, w = o.row(k, ray)
            c2, w2 = o.rebin_row(k, ray)
            assert np.array_equal(c, c2), (case, k, ray)
            assert np.all(w2 == 1.0)


def test_segment_lengths_sum_to_chord_and_counts():
    """The segments of a first-view ray tile its chord (closed form), each
    lies in one ring; a ray has at most 2N + slabs + 1 segments."""
    spec = synth.workload("2d-fan-128r-50v-101")
    o = _binary(spec)
    for a in range(101):
        rg, sb, fa, fb, ln, dr = o.segments(a)
        d = _fan_axis_distance((2 * a - 100) * 0.025)
        assert abs(ln.sum() - 2.0 * math.sqrt(max(1.0 - d * d, 0.0))) < 1e-12
        assert len(rg) <= 2 * 128 + 1 + 1
        if len(rg):  # the centre bin passes through the axis; the outermost bins miss the disk
            assert dr == (0 if a == 50 else (1 if a < 50 else -1))
    spec3 = cone3d(8, 6, 5, 16)
    o3 = _binary(spec3)
    S, D = synth.ray_endpoints(spec3, 0)
    for ray in range(0, o3.n_rays, 7):
        rg, sb, fa, fb, ln, dr = o3.segments(ray)
        assert abs(ln.sum() - _cylinder_chord_3d(S[ray], D[ray], 1.0, -1.0, 1.0)) < 1e-12
        assert len(rg) <= 2 * 8 + 6 + 1


def test_view_turns_are_exact_fixed_point():
    o = _binary(synth.workload("2d-fan-128r-50v-101"))
    for k in range(50):
        assert o.view_turns(k) == (k * (1 << 64)) // 50
    o2 = _binary(synth.workload("2d-parallel-64r-36v"))
    for k in range(36):
        assert o2.view_turns(k) == (k * (1 << 64)) // 72  # half a turn over 36 views


def test_segment_store_mart_equals_direct_binary_mart():
    """Sequential MART (Eq. 18) over the re-binned rows equals MART over the
    directly traced binary rows (same rows, same order)."""
    spec = synth.fan_workload(32, 12, 41, 0.1)
    proj = synth.projections(spec)
    o = _binary(spec)
    os_ = _binary(spec, oracle.STORE_SEGMENTS)
    f0 = np.ones(o.n_cells)
    a, _ = o.mart_sequential(proj, f0, 3, 0.4, rule=oracle.LINEAR_EQ18)
    b, _ = os_.mart_sequential(proj, f0, 3, 0.4, rule=oracle.LINEAR_EQ18)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("case", ["fan", "cone"])
def test_quarter_symmetry_of_first_view_lines(case):
    """Sec. III.C: reflections of the first view's lines in the transverse
    plane (u -> -u, y -> -y) and, for a centred cone scan, in the axial
    mid-plane (v -> -v, z -> -z) give the other lines' crossings, so a quarter
    of the lines determine all.  The mirror line has the same segments (ring,
    length) with negated azimuths and reversed turn, or with mirrored slabs."""
    if case == "fan":
        spec = fan2d(16, 1, 41, 0.05)
    else:
        spec = cone3d(8, 6, 1, 16)
    o = _binary(spec)
    n_u, n_v = spec["n_u"], spec["n_v"]
    n_s = spec["n_slabs"] if case == "cone" else 1
    window = 1 << 24  # fixed-turn units: rounding of the two atan2 evaluations stays far inside
    for ray in range(o.n_rays):
        a, c = ray % n_u, ray // n_u
        rg, sb, fa, fb, ln, dr = o.segments(ray)
        mu = c * n_u + (n_u - 1 - a)  # transverse mirror
        rg2, sb2, fa2, fb2, ln2, dr2 = o.segments(mu)
        assert np.array_equal(rg, rg2) and np.array_equal(sb, sb2) and dr2 == -dr
        assert np.allclose(ln, ln2, rtol=1e-12, atol=1e-15)
        for x, y in ((fa, fa2), (fb, fb2)):
            s = (x.astype(object) + y.astype(object)) % (1 << 64)  # -F mod 2^64 plus F
            assert all(min(int(v), (1 << 64) - int(v)) < window for v in s)
        if case == "cone":
            mv = (n_v - 1 - c) * n_u + a  # axial mirror
            rg3, sb3, fa3, fb3, ln3, dr3 = o.segments(mv)
            assert np.array_equal(rg, rg3) and np.array_equal(sb, n_s - 1 - sb3) and dr3 == dr
            assert np.allclose(ln, ln3, rtol=1e-12, atol=1e-15)
            assert all(min(int((x - y) % (1 << 64)), int((y - x) % (1 << 64))) < window
                       for x, y in zip(fa.tolist(), fa3.tolist()))


def _mirror_rows_agree(spec, column_mirror):
    """Rows of every representative rebuilt from its partner's under the
    reflection y -> -y (Sec. III.C quarter symmetry): view theta -> view
    -theta, sector j -> -1-j, then a whole number of 1/G turns up to the
    partner's own angle; fan and cone rays swap column a <-> n_u-1-a.
    Returns (rows compared, rows whose lists differ)."""
    o = oracle.Oracle(spec)
    ng, head = o.grid_tables()
    G, V = o.G, spec["n_views"]
    den = spec["arc_den"] * V
    n_reps, rep_of_view, _ = o.view_classes()
    reps = [int(np.flatnonzero(rep_of_view == q)[0]) for q in range(n_reps)]
    key = {k: (k * spec["arc_num"] * G) % den for k in reps}
    m = {k: (k * spec["arc_num"] * G) // den for k in reps}
    view_of_key = {key[k]: k for k in reps}
    n_u = spec["n_u"]
    ring_of = np.repeat(np.arange(len(ng)), ng)
    compared = differ = 0
    for k in reps:
        k2 = view_of_key.get((den - key[k]) % den)
        if k2 is None:
            continue
        M = (m[k] + m[k2] + (1 if key[k] else 0)) % G
        for ray in range(o.n_rays):
            src = ray - ray % n_u + (n_u - 1 - ray % n_u) if column_mirror else ray
            c, w = o.row(k, src)
            slab, within = c // o.cells_per_slab, c % o.cells_per_slab
            ring = ring_of[within]
            sec = (M * (ng[ring] // G) - 1 - (within - head[ring])) % ng[ring]
            mc = slab * o.cells_per_slab + head[ring] + sec
            order = np.argsort(mc)
            c2, w2 = o.row(k2, ray)
            compared += 1
            if not np.array_equal(mc[order], c2):
                differ += 1
            else:
                assert np.allclose(w[order], w2, rtol=1e-8, atol=1e-14)  # independently rounded crossings
    return compared, differ


@pytest.mark.parametrize("case", ["parallel", "fan", "cone"])
def test_partner_representatives_are_mirror_images(case):
    """Sec. III.C: the lines of the view at -theta are the reflections of the
    lines at theta, so representatives pair up as (rho, 1/G - rho) and only
    one of each pair needs tracing.  Directly traced rows equal the
    reflected, rotated rows of the partner (same lengths), on every row of
    every pair -- a parallel scan (bins unchanged), Table 1's fan and a cone
    (columns mirrored); the scans avoid rays through the axis."""
    if case == "parallel":
        spec = par2d(12, views=36, bins=26)
        col = False
    elif case == "fan":
        spec = fan2d(24, 20, 40, 0.05)
        col = True
    else:
        spec = cone3d(8, 6, 18, 16)
        col = True
    compared, differ = _mirror_rows_agree(spec, col)
    assert compared > 0 and differ == 0, (compared, differ)
