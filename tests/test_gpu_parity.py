"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Bars: cell index lists bit-exact; stored FP32 weights within 1e-6 relative;
MART images within 1e-4 relative L2 of the FP64 oracle after the stated
iterations; resampled images exact (the resample is a gather of FP32 image
values, the cell choice is an integer decision taken in FP64 on both sides).
"""
import numpy as np
import pytest

import oracle
from gpu_util import Gpu, assert_rows_equal, oracle_for, rel_l2
from paper_2208_12964_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_W = 1e-6
TOL_IMG = 1e-4


# -------------------------------------------------------------- generator ---

def test_rows_2d_parallel_all_views_all_rays(torch_cuda):
    from paper_2208_12964_gb300 import uspg

    spec = synth.workload("2d-parallel-64r-36v")
    assert Gpu(spec).build().stats()["walked_rows"] == 12 * 65  # AUTO: a store this small is walked whole
    spec["symmetry"] = uspg.SYMMETRY_ALWAYS  # every derived row below is checked
    g = Gpu(spec).build()
    o = oracle_for(spec)
    st = g.stats()
    assert st["n_reps"] == 12 and st["n_cells"] == 12480 and st["gcd"] == 6
    # representatives at 5..25 degrees are walked, 35..55 are their mirror
    # images; 0 and 30 degrees are their own (a parallel ray is its own mirror)
    assert 7 * 65 <= st["walked_rows"] < 12 * 65, st["walked_rows"]
    total = 0
    for k in range(36):
        for b in range(65):
            gc, gw = g.row(k, b)
            oc, ow = o.row(k, b)
            assert_rows_equal(gc, gw, oc, ow, TOL_W, where=f"view {k} ray {b}")
            total += len(oc)
    assert total == st["nnz_all_views"]


def test_rows_2d_fan_table1_all_views_all_rays(torch_cuda):
    """The paper's 2-D fan scan (Table 1): 128 rings of 4(2n-1) sectors,
    50 views over a full turn, 101 bins of 0.05, source (-8,0), detector
    (8,0); every row of every view against the oracle's direct trace."""
    from paper_2208_12964_gb300 import uspg

    spec = dict(synth.workload("2d-fan-128r-50v-101"), symmetry=uspg.SYMMETRY_ALWAYS)
    g = Gpu(spec).build()
    o = oracle_for(spec)
    st = g.stats()
    assert st["n_reps"] == 25 and st["n_cells"] == 65536 and st["gcd"] == 4 and not st["mirrored"]
    assert st["walked_rows"] < 25 * 101  # mirror-image representatives derived
    total = 0
    for k in range(50):
        for a in range(101):
            gc, gw = g.row(k, a)
            oc, ow = o.row(k, a)
            assert_rows_equal(gc, gw, oc, ow, TOL_W, where=f"view {k} bin {a}")
            total += len(oc)
    assert total == st["nnz_all_views"]


@pytest.mark.parametrize("case", ["6n", "4_2n1", "custom"])
def test_rows_3d_cone_small_all_rays(torch_cuda, case):
    from paper_2208_12964_gb300 import uspg

    spec = dict(synth.cone_workload(12, 8, 18, 24, noise=False), symmetry=uspg.SYMMETRY_ALWAYS)
    if case == "4_2n1":
        spec["sector_rule"] = synth.SECT_4_2N1
    elif case == "custom":
        spec["sector_rule"] = synth.SECT_CUSTOM
        spec["custom_sectors"] = [5, 9, 12, 14, 20, 22, 27, 30, 33, 40, 41, 48]
    g = Gpu(spec).build()
    o = oracle_for(spec)
    for k in range(18):
        for ray in range(24 * 24):
            gc, gw = g.row(k, ray)
            oc, ow = o.row(k, ray)
            assert_rows_equal(gc, gw, oc, ow, TOL_W, where=f"{case} view {k} ray {ray}")


@pytest.mark.parametrize("case", ["mirror_odd", "no_mirror"])
def test_z_mirror_store(torch_cuda, case):
    """Centred cone scans store only the lower detector rows and the lower
    and middle slabs of the cell-major store (z-mirror, Sec. III.C symmetry).
    mirror_odd: odd detector rows and odd slab count, so a detector row and a
    slab are their own mirrors; no_mirror: an off-centre slab stack, every
    row stored.  Every row of every view is compared with the oracle's direct
    trace, the store size with the oracle's counts, and both MART schedules
    with the oracle."""
    from paper_2208_12964_gb300 import uspg

    if case == "mirror_odd":
        spec = synth.cone_workload(10, 9, 12, 21, iterations=2, lam=0.2, seed=13, noise=False)
    else:
        spec = synth.cone_workload(10, 8, 12, 20, iterations=2, lam=0.2, seed=14, noise=False)
        spec["z_min"] = -0.75  # stack [-0.75, 1.25]: not symmetric about the source plane
    spec["symmetry"] = uspg.SYMMETRY_ALWAYS  # transverse mirror on every row checked below
    g = Gpu(spec).build()
    o = oracle_for(spec)
    n_u = n_v = spec["n_u"]
    st = g.stats()
    total = 0
    for k in range(spec["n_views"]):
        for ray in range(n_u * n_v):
            gc, gw = g.row(k, ray)
            oc, ow = o.row(k, ray)
            assert_rows_equal(gc, gw, oc, ow, TOL_W, where=f"{case} view {k} ray {ray}")
            total += len(oc)
    assert total == st["nnz_all_views"]
    _, rep, _ = o.view_classes()
    rep_views = [int(np.flatnonzero(rep == q)[0]) for q in range(int(rep.max()) + 1)]
    full = sum(o.view_nnz(k) for k in rep_views)
    if case == "mirror_odd":
        mid = (n_v - 1) // 2
        self_mirror = sum(len(o.row(k, mid * n_u + u)[0]) for k in rep_views for u in range(n_u))
        assert st["nnz_store"] == (full + self_mirror) // 2
    else:
        assert st["nnz_store"] == full
    proj = synth.projections(spec)
    f0 = np.ones(o.n_cells)
    ref = o.mart_per_view(proj, f0, 2, 0.2)
    assert rel_l2(_run_mart(g, proj, f0, 2, 0.2, 1), ref) < TOL_IMG
    ref, _ = o.mart_sequential(proj, f0, 1, 0.2)
    assert rel_l2(_run_mart(g, proj, f0, 1, 0.2, 0), ref) < TOL_IMG


@pytest.mark.parametrize("name", ["cone_mirror", "cone_16", "fan"])
def test_derived_columns_equal_built_columns(torch_cuda, name):
    """A representative whose rows are all mirror images of its source's
    (transverse symmetry, Sec. III.C) gets its cell-major columns from the
    source's finished columns, with each ray replaced by its mirror column.
    Built with the symmetry (rows and columns derived) and without it (every
    row walked, every column built from its rows), two per-view MART
    iterations from the same start agree to the FP32 rounding of the ray
    sums, and both agree with the oracle.  (A representative with a row
    whose walk went the other way at a tie builds its own columns.)"""
    from paper_2208_12964_gb300 import uspg

    if name == "cone_mirror":
        spec = synth.cone_workload(12, 8, 18, 24, iterations=2, lam=0.2, seed=21, noise=False)
    elif name == "cone_16":
        spec = synth.cone_workload(16, 16, 30, 32, iterations=2, lam=0.2, seed=22, noise=False)
    else:  # an even bin count: no ray through the axis, whose tie rule breaks the mirror
        spec = synth.fan_workload(64, 40, bins=100)
    imgs, stats = {}, {}
    proj = synth.projections(spec)
    for mode in (uspg.SYMMETRY_ALWAYS, uspg.SYMMETRY_NEVER):
        g = Gpu(dict(spec, symmetry=mode)).build()
        try:
            stats[mode] = g.stats()
            f0 = np.ones(stats[mode]["n_cells"])
            imgs[mode] = _run_mart(g, proj, f0, 2, 0.2, 1)
        finally:
            g.close()
    assert stats[uspg.SYMMETRY_ALWAYS]["derived_reps"] > 0
    assert stats[uspg.SYMMETRY_NEVER]["derived_reps"] == 0
    assert stats[uspg.SYMMETRY_NEVER]["walked_rows"] > stats[uspg.SYMMETRY_ALWAYS]["walked_rows"]
    a, b = imgs[uspg.SYMMETRY_ALWAYS], imgs[uspg.SYMMETRY_NEVER]
    assert np.array_equal(a == 0.0, b == 0.0)
    assert rel_l2(a, b) < 1e-6 and np.max(np.abs(a - b)) <= 1e-5 * np.max(np.abs(b))
    o = oracle_for(spec)
    ref = o.mart_per_view(proj, np.ones(o.n_cells), 2, 0.2)
    assert rel_l2(a, ref) < TOL_IMG


def test_rows_3d_cone_full_size_sampled(torch_cuda):
    """The 128-ring, 128-slab, 90-view, 256x256 workload: 400 sampled rows
    (oracle traces each one directly)."""
    spec = synth.workload("3d-cone-128r-128s-90v-256")
    g = Gpu(spec).build()
    o = oracle_for(spec)
    st = g.stats()
    assert st["n_reps"] == 15 and st["n_cells"] == 6340608
    # transverse symmetry: representatives 1..7 are walked, 8..14 are their
    # mirror images, representative 0 walks columns 0..127 (rows with a tied
    # piece are walked after all)
    base = 7 * 32768 + 128 * 128
    assert base <= st["walked_rows"] <= base + 0.01 * 15 * 32768, st["walked_rows"]
    rng = np.random.default_rng(7)
    for _ in range(400):
        k = int(rng.integers(90))
        ray = int(rng.integers(256 * 256))
        gc, gw = g.row(k, ray)
        oc, ow = o.row(k, ray)
        assert_rows_equal(gc, gw, oc, ow, TOL_W, where=f"view {k} ray {ray}")


def test_cone256_full_size(torch_cuda):
    """The 256-ring, 256-slab, 180-view cone with a 512x512 detector, built as
    bench.py builds it.  FP16 store: 200 sampled rows against the oracle's
    direct trace (index lists exact; each weight the FP64 length rounded once
    to FP16 in units of the cell size).  FP32 store: one per-view step of
    view 0 from f0 = 1 over all 50.5 M cells against the oracle's step."""
    from paper_2208_12964_gb300 import uspg

    spec = synth.workload("3d-cone-256r-256s-180v-512")
    o = oracle_for(spec)
    o.set_threads(16)
    g = Gpu(spec, dtype=uspg.F16).build()
    st = g.stats()
    assert st["n_reps"] == 30 and st["n_cells"] == 50528256 and st["mirrored"] == 1
    unit = min(spec["r"], spec["h"])
    rng = np.random.default_rng(11)
    for _ in range(200):
        k, ray = int(rng.integers(180)), int(rng.integers(512 * 512))
        gc, gw = g.row(k, ray)
        oc, ow = o.row(k, ray)
        assert np.array_equal(gc, oc), f"view {k} ray {ray}"
        big = ow > 1e-4 * unit
        if big.any():
            assert np.max(np.abs(gw[big] - ow[big]) / ow[big]) <= 2 ** -10
    g.close()
    # view 0's projections (noise-free line integrals); no other view is used
    S, D = synth.ray_endpoints(spec, 0)
    proj = np.zeros((180, 512 * 512), np.float32)
    proj[0] = synth.line_integrals(synth.phantom_for(spec), S, D, planar=False)
    g = Gpu(spec).build()
    U = g.U
    U.uspg_set_projections(g.ctx, proj, False)
    U.uspg_fill_image(g.ctx, 1.0)
    U.uspg_autotune(g.ctx)
    opts, keep = U.mart_opts(1, 0.1, U.PER_VIEW, view_steps=1)
    U.uspg_mart(g.ctx, opts)
    U.uspg_sync(g.ctx)
    got = np.zeros(o.n_cells, np.float32)
    U.uspg_get_image(g.ctx, got, False)
    g.close()
    ref = np.ones(o.n_cells)
    o.mart_views_sample(proj, ref, [0], 0.1)
    hit = ref != 1.0
    assert hit.sum() > 0.5 * o.n_cells
    assert np.all(got[~hit] == 1.0)
    nz = ref > 0
    assert np.all(got[~nz] == 0.0)
    assert np.max(np.abs(got[nz] - ref[nz]) / ref[nz]) < 2e-5


def test_binary_weights(torch_cuda):
    from paper_2208_12964_gb300 import uspg

    spec = synth.parallel_workload(9, 10, 19)
    g = Gpu(spec, weight_mode=uspg.BINARY).build()
    o = oracle_for(spec, weight_mode=1)
    for k in range(10):
        for b in range(19):
            gc, gw = g.row(k, b)
            oc, ow = o.row(k, b)
            assert np.array_equal(gc, oc) and np.all(gw == 1.0)


# ---------------------------------------------------------------- forward ---

def test_forward_projection_matches_oracle(torch_cuda):
    torch = torch_cuda
    spec = synth.cone_workload(10, 6, 12, 20, noise=False)
    g = Gpu(spec).build()
    o = oracle_for(spec)
    rng = np.random.default_rng(3)
    f = (0.2 + rng.random(o.n_cells)).astype(np.float32)
    g.U.uspg_set_image(g.ctx, f, False)
    out = torch.zeros(o.n_rays, dtype=torch.float32, device="cuda")
    for k in range(12):
        g.U.uspg_forward_project(g.ctx, k, out)
        g.U.uspg_sync(g.ctx)
        ref = o.forward(k, f.astype(np.float64))
        got = out.cpu().numpy().astype(np.float64)
        hit = ref > 0
        assert np.all(got[~hit] == 0.0)
        assert np.max(np.abs(got[hit] - ref[hit]) / ref[hit]) < 2e-6


# ------------------------------------------------------------------- MART ---

def _run_mart(g, proj, f0, iters, lam, schedule, rule=0, order=None, tol=0.0):
    U = g.U
    U.uspg_set_projections(g.ctx, np.ascontiguousarray(proj, np.float32), False)
    U.uspg_set_image(g.ctx, np.ascontiguousarray(f0, np.float32), False)
    o, keep = U.mart_opts(iters, lam, schedule, rule, tol, order)
    U.uspg_mart(g.ctx, o)
    U.uspg_sync(g.ctx)
    f = np.zeros(len(f0), np.float32)
    U.uspg_get_image(g.ctx, f, False)
    return f


def test_mart_sequential_2d_workload(torch_cuda):
    """The 64-ring, 36-view parallel workload, 10 ray-sequential iterations,
    lambda 0.2, f0 = 1 (the paper's ray order)."""
    spec = synth.workload("2d-parallel-64r-36v")
    proj = synth.projections(spec)
    g = Gpu(spec).build()
    o = oracle_for(spec)
    f0 = np.ones(o.n_cells)
    ref, _ = o.mart_sequential(proj, f0, 10, 0.2)
    got = _run_mart(g, proj, f0, 10, 0.2, 0)
    assert rel_l2(got, ref) < TOL_IMG
    assert np.all(got >= 0)


def test_mart_2d_fan_table1(torch_cuda):
    """Table 1's 2-D reconstruction: ray-sequential MART with the update of
    Eq. 18 and relaxation 0.4, 10 iterations, f0 = 1; then the per-view
    schedule (power form) on the same scan."""
    from paper_2208_12964_gb300 import uspg

    spec = synth.workload("2d-fan-128r-50v-101")
    proj = synth.projections(spec)
    g = Gpu(spec).build()
    o = oracle_for(spec)
    f0 = np.ones(o.n_cells)
    ref, _ = o.mart_sequential(proj, f0, 10, 0.4, rule=1)
    got = _run_mart(g, proj, f0, 10, 0.4, uspg.SEQUENTIAL, rule=uspg.LINEAR_EQ18)
    assert rel_l2(got, ref) < TOL_IMG
    assert np.all(got >= 0)
    ref = o.mart_per_view(proj, f0, 3, 0.4)
    got = _run_mart(g, proj, f0, 3, 0.4, uspg.PER_VIEW)
    assert rel_l2(got, ref) < TOL_IMG


@pytest.mark.parametrize("rings,placement", [(90, "shared memory"), (150, "split"), (300, "split"),
                                           (400, "global memory")])
def test_mart_sequential_image_placement(torch_cuda, rings, placement):
    """The ray-sequential kernel keeps the image in its block's shared memory
    when it fits (6n grid of 24,570 cells), its inner rings in shared memory
    and the rest in global memory when at least an eighth fits (67,950 and
    270,900 cells), else all of it in global memory (481,200 cells)."""
    spec = synth.parallel_workload(rings, 5, 2 * rings + 1, seed=rings)
    proj = synth.projections(spec)
    g = Gpu(spec).build()
    o = oracle_for(spec)
    f0 = np.ones(o.n_cells)
    ref, _ = o.mart_sequential(proj, f0, 2, 0.3)
    got = _run_mart(g, proj, f0, 2, 0.3, 0)
    assert rel_l2(got, ref) < TOL_IMG, placement


@pytest.mark.parametrize("rule", [0, 1])
def test_mart_sequential_rules_and_stop(torch_cuda, rule):
    from paper_2208_12964_gb300 import uspg

    spec = synth.parallel_workload(12, 18, 25, seed=5)
    proj = synth.projections(spec)
    g = Gpu(spec).build()
    o = oracle_for(spec)
    f0 = np.ones(o.n_cells)
    ref, _ = o.mart_sequential(proj, f0, 4, 0.3, rule=rule)
    got = _run_mart(g, proj, f0, 4, 0.3, 0, rule=rule)
    assert rel_l2(got, ref) < TOL_IMG
    # Eq. 19: consistent data from the oracle's own forward projection
    fstar = 0.5 + np.random.default_rng(1).random(o.n_cells)
    p = np.stack([o.forward(k, fstar) for k in range(18)]).astype(np.float32)
    _run_mart(g, p, fstar, 30, 0.3, 0, rule=rule, tol=1e-3)
    assert uspg.uspg_mart_sweeps(g.ctx) == 1


def test_mart_per_view_3d_noisy(torch_cuda):
    spec = synth.cone_workload(16, 12, 24, 32, iterations=3, lam=0.1, seed=9)
    proj = synth.projections(spec)
    g = Gpu(spec).build()
    o = oracle_for(spec)
    f0 = np.ones(o.n_cells)
    ref = o.mart_per_view(proj, f0, 3, 0.1)
    # tuning the stage ring leaves the image untouched and the result equal
    g.U.uspg_set_projections(g.ctx, proj, False)
    g.U.uspg_set_image(g.ctx, np.full(o.n_cells, 0.5, np.float32), False)
    choice = g.U.uspg_autotune(g.ctx)
    assert choice[0] in (0, 2, 4, 6, 8) and choice[1] in (0, 2, 4, 6, 8)
    kept = np.zeros(o.n_cells, np.float32)
    g.U.uspg_get_image(g.ctx, kept, False)
    assert np.all(kept == 0.5)
    got = _run_mart(g, proj, f0, 3, 0.1, 1)
    assert rel_l2(got, ref) < TOL_IMG
    assert np.all(got >= 0) and np.any(got == 0)  # noisy zero rays zero their cells


def test_mart_per_view_2d_custom_order(torch_cuda):
    spec = synth.parallel_workload(40, 30, 81, seed=4)
    proj = synth.projections(spec)
    g = Gpu(spec).build()
    o = oracle_for(spec)
    order = np.random.default_rng(2).permutation(30)
    f0 = np.ones(o.n_cells)
    ref = o.mart_per_view(proj, f0, 4, 0.3, order=order)
    got = _run_mart(g, proj, f0, 4, 0.3, 1, order=order)
    assert rel_l2(got, ref) < TOL_IMG


def test_mart_per_view_full_size_first_view(torch_cuda):
    """The 128-ring, 128-slab, 90-view cone at full size, in the bench's launch
    configuration: one per-view step (view 0, f0 = 1) against the oracle's
    one-step image over all 6.3 M cells; then the whole first sweep's image
    stays finite, non-negative and changes only where rays pass."""
    spec = synth.workload("3d-cone-128r-128s-90v-256")
    proj = synth.projections(spec)
    g = Gpu(spec).build()
    o = oracle_for(spec)
    U = g.U
    U.uspg_set_projections(g.ctx, proj, False)
    U.uspg_fill_image(g.ctx, 1.0)
    U.uspg_autotune(g.ctx)
    opts, keep = U.mart_opts(1, 0.1, U.PER_VIEW, view_steps=1)
    U.uspg_mart(g.ctx, opts)
    U.uspg_sync(g.ctx)
    got = np.zeros(o.n_cells, np.float32)
    U.uspg_get_image(g.ctx, got, False)
    ref = np.ones(o.n_cells)
    o.set_threads(16)
    o.mart_views_sample(proj, ref, [0], 0.1)
    hit = ref != 1.0
    assert hit.sum() > 0.5 * o.n_cells
    assert np.all(got[~hit] == 1.0)
    nz = ref > 0
    assert np.all(got[~nz] == 0.0)
    assert np.max(np.abs(got[nz] - ref[nz]) / ref[nz]) < 2e-5
# --------------------------------------------------------------- resample ---

def test_resample_point_and_bijection(torch_cuda):
    from paper_2208_12964_gb300 import uspg

    spec = synth.parallel_workload(16, 4, 33, sector_rule=synth.SECT_4_2N1)
    g = Gpu(spec)
    o = oracle_for(spec)
    f = np.random.default_rng(0).random(o.n_cells).astype(np.float32)
    uspg.uspg_set_image(g.ctx, f, False)
    for nx, ny in ((64, 64), (37, 53), (1, 1)):
        out = np.zeros((1, ny, nx), np.float32)
        uspg.uspg_resample_cartesian(g.ctx, uspg.RESAMPLE_POINT, nx, ny, out, False)
        ref = o.resample_point(f.astype(np.float64), nx, ny)
        assert np.array_equal(out, ref.astype(np.float32))
    out = np.zeros((1, 32, 32), np.float32)
    uspg.uspg_resample_cartesian(g.ctx, uspg.RESAMPLE_BIJECTION, 32, 32, out, False)
    assert np.array_equal(out, o.resample_bijection(f.astype(np.float64)).astype(np.float32))


def test_resample_3d_slabs(torch_cuda):
    from paper_2208_12964_gb300 import uspg

    spec = synth.cone_workload(8, 5, 6, 16, noise=False)
    g = Gpu(spec)
    o = oracle_for(spec)
    f = np.random.default_rng(1).random(o.n_cells).astype(np.float32)
    uspg.uspg_set_image(g.ctx, f, False)
    out = np.zeros((5, 24, 24), np.float32)
    uspg.uspg_resample_cartesian(g.ctx, uspg.RESAMPLE_POINT, 24, 24, out, False)
    assert np.array_equal(out, o.resample_point(f.astype(np.float64), 24, 24).astype(np.float32))


# ------------------------------------------------------------- edge cases ---

def test_errors_and_degenerate_inputs(torch_cuda):
    from paper_2208_12964_gb300 import uspg

    spec = synth.parallel_workload(4, 3, 9)
    g = Gpu(spec)
    o, _ = uspg.mart_opts(1, 0.5, uspg.PER_VIEW)
    with pytest.raises(uspg.UspgError) as e:
        uspg.uspg_mart(g.ctx, o)
    assert e.value.status == uspg.ENOTREADY
    g.build()
    with pytest.raises(uspg.UspgError):
        uspg.uspg_mart(g.ctx, uspg.mart_opts(1, 2.5, uspg.PER_VIEW)[0])
    bad = dict(spec, n_rings=0)
    with pytest.raises(uspg.UspgError) as e:
        Gpu(bad)
    assert e.value.status == uspg.EINVAL
    # detector wider than the disk: outer rays miss and keep empty rows (the
    # pitch keeps every ray off the ring circles: an exactly tangent ray's
    # chord is the square root of a rounding error)
    wide = synth.parallel_workload(4, 3, 9)
    wide["du"] = 0.47
    gw = Gpu(wide).build()
    ow = oracle_for(wide)
    for k in range(3):
        for b in range(9):
            gc, gwt = gw.row(k, b)
            oc, owt = ow.row(k, b)
            assert_rows_equal(gc, gwt, oc, owt, TOL_W)
    assert len(gw.row(0, 0)[0]) == 0
    # zero iterations leave the image unchanged
    f0 = np.full(ow.n_cells, 0.7, np.float32)
    got = _run_mart(gw, np.ones((3, 9), np.float32), f0, 0, 0.5, 1)
    assert np.array_equal(got, f0)


# -------------------------------------------------------------- precision ---

@pytest.mark.parametrize("dtype,wtol", [("f16", 2 ** -10), ("bf16", 2 ** -7)])
def test_reduced_precision_rows(torch_cuda, dtype, wtol):
    """FP16/BF16 stores keep the index lists exact; each weight is the FP64
    length rounded once to the storage format (relative error <= one unit in
    the last place; FP16 weights are stored in units of the cell size)."""
    from paper_2208_12964_gb300 import uspg

    spec = synth.cone_workload(12, 8, 18, 24, noise=False)
    g = Gpu(spec, dtype=uspg.F16 if dtype == "f16" else uspg.BF16).build()
    o = oracle_for(spec)
    rng = np.random.default_rng(21)
    for _ in range(300):
        k, ray = int(rng.integers(18)), int(rng.integers(24 * 24))
        gc, gw = g.row(k, ray)
        oc, ow = o.row(k, ray)
        assert np.array_equal(gc, oc)
        big = ow > 1e-4 * spec["r"]  # below that, FP16 subnormals round coarser
        if big.any():
            assert np.max(np.abs(gw[big] - ow[big]) / ow[big]) <= wtol


def test_reduced_precision_mart_error(torch_cuda):
    """Image error of the per-view MART against the FP64 oracle for FP32, FP16
    and BF16 coefficient stores (FP32 accumulation throughout)."""
    from paper_2208_12964_gb300 import uspg

    spec = synth.cone_workload(16, 12, 24, 32, iterations=3, lam=0.1, seed=9)
    proj = synth.projections(spec)
    o = oracle_for(spec)
    f0 = np.ones(o.n_cells)
    ref = o.mart_per_view(proj, f0, 3, 0.1)
    err = {}
    for name, dt in (("f32", uspg.F32), ("f16", uspg.F16), ("bf16", uspg.BF16)):
        g = Gpu(spec, dtype=dt).build()
        got = _run_mart(g, proj, f0, 3, 0.1, 1)
        err[name] = rel_l2(got, ref)
    print("rel-L2 vs FP64 oracle:", err)
    assert err["f32"] < TOL_IMG
    assert err["f16"] < 2e-3
    assert err["bf16"] < 1e-2


# ---------------------------------------------------------------- batched ---

def test_batched_instances_match_single_runs(torch_cuda):
    """Contexts of different grids, view counts and detectors advanced together
    in one graph give each context the image its own uspg_mart gives."""
    from paper_2208_12964_gb300 import uspg

    specs = [synth.parallel_workload(12, 18, 25, seed=31, iterations=3, lam=0.3),
             synth.parallel_workload(20, 36, 41, seed=32, iterations=3, lam=0.3),
             synth.parallel_workload(7, 10, 15, seed=33, iterations=3, lam=0.3),
             synth.cone_workload(10, 6, 12, 16, iterations=3, lam=0.2, seed=34),
             synth.cone_workload(14, 10, 18, 24, iterations=3, lam=0.2, seed=35)]
    gs, projs, refs = [], [], []
    for sp in specs:
        g = Gpu(sp).build()
        p = synth.projections(sp)
        n = g.stats()["n_cells"]
        refs.append(_run_mart(g, p, np.ones(n), 3, 0.3 if sp["geometry"] == 0 else 0.2, 1))
        gs.append(g)
        projs.append(p)
    # lambda differs between the two families: run one batch per family
    for fam, lam in ((0, 0.3), (1, 0.2)):
        sel = [i for i, sp in enumerate(specs) if sp["geometry"] == fam]
        for i in sel:
            uspg.uspg_fill_image(gs[i].ctx, 1.0)
        opts, _ = uspg.mart_opts(3, lam, uspg.PER_VIEW)
        b = uspg.uspg_batch_create([gs[i].ctx for i in sel], opts)
        try:
            info = uspg.uspg_batch_info(b)
            assert info["steps"] == 3 * max(specs[i]["n_views"] for i in sel)
            uspg.uspg_batch_run(b)
            torch_cuda.cuda.synchronize()
        finally:
            uspg.uspg_batch_destroy(b)
        for i in sel:
            got = np.zeros(gs[i].stats()["n_cells"], np.float32)
            uspg.uspg_get_image(gs[i].ctx, got, False)
            assert rel_l2(got, refs[i]) < 1e-5, i


# ------------------------------------------ first-view segment store (binary) ---

def _segment_case(case):
    if case == "parallel64":
        return synth.workload("2d-parallel-64r-36v")
    if case == "fan128":
        return synth.workload("2d-fan-128r-50v-101-segments")
    spec = synth.cone_workload(12, 8, 18, 24, noise=False)
    if case == "cone12_4n":
        spec["sector_rule"] = synth.SECT_4_2N1
    return spec


@pytest.mark.parametrize("case", ["parallel64", "fan128", "cone12_6n", "cone12_4n"])
def test_segment_store_rows_all_views(torch_cuda, case):
    """The paper's store (Algorithm 1): one set of first-view segments; every
    view's binary row enumerated on the GPU from the segments turned by the
    view's source angle, against the oracle's re-binned row, bit for bit."""
    from paper_2208_12964_gb300 import uspg

    spec = _segment_case(case)
    g = Gpu(spec, weight_mode=uspg.BINARY, store_form=uspg.STORE_SEGMENTS).build()
    o = oracle_for(spec, weight_mode=1, store_form=1)
    st = g.stats()
    assert st["n_reps"] == 1 and st["mirrored"] == 0
    assert st["nnz_store"] == sum(len(o.segments(r)[0]) for r in range(o.n_rays))
    total = 0
    for k in range(spec["n_views"]):
        for ray in range(o.n_rays):
            gc, gw = g.row(k, ray)
            oc, ow = o.rebin_row(k, ray)
            assert np.array_equal(gc, oc), f"{case} view {k} ray {ray}"
            assert np.all(gw == 1.0)
            total += len(oc)
    assert total == st["nnz_all_views"]
    assert st["store_bytes"] < st["full_matrix_bytes"]


@pytest.mark.parametrize("case,rule", [("fan128", 1), ("fan128", 0), ("cone12_6n", 1)])
def test_segment_store_sequential_mart(torch_cuda, case, rule):
    """Ray-sequential MART over the segment store (unit coefficients: the
    power update is (P/Pbar)^lambda, Eq. 18 is 1 - lambda (1 - P/Pbar))
    against the oracle; the 128-ring fan keeps its outer rings in shared
    memory, the 12-ring cone all of it."""
    from paper_2208_12964_gb300 import uspg

    spec = _segment_case(case)
    proj = synth.projections(spec)
    g = Gpu(spec, weight_mode=uspg.BINARY, store_form=uspg.STORE_SEGMENTS).build()
    o = oracle_for(spec, weight_mode=1, store_form=1)
    f0 = np.ones(o.n_cells)
    ref, _ = o.mart_sequential(proj, f0, 3, 0.4, rule=rule)
    got = _run_mart(g, proj, f0, 3, 0.4, uspg.SEQUENTIAL, rule=rule)
    assert rel_l2(got, ref) < TOL_IMG
    assert np.all(got >= 0)
    with pytest.raises(uspg.UspgError) as e:
        uspg.uspg_mart(g.ctx, uspg.mart_opts(1, 0.4, uspg.PER_VIEW)[0])
    assert e.value.status == uspg.EUNSUPPORTED


def test_batched_instances_match_oracle(torch_cuda):
    """An uneven batch shaped like the 64-instance batched workload (2D
    parallel instances with 64, 128, 256 and 512 rings, 18 to 90 views, 2R+1
    bins), plus a mirrored cone (odd detector rows and slab count, Poisson
    noise) and an off-centre cone (every row stored), advanced together in one
    graph: every instance's image against the oracle's per-view MART."""
    import os

    from paper_2208_12964_gb300 import uspg

    specs = [synth.parallel_workload(64, 18, 129, seed=41, iterations=3, lam=0.2),
             synth.parallel_workload(128, 36, 257, seed=42, iterations=3, lam=0.2),
             synth.parallel_workload(256, 18, 513, seed=43, iterations=3, lam=0.2),
             synth.parallel_workload(512, 18, 1025, seed=44, iterations=3, lam=0.2),
             synth.parallel_workload(64, 90, 129, seed=45, iterations=3, lam=0.2),
             synth.cone_workload(10, 9, 12, 21, iterations=3, lam=0.2, seed=46),
             synth.cone_workload(10, 8, 12, 20, iterations=3, lam=0.2, seed=47, noise=False)]
    specs[-1]["z_min"] = -0.75  # off-centre stack: no z-mirror
    gs, projs = [], []
    for sp in specs:
        g = Gpu(sp).build()
        p = synth.projections(sp)
        uspg.uspg_set_projections(g.ctx, p, False)
        uspg.uspg_fill_image(g.ctx, 1.0)
        gs.append(g)
        projs.append(p)
    assert [g.stats()["mirrored"] for g in gs[-2:]] == [1, 0]
    opts, _ = uspg.mart_opts(3, 0.2, uspg.PER_VIEW)
    b = uspg.uspg_batch_create([g.ctx for g in gs], opts)
    try:
        tun = uspg.uspg_batch_tuning(b)  # one launch shape per ring count
        assert sorted(q["rings"] for q in tun["buckets"]) == sorted({sp["n_rings"] for sp in specs})
        assert tun["ms_default"] > 0 and tun["ms_tuned"] > 0
        uspg.uspg_batch_run(b)
        torch_cuda.cuda.synchronize()
    finally:
        uspg.uspg_batch_destroy(b)
    for i, (sp, g, p) in enumerate(zip(specs, gs, projs)):
        n = g.stats()["n_cells"]
        got = np.zeros(n, np.float32)
        uspg.uspg_get_image(g.ctx, got, False)
        o = oracle_for(sp, threads=os.cpu_count() or 8)
        ref = o.mart_per_view(p, np.ones(n), 3, 0.2)
        err = rel_l2(got, ref)
        worst = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        print(f"instance {i} ({sp['name']}): rel-L2 {err:.2e}, max |diff| / max |f| {worst:.2e}")
        assert err < TOL_IMG, i
        assert worst < 10 * TOL_IMG, i
        g.close()


@pytest.mark.parametrize("case", ["parallel", "cone_mirror_odd", "cone_off_centre", "cone_f16"])
def test_mart_per_view_linear_eq18(torch_cuda, case):
    """Per-view MART with the update of Eq. 18: every cell is corrected once
    per view by the weighted mean of its rays' factors 1 - beta (1 - P/Pbar),
    against the oracle (FP32 stores within 1e-4 relative L2; an FP16 store
    within its rounding)."""
    from paper_2208_12964_gb300 import uspg

    dtype, tol, beta = uspg.F32, TOL_IMG, 0.2
    if case == "parallel":
        spec, beta = synth.parallel_workload(40, 30, 81, seed=7), 0.4
    elif case == "cone_mirror_odd":
        spec = synth.cone_workload(10, 9, 12, 21, seed=8)
    elif case == "cone_off_centre":
        spec = synth.cone_workload(10, 8, 12, 20, seed=9, noise=False)
        spec["z_min"] = -0.75
    else:
        spec, dtype, tol = synth.cone_workload(16, 12, 24, 32, seed=10), uspg.F16, 2e-3
    proj = synth.projections(spec)
    g = Gpu(spec, dtype=dtype).build()
    o = oracle_for(spec)
    f0 = np.ones(o.n_cells)
    ref = o.mart_per_view(proj, f0, 3, beta, rule=oracle.LINEAR_EQ18)
    got = _run_mart(g, proj, f0, 3, beta, uspg.PER_VIEW, rule=uspg.LINEAR_EQ18)
    err = rel_l2(got, ref)
    print(f"{case}: rel-L2 {err:.2e}")
    assert err < tol
    assert np.all(got > 0)  # Eq. 18 factors stay positive for beta < 1 and P >= 0


@pytest.mark.parametrize("rule", [0, 1])
def test_mart_per_view_eq19_stop(torch_cuda, rule):
    """Eq. 19 in the per-view schedule.  Consistent data p = A f* (the
    oracle's forward projection) started at f*: the first sweep moves no cell
    by more than 1e-3 of its value, so one sweep runs and the image stays f*.
    Started at f = 1, with a tolerance chosen where the oracle's decision is
    robust (the same sweep count for 0.98 and 1.02 times it): the GPU stops
    after the same sweep as the oracle, with the same image."""
    from paper_2208_12964_gb300 import uspg

    spec = synth.parallel_workload(12, 18, 25, seed=5)
    g = Gpu(spec).build()
    o = oracle_for(spec)
    fstar = 0.5 + np.random.default_rng(1).random(o.n_cells)
    p = np.stack([o.forward(k, fstar) for k in range(18)]).astype(np.float32)
    got = _run_mart(g, p, fstar, 30, 0.3, uspg.PER_VIEW, rule=rule, tol=1e-3)
    assert uspg.uspg_mart_sweeps(g.ctx) == 1
    assert np.max(np.abs(got / fstar - 1)) < 1e-5
    f0 = np.ones(o.n_cells)
    pick = None
    for t in np.logspace(-1, -5, 33):
        n = [o.mart_per_view(p, f0, 12, 0.3, rule=rule, tol=t * m, return_sweeps=True)[1] for m in (0.98, 1, 1.02)]
        if n[0] == n[1] == n[2] and 3 <= n[1] < 12:
            pick = (t, n[1])
            break
    assert pick is not None
    t, n_ref = pick
    ref = o.mart_per_view(p, f0, 12, 0.3, rule=rule, tol=t)
    got = _run_mart(g, p, f0, 12, 0.3, uspg.PER_VIEW, rule=rule, tol=t)
    assert uspg.uspg_mart_sweeps(g.ctx) == n_ref
    assert rel_l2(got, ref) < TOL_IMG
    # without a tolerance every sweep runs
    _run_mart(g, p, f0, 4, 0.3, uspg.PER_VIEW, rule=rule)
    assert uspg.uspg_mart_sweeps(g.ctx) == 4
    with pytest.raises(uspg.UspgError) as e:  # Eq. 19 is checked on whole sweeps only
        uspg.uspg_mart(g.ctx, uspg.mart_opts(2, 0.3, uspg.PER_VIEW, rule, 1e-3, view_steps=5)[0])
    assert e.value.status == uspg.EINVAL


@pytest.mark.parametrize("bad", [float("nan"), -1.0])
def test_device_projections_with_bad_values_are_flagged(torch_cuda, bad):
    """Projections handed over in device memory are checked while they are
    copied: a value that is not finite and >= 0 raises the context's device
    flag, which uspg_sync reports as EDEVICE (and then clears).  A ray that
    carries such a value is skipped by both schedules: the image stays finite
    and non-negative."""
    torch = torch_cuda
    from paper_2208_12964_gb300 import uspg

    spec = synth.parallel_workload(12, 18, 25, seed=5)
    g = Gpu(spec).build()
    p = torch.from_numpy(synth.projections(spec)).cuda()
    p[3, 7] = bad
    uspg.uspg_set_projections(g.ctx, p, True)
    with pytest.raises(uspg.UspgError) as e:
        uspg.uspg_sync(g.ctx)
    assert e.value.status == uspg.EDEVICE
    assert "finite" in uspg.uspg_last_error(g.ctx)
    uspg.uspg_sync(g.ctx)  # the flag was cleared when it was reported
    n = g.stats()["n_cells"]
    for schedule in (uspg.PER_VIEW, uspg.SEQUENTIAL):
        uspg.uspg_fill_image(g.ctx, 1.0)
        uspg.uspg_mart(g.ctx, uspg.mart_opts(2, 0.3, schedule)[0])
        uspg.uspg_sync(g.ctx)
        f = np.zeros(n, np.float32)
        uspg.uspg_get_image(g.ctx, f, False)
        assert np.all(np.isfinite(f)) and np.all(f >= 0), schedule
