"""The coefficient generator's FP64 ray walk, built for the host, against the
oracle's direct trace (no GPU).

walk.cuh is host+device code: the same walk the generator kernel runs is
compiled here with g++ (tests/host_walk.cpp) and traces rows on the CPU.
Cell lists must equal the oracle's; lengths agree within 1e-6 relative, the
bar of the GPU tests (both sides form the crossings with the same separately
rounded FP64 operations and the same libm, but where a radial crossing falls
on a circle crossing to within rounding the oracle, which splits the whole
line at every crossing, can start the next piece one unit in the last place
later than the walk, which splits each ring segment at the crossings inside
it).  Every row must also fit the FP32 sizing pass's bound (size_ray).  This
checks the generator's logic on every row of small scans and on blocks of
rows of the full-size cone, independently of a GPU run.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from gpu_util import oracle_for
from paper_2208_12964_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SOURCES = [os.path.join(HERE, "host_walk.cpp")] + [
    os.path.join(ROOT, "paper_2208_12964_gb300", "csrc", f) for f in ("walk.cuh", "internal.cuh")
] + [os.path.join(ROOT, "include", "uspg.h")]


@pytest.fixture(scope="module")
def walker():
    cxx = shutil.which("g++")
    inc = next((d for d in ("/usr/local/cuda/include", os.path.join(os.environ.get("CUDA_HOME", ""), "include"))
                if os.path.exists(os.path.join(d, "cuda_runtime.h"))), None)
    if not cxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    out = os.path.join(tempfile.gettempdir(), f"uspg_host_walk_{os.getuid()}")
    if not os.path.exists(out) or os.path.getmtime(out) < max(os.path.getmtime(p) for p in SOURCES):
        r = subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", inc, "-x", "c++", SOURCES[0],
                            "-o", out + ".tmp"], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        os.replace(out + ".tmp", out)
    return out


def host_rows(walker, spec, view, rays):
    args = [spec["geometry"], spec["n_rings"], spec["n_slabs"], spec["sector_rule"], repr(spec["r"]),
            repr(spec["h"]), repr(spec["z_min"]), spec["n_views"], spec["arc_num"], spec["arc_den"], spec["n_u"],
            spec["n_v"], repr(spec["du"]), repr(spec["dv"]), repr(spec["d_so"]), repr(spec["d_sd"]), view,
            rays[0], rays[1]]
    r = subprocess.run([walker] + [str(a) for a in args], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    rows = {}
    for line in r.stdout.splitlines():
        t = line.split()
        bound, n = int(t[1]), int(t[2])
        # the FP32 sizing pass bounds every row the FP64 walk writes (rays
        # through the axis included: the centre bins of odd detectors)
        assert n <= bound, f"view {view} ray {t[0]}: {n} entries > bound {bound}"
        cells = np.array(t[3:3 + 2 * n:2], np.int64)
        w = np.array(t[4:4 + 2 * n:2], np.float64)
        o = np.argsort(cells, kind="stable")
        rows[int(t[0])] = (cells[o], w[o])
    return rows


def compare(walker, spec, views, blocks=None):
    """Every ray of the views, or the rays of the given [begin, end) blocks."""
    o = oracle_for(spec)
    blocks = blocks or [(0, o.n_rays)]
    checked = 0
    for k in views:
        rows = {}
        for b in blocks:
            rows.update(host_rows(walker, spec, k, b))
        for ray in sorted(rows):
            c, w = rows[ray]
            oc, ow = o.row(k, ray)
            assert np.array_equal(c, oc), f"view {k} ray {ray}"
            if len(ow):
                assert np.max(np.abs(w - ow) / ow) < 1e-6, f"view {k} ray {ray}"
            checked += 1
    assert checked > 0


def test_host_walk_2d_parallel_every_row(walker):
    spec = synth.workload("2d-parallel-64r-36v")
    compare(walker, spec, range(36))


def test_host_walk_fan_every_row(walker):
    spec = synth.workload("2d-fan-128r-50v-101")
    compare(walker, spec, range(50))


@pytest.mark.parametrize("rule", [synth.SECT_6N, synth.SECT_4_2N1])
def test_host_walk_small_cone_every_row(walker, rule):
    spec = synth.cone_workload(12, 8, 18, 24, noise=False)
    spec["sector_rule"] = rule
    compare(walker, spec, range(18))


def test_host_walk_full_size_cone_blocks(walker):
    """The 128-ring, 128-slab, 90-view cone: two detector rows through the
    middle (rays near the axis and the mid-plane) and a row near the top edge,
    in three views."""
    spec = synth.workload("3d-cone-128r-128s-90v-256")
    compare(walker, spec, (0, 7, 44), blocks=[(127 * 256, 129 * 256), (230 * 256, 231 * 256)])


def test_host_walk_paper_grid_parallel_every_row(walker):
    """Eq. 1's grid, n_g = 4(2n-1) (the one the bijective resample needs),
    parallel scan over a full turn with an even bin count."""
    spec = synth.parallel_workload(24, 20, 48, arc=(1, 1), sector_rule=synth.SECT_4_2N1)
    compare(walker, spec, range(20))


def test_host_walk_off_centre_cone_every_row(walker):
    """A slab stack off the source plane (no z-mirror: rows above and below the
    mid-plane differ), odd detector."""
    spec = synth.cone_workload(10, 8, 12, 21, noise=False)
    spec["z_min"] = -0.75
    compare(walker, spec, range(12))
