"""The C ABI library builds, loads and exports every entry point that
include/uspg.h declares; host-side validation works without a GPU; the
product path does not reach the oracle."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "uspg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(uspg_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def U():
    from paper_2208_12964_gb300 import build

    build.build()
    from paper_2208_12964_gb300 import uspg

    return uspg


def test_every_declared_symbol_is_exported(U):
    import ctypes

    lib = ctypes.CDLL(U.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header(U):
    for n in declared_functions():
        assert hasattr(U, n), f"binding lacks {n}"


def test_create_validates_on_host(U):
    from paper_2208_12964_gb300 import synth

    spec = synth.workload("2d-parallel-64r-36v")
    g, s, o, _ = U.descs_from_spec(spec)
    ctx = U.uspg_create(g, s, o)
    assert ctx
    U.uspg_destroy(ctx)
    for field, val in (("n_rings", 0), ("n_rings", 2000), ("ring_width", -1.0)):
        g2, s2, o2, _ = U.descs_from_spec(spec)
        setattr(g2, field, val)
        with pytest.raises(U.UspgError) as e:
            U.uspg_create(g2, s2, o2)
        assert e.value.status == U.EINVAL
    g3, s3, o3, _ = U.descs_from_spec(spec)
    s3.n_views = 0
    with pytest.raises(U.UspgError):
        U.uspg_create(g3, s3, o3)
    g4, s4, o4, _ = U.descs_from_spec(synth.workload("3d-cone-128r-128s-90v-256"))
    s4.src_to_axis = 0.5  # source inside the cylinder
    with pytest.raises(U.UspgError):
        U.uspg_create(g4, s4, o4)
    g5, s5, o5, _ = U.descs_from_spec(spec)
    o5.coeff_dtype = 9
    with pytest.raises(U.UspgError):
        U.uspg_create(g5, s5, o5)
    assert "coeff_dtype" in U.uspg_last_error(None)


def test_product_path_never_reaches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2208_12964_gb300")
    for dp, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dp, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text and "uspg_oracle" not in text, f


def test_oracle_and_library_share_no_source():
    csrc = os.path.join(ROOT, "paper_2208_12964_gb300", "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        assert "oracle" not in text.lower() or "oracle" not in re.findall(r'#include\s+"([^"]+)"', text), f
    orc = open(os.path.join(ROOT, "oracle", "uspg_oracle.c")).read()
    assert "#include \"" not in orc  # only system headers


def test_server_create_validates_on_host(U):
    for budget, active, chunk in ((0, 2, 4), (1 << 30, 0, 4), (1 << 30, 2, 0)):
        with pytest.raises(U.UspgError) as e:
            U.uspg_server_create(budget, active, chunk)
        assert e.value.status == U.EINVAL
    with pytest.raises(U.UspgError) as e:
        U._check(U.lib().uspg_server_submit(None, None, None))
    assert e.value.status == U.EINVAL


def test_create_validates_fan_scans_and_store_forms(U):
    """Host-side checks of the fan geometry (Table 1) and of the coefficient
    stores: a fan scan is 2D (n_v = 1, n_slabs = 1) with its source outside
    the grid; the first-view segment store holds binary coefficients only."""
    from paper_2208_12964_gb300 import synth

    fan = synth.workload("2d-fan-128r-50v-101")
    g, s, o, _ = U.descs_from_spec(fan)
    U.uspg_destroy(U.uspg_create(g, s, o))
    bad = []
    g1, s1, o1, _ = U.descs_from_spec(fan)
    s1.n_v = 2
    bad.append((g1, s1, o1, "n_v"))
    g2, s2, o2, _ = U.descs_from_spec(fan)
    s2.src_to_axis = 0.5  # inside the disk
    bad.append((g2, s2, o2, "src_to_det"))
    g3, s3, o3, _ = U.descs_from_spec(fan)
    o3.store_form = U.STORE_SEGMENTS  # with length weights
    bad.append((g3, s3, o3, "binary"))
    g4, s4, o4, _ = U.descs_from_spec(fan)
    o4.store_form = 7
    bad.append((g4, s4, o4, "store_form"))
    for g_, s_, o_, word in bad:
        with pytest.raises(U.UspgError) as e:
            U.uspg_create(g_, s_, o_)
        assert e.value.status == U.EINVAL
        assert word in U.uspg_last_error(None)
    seg = synth.workload("2d-fan-128r-50v-101-segments")
    g5, s5, o5, _ = U.descs_from_spec(seg)
    assert o5.weight_mode == U.BINARY and o5.store_form == U.STORE_SEGMENTS
    U.uspg_destroy(U.uspg_create(g5, s5, o5))


@pytest.mark.parametrize("bad", [float("nan"), -0.25, float("inf"), -float("inf")])
def test_set_projections_refuses_bad_host_data(U, bad):
    """Projections are measured line integrals: finite and >= 0 (noisy data
    clamped at 0).  Host data holding anything else are refused with EINVAL
    before any device work, and the message names the first bad value."""
    import numpy as np

    from paper_2208_12964_gb300 import synth

    spec = synth.parallel_workload(4, 3, 9)
    g, s, o, _ = U.descs_from_spec(spec)
    ctx = U.uspg_create(g, s, o)
    try:
        p = np.ones((3, 9), np.float32)
        p[0, 0] = 0.0
        p[1, 0] = -0.0  # minus zero is zero
        p[2, 4] = bad
        with pytest.raises(U.UspgError) as e:
            U.uspg_set_projections(ctx, p, False)
        assert e.value.status == U.EINVAL
        msg = U.uspg_last_error(ctx)
        assert "projection 22 (view 2, ray 4)" in msg and "finite and >= 0" in msg
    finally:
        U.uspg_destroy(ctx)


def test_create_refuses_unknown_symmetry_mode(U):
    from paper_2208_12964_gb300 import synth

    spec = dict(synth.parallel_workload(4, 3, 9), symmetry=7)
    g, s, o, _ = U.descs_from_spec(spec)
    with pytest.raises(U.UspgError) as e:
        U.uspg_create(g, s, o)
    assert e.value.status == U.EINVAL and "symmetry" in U.uspg_last_error(None)
    for mode in (U.SYMMETRY_AUTO, U.SYMMETRY_ALWAYS, U.SYMMETRY_NEVER):
        g, s, o, _ = U.descs_from_spec(dict(spec, symmetry=mode))
        U.uspg_destroy(U.uspg_create(g, s, o))


@pytest.mark.gpu
def test_set_projections_reports_the_first_bad_value_of_a_large_set(U, torch_cuda):
    """A projection set of a million values or more is copied to a staging
    buffer and checked on the device before the context's projections
    change; the reported value is the first bad one, and a refused set
    leaves the projections as they were."""
    import numpy as np

    from paper_2208_12964_gb300 import synth

    spec = synth.parallel_workload(4, 640, 4099)
    g, s, o, _ = U.descs_from_spec(spec)
    ctx = U.uspg_create(g, s, o)
    try:
        p = np.ones((640, 4099), np.float32)
        n = p.size
        for first in (n // 2 + 7, 5, n - 1):
            q = p.reshape(-1).copy()
            q[first] = np.nan
            q[-1] = -1.0  # a later bad value in the last part
            with pytest.raises(U.UspgError) as e:
                U.uspg_set_projections(ctx, q.reshape(p.shape), False)
            assert e.value.status == U.EINVAL
            v, r = divmod(first, 4099)
            assert f"projection {first} (view {v}, ray {r})" in U.uspg_last_error(ctx)
        U.uspg_set_projections(ctx, p, False)  # a good set goes through
        U.uspg_sync(ctx)
    finally:
        U.uspg_destroy(ctx)
