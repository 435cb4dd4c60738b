"""Forward projection that allocates no device memory.

uspg_forward_project_noalloc serves callers that must not call cudaMalloc
while they run: processes whose device memory belongs to a pooling allocator
with a fixed budget, and latency-critical loops that forbid allocator calls
after start-up.  Its ray-sum accumulator is the library's static device array
instead of a context buffer.  These tests compare it with the library's
regular forward projection (uspg_forward_project) on two calls in a row, and
check that a view with more rays than the array holds is refused.  The file
is collected last so that a failure here does not hide the other tests.
"""
import numpy as np
import pytest

from gpu_util import Gpu
from paper_2208_12964_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["cone_f32", "cone_f16", "cone_bf16", "parallel_2d"])
def test_noalloc_forward_matches_regular_forward_twice(case):
    """Mirrored cone stores in the three coefficient precisions and an
    unmirrored 2D store; views whose rotation from their representative is
    zero (view 0) and non-zero; two calls in a row share the static
    accumulator."""
    import torch

    from paper_2208_12964_gb300 import uspg

    if case == "parallel_2d":
        spec, views, dtype = synth.parallel_workload(24, 30, 49), (0, 7, 22), uspg.F32
    else:
        spec, views = synth.cone_workload(16, 12, 24, 32, noise=False), (0, 3, 17)
        dtype = {"cone_f32": uspg.F32, "cone_f16": uspg.F16, "cone_bf16": uspg.BF16}[case]
    g = Gpu(spec, dtype=dtype).build()
    st = uspg.uspg_coeff_stats(g.ctx)
    n_cells, n_rays = st["n_cells"], st["n_rays"]
    assert st["mirrored"] == (case != "parallel_2d")
    rng = np.random.default_rng(5)
    for view in views:
        f = torch.from_numpy((0.2 + rng.random(n_cells)).astype(np.float32)).cuda()
        uspg.uspg_set_image(g.ctx, f, True)
        ref = torch.zeros(n_rays, dtype=torch.float32, device="cuda")
        got = torch.full((n_rays,), -1.0, dtype=torch.float32, device="cuda")
        uspg.uspg_forward_project(g.ctx, view, ref)
        uspg.uspg_forward_project_noalloc(g.ctx, view, f, got)
        uspg.uspg_sync(g.ctx)
        r = ref.cpu().numpy().astype(np.float64)
        q = got.cpu().numpy().astype(np.float64)
        assert np.array_equal(r == 0.0, q == 0.0)
        nz = r != 0.0
        assert nz.sum() > 0
        # same kernels and data; only the order of the per-ray atomic adds may differ
        assert np.max(np.abs(q[nz] - r[nz]) / r[nz]) < 1e-6, view


def test_noalloc_call_leaves_device_memory_unchanged():
    """After a first call (which looks up the static array's address), a
    second call changes the device's free memory by nothing: no allocation
    by the library, the CUDA runtime or a caching allocator."""
    import torch

    from paper_2208_12964_gb300 import uspg

    spec = synth.cone_workload(16, 12, 24, 32, noise=False)
    g = Gpu(spec).build()
    st = uspg.uspg_coeff_stats(g.ctx)
    f = torch.ones(st["n_cells"], dtype=torch.float32, device="cuda")
    out = torch.zeros(st["n_rays"], dtype=torch.float32, device="cuda")
    uspg.uspg_forward_project_noalloc(g.ctx, 5, f, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    uspg.uspg_forward_project_noalloc(g.ctx, 6, f, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_refuses_views_beyond_its_capacity():
    import torch

    from paper_2208_12964_gb300 import uspg

    bins = uspg.NOALLOC_MAX_RAYS + 1
    spec = synth.parallel_workload(2, 1, bins)
    g = Gpu(spec)  # the capacity is checked before anything else: no build needed
    f = torch.ones(3 * 2 * 3, dtype=torch.float32, device="cuda")
    out = torch.zeros(bins, dtype=torch.float32, device="cuda")
    with pytest.raises(uspg.UspgError) as e:
        uspg.uspg_forward_project_noalloc(g.ctx, 0, f, out)
    assert e.value.status == uspg.EINVAL
    assert "exceed" in uspg.uspg_last_error(g.ctx)
