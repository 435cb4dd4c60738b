"""Reconstruction server (uspg_server_*): many MART jobs of different grids
and scans run concurrently by the library's scheduler thread.  Each job must
give the image its own uspg_mart gives when run alone (the same kernels on the
same store; only the order of the forward kernel's atomic additions may
differ), a repeated geometry must reuse its stored coefficients, and a job
whose store exceeds the device budget must be refused without disturbing the
others."""
import numpy as np
import pytest

from gpu_util import Gpu, oracle_for, rel_l2
from paper_2208_12964_gb300 import synth

pytestmark = pytest.mark.gpu


def _solo(sp, proj, iters, lam, schedule, rule=0):
    g = Gpu(sp).build()
    U = g.U
    U.uspg_set_projections(g.ctx, np.ascontiguousarray(proj, np.float32), False)
    U.uspg_fill_image(g.ctx, 1.0)
    o, _ = U.mart_opts(iters, lam, schedule, rule)
    U.uspg_mart(g.ctx, o)
    U.uspg_sync(g.ctx)
    f = np.zeros(g.stats()["n_cells"], np.float32)
    U.uspg_get_image(g.ctx, f, False)
    return f


def _wait(U, srv, ids, n_cells, timeout=300.0):
    U.uspg_server_drain(srv, timeout)
    out = {}
    for jid in ids:
        img = np.zeros(n_cells[jid], np.float32)
        r = U.uspg_server_poll(srv, jid, img)
        assert r is not None
        out[jid] = (r, img)
    return out


def test_mixed_jobs_match_their_solo_runs(torch_cuda):
    from paper_2208_12964_gb300 import uspg as U

    jobs = [  # (spec, iterations, lambda, schedule, rule)
        (synth.parallel_workload(20, 36, 41, seed=41, iterations=3, lam=0.3), 3, 0.3, U.PER_VIEW, U.POWER),
        (synth.cone_workload(10, 6, 12, 16, iterations=2, lam=0.2, seed=42), 2, 0.2, U.PER_VIEW, U.POWER),
        (synth.parallel_workload(12, 18, 25, seed=43, iterations=4, lam=0.25), 4, 0.25, U.SEQUENTIAL,
         U.LINEAR_EQ18),
        (synth.parallel_workload(20, 36, 41, seed=44, iterations=2, lam=0.3), 2, 0.3, U.PER_VIEW, U.POWER),
        (synth.cone_workload(14, 10, 18, 24, iterations=2, lam=0.2, seed=45), 2, 0.2, U.PER_VIEW, U.POWER),
        (synth.parallel_workload(20, 36, 41, seed=46, iterations=3, lam=0.1), 3, 0.1, U.PER_VIEW, U.POWER),
    ]
    projs = [synth.projections(sp) for sp, *_ in jobs]
    refs = [_solo(sp, p, it, lam, sch, rule) for (sp, it, lam, sch, rule), p in zip(jobs, projs)]
    srv = U.uspg_server_create(4 << 30, 3, 1)  # one sweep per chunk: jobs interleave sweep by sweep
    try:
        ids, n_cells = [], {}
        for q, ((sp, it, lam, sch, rule), p, ref) in enumerate(zip(jobs, projs, refs)):
            o, _ = U.mart_opts(it, lam, sch, rule)
            jid = U.uspg_server_submit(srv, sp, p, o, borrow=q % 2 == 1)  # projs stay alive until polled
            ids.append(jid)
            n_cells[jid] = len(ref)
        res = _wait(U, srv, ids, n_cells)
        st = U.uspg_server_stats(srv)
    finally:
        U.uspg_server_destroy(srv)
    for jid, ref, (sp, it, *_) in zip(ids, refs, jobs):
        r, img = res[jid]
        assert r["status"] == U.OK, (jid, r["message"])
        assert r["n_cells"] == len(ref)
        assert r["latency_s"] >= r["run_s"] > 0
        assert rel_l2(img, ref) < 1e-5, jid
    # jobs 0, 3 and 5 share one geometry: at least the last of them found it resident
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert st["store_reuses"] >= 1
    assert res[ids[5]][0]["reused_store"] == 1 or res[ids[3]][0]["reused_store"] == 1
    assert 0 < st["p50_s"] <= st["p99_s"]
    assert st["peak_device_bytes"] > 0


def test_concurrent_jobs_share_one_store(torch_cuda):
    """Four jobs of one geometry (different phantoms) submitted together: the
    first builds the store, the other three read it through contexts of their
    own while all four run at once."""
    from paper_2208_12964_gb300 import uspg as U

    specs = [synth.parallel_workload(24, 36, 49, seed=60 + q, iterations=3, lam=0.25) for q in range(4)]
    projs = [synth.projections(sp) for sp in specs]
    refs = [_solo(sp, p, 3, 0.25, U.PER_VIEW) for sp, p in zip(specs, projs)]
    srv = U.uspg_server_create(1 << 30, 4, 1)
    try:
        o, _ = U.mart_opts(3, 0.25, U.PER_VIEW)
        ids = [U.uspg_server_submit(srv, sp, p, o) for sp, p in zip(specs, projs)]
        res = _wait(U, srv, ids, {jid: len(ref) for jid, ref in zip(ids, refs)})
        st = U.uspg_server_stats(srv)
    finally:
        U.uspg_server_destroy(srv)
    for jid, ref in zip(ids, refs):
        r, img = res[jid]
        assert r["status"] == U.OK, r["message"]
        assert rel_l2(img, ref) < 1e-5, jid
    assert st["completed"] == 4 and st["store_reuses"] == 3
    assert sum(res[j][0]["reused_store"] for j in ids) == 3


@pytest.mark.parametrize("rule", [0, 1])
def test_server_job_matches_the_oracle(torch_cuda, rule):
    """One 2D per-view job through the server against the FP64 oracle, with
    the power update and with the per-view form of Eq. 18."""
    from paper_2208_12964_gb300 import uspg as U

    sp = synth.parallel_workload(16, 24, 33, seed=47, iterations=2, lam=0.3)
    p = synth.projections(sp)
    o = oracle_for(sp)
    ref = o.mart_per_view(p, np.ones(o.n_cells), 2, 0.3, rule=rule)
    srv = U.uspg_server_create(1 << 30, 2, 5)
    try:
        opts, _ = U.mart_opts(2, 0.3, U.PER_VIEW, rule)
        jid = U.uspg_server_submit(srv, sp, p, opts)
        res = _wait(U, srv, [jid], {jid: o.n_cells})
    finally:
        U.uspg_server_destroy(srv)
    r, img = res[jid]
    assert r["status"] == U.OK
    assert r["updates"] == 2 * Gpu(sp).build().stats()["nnz_all_views"]
    assert rel_l2(img, ref) < 1e-4


def test_over_budget_and_invalid_jobs_are_refused(torch_cuda):
    from paper_2208_12964_gb300 import uspg as U

    small = synth.parallel_workload(7, 10, 15, seed=48, iterations=2, lam=0.3)
    big = synth.parallel_workload(128, 90, 257, seed=49, iterations=1, lam=0.3)
    bad = dict(small, n_rings=0)
    ps, pb = synth.projections(small), synth.projections(big)
    ref = _solo(small, ps, 2, 0.3, U.PER_VIEW)
    srv = U.uspg_server_create(4 << 20, 2, 4)  # 4 MiB: the small store fits, the big one does not
    try:
        opts, _ = U.mart_opts(2, 0.3, U.PER_VIEW)
        o1, _ = U.mart_opts(1, 0.3, U.PER_VIEW)
        j_big = U.uspg_server_submit(srv, big, pb, o1)
        j_bad = U.uspg_server_submit(srv, bad, ps, opts)
        j_small = U.uspg_server_submit(srv, small, ps, opts)
        res = _wait(U, srv, [j_big, j_bad, j_small], {j_big: 1, j_bad: 1, j_small: len(ref)})
        st = U.uspg_server_stats(srv)
        with pytest.raises(U.UspgError) as e:
            U.uspg_server_poll(srv, j_small)  # already collected
        assert e.value.status == U.EINVAL
        with pytest.raises(U.UspgError) as e:
            bad_opts, _ = U.mart_opts(0, 0.3, U.PER_VIEW)
            U.uspg_server_submit(srv, small, ps, bad_opts)
        assert e.value.status == U.EINVAL
    finally:
        U.uspg_server_destroy(srv)
    assert res[j_big][0]["status"] == U.ENOMEM
    assert res[j_bad][0]["status"] == U.EINVAL
    r, img = res[j_small]
    assert r["status"] == U.OK
    assert rel_l2(img, ref) < 1e-5
    assert st["failed"] == 2 and st["completed"] == 1
    assert st["device_bytes"] <= 4 << 20
