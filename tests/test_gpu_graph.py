"""Captured batches (CUDA graphs): a graph replay gives the same results as
releasing and tracking the same requests through mp_release_group and
mp_track_batch; replays repeat, new release descriptors take effect, and
the graph's requests are read like any others."""
import time

import numpy as np
import pytest

from paper_2302_13590_gb300 import inputs as I
from paper_2302_13590_gb300 import mp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    ctx = mp.Context(0)
    w = I.workload("cfg2")
    fh = ctx.field(w.field)
    yield torch, ctx, w, fh
    ctx.close()


def _specs(w, n_req, seed, n_lo=100, n_hi=20000):
    rng = np.random.default_rng(seed)
    Lx, Ly, Lz = w.field.extent
    rels, opts = [], []
    for i in range(n_req):
        n = int(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        lo = rng.uniform(0, 1, 3) * np.array([0.3 * Lx, Ly, Lz]) * 0.5
        hi = lo + rng.uniform(0.05, 0.5, 3) * np.array([0.3 * Lx, Ly, Lz])
        rels.append(I.Release(n, tuple(lo), tuple(np.minimum(hi, [Lx, Ly, Lz])), seed=1000 + i, id_offset=7 * i))
        ts = i % 3 == 1
        prec = mp.PREC_MIXED if i % 2 else mp.PREC_FP64
        mode = mp.MODE_ENDPOINT | (mp.MODE_TIMESERIES if ts else 0) | (mp.MODE_PATHLINE if i % 5 == 4 else 0)
        # room for every point (paths here average ~270 cell-steps): with
        # overflow, which points are kept depends on the warps' timing
        opts.append(mp.make_opts(mode=mode, precision=prec, times=w.times[::10] if ts else None,
                                 path_capacity=2000 * n if mode & mp.MODE_PATHLINE else 0))
    return rels, opts


def _direct(ctx, fh, rels, opts):
    groups = [mp.mp_release_group(ctx.h, fh, n=r.n, lo=r.lo, hi=r.hi, seed=r.seed, id_offset=r.id_offset)
              for r in rels]
    ids = mp.mp_track_batch(ctx.h, groups, opts)
    out = [_read(ctx, rid, r.n, o) for rid, r, o in zip(ids, rels, opts)]
    for rid in ids:
        mp.mp_req_free(ctx.h, rid)
    for g in groups:
        mp.mp_group_free(g)
    return out


def _read(ctx, rid, n, o):
    mp.mp_wait(ctx.h, rid)
    res = {"ep": mp.mp_get_endpoints(ctx.h, rid, n), "st": mp.mp_get_stats(ctx.h, rid)}
    if o.mode & mp.MODE_TIMESERIES:
        res["ts"] = mp.mp_get_timeseries(ctx.h, rid, n, o.n_times)
    if o.mode & mp.MODE_PATHLINE:
        p = mp.mp_get_pathlines(ctx.h, rid)
        res["path"] = np.sort(p, order=["particle", "seq"])
    return res


def _same(a, b):
    for k in a["ep"]:
        assert np.array_equal(a["ep"][k], b["ep"][k], equal_nan=True), k
    assert a["st"]["cell_steps"] == b["st"]["cell_steps"] and a["st"]["n_status"] == b["st"]["n_status"]
    for k in ("ts", "path"):
        if k in a:
            assert np.array_equal(a[k], b[k]), k


def test_graph_equals_direct_batch(setup):
    torch, ctx, w, fh = setup
    rels, opts = _specs(w, 12, seed=3)
    ref = _direct(ctx, fh, rels, opts)
    s = torch.cuda.Stream()
    g, ids = mp.mp_graph_create(ctx.h, fh, rels, opts, stream=s)
    for rep in range(2):   # a replay repeats the same results
        mp.mp_graph_launch(g, stream=s)
        for rid, r, o, want in zip(ids, rels, opts, ref):
            _same(_read(ctx, rid, r.n, o), want)
    with pytest.raises(mp.MPError):
        mp.mp_req_free(ctx.h, ids[0])
    # new descriptors: the same as a direct batch with them
    rels2 = [I.Release(r.n, r.lo, r.hi, seed=r.seed + 17, id_offset=r.id_offset + 3) for r in rels]
    for i, r in enumerate(rels2):
        mp.mp_graph_set_release(g, i, r.n, r.lo, r.hi, r.seed, r.id_offset, stream=s)
    with pytest.raises(mp.MPError) as e:
        mp.mp_graph_set_release(g, 0, rels[0].n + 1, rels[0].lo, rels[0].hi)
    assert e.value.code == mp.ERR_SHAPE
    mp.mp_graph_launch(g, stream=s)
    ref2 = _direct(ctx, fh, rels2, opts)
    for rid, r, o, want in zip(ids, rels2, opts, ref2):
        _same(_read(ctx, rid, r.n, o), want)
    mp.mp_graph_free(g)


def test_graph_launch_overhead(setup):
    """Many small requests: one graph launch against the host-side sequence
    (a release per group, the batch table, one tracking launch per
    precision).  Printed, not asserted: the host side differs by machine."""
    torch, ctx, w, fh = setup
    rels, _ = _specs(w, 128, seed=4, n_lo=200, n_hi=2000)
    opts = [mp.make_opts(precision=mp.PREC_MIXED) for _ in rels]
    s = torch.cuda.Stream()
    g, ids = mp.mp_graph_create(ctx.h, fh, rels, opts, stream=s)
    reps = 20

    def direct_once():
        groups = [mp.mp_release_group(ctx.h, fh, n=r.n, lo=r.lo, hi=r.hi, seed=r.seed, stream=s) for r in rels]
        rids = mp.mp_track_batch(ctx.h, groups, opts, s)
        s.synchronize()
        for rid in rids:
            mp.mp_req_free(ctx.h, rid)
        for gg in groups:
            mp.mp_group_free(gg)

    for _ in range(3):
        direct_once()
        mp.mp_graph_launch(g, stream=s)
        s.synchronize()
    t = time.perf_counter()
    for _ in range(reps):
        direct_once()
    t_direct = (time.perf_counter() - t) / reps
    t = time.perf_counter()
    for _ in range(reps):
        mp.mp_graph_launch(g, stream=s)
        s.synchronize()
    t_graph = (time.perf_counter() - t) / reps
    st = mp.mp_get_stats(ctx.h, ids[0])
    assert st["device_error"] == 0
    print(f"128 small requests ({sum(r.n for r in rels)} particles): direct {t_direct * 1e3:.2f} ms, "
          f"graph {t_graph * 1e3:.2f} ms per batch")
    mp.mp_graph_free(g)
