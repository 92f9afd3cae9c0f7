"""Pathline mode on the GPU (Methods, "MODPATH": pathline simulations)
against the oracle.  The GPU appends points in the order its warps produce
them; both sides are sorted by (particle, seq) before comparing.  FP64:
particle, cell, seq and status bit-exact, positions and times within 1e-10."""
import numpy as np
import pytest

import oracle as O
from paper_2302_13590_gb300 import inputs as I
from paper_2302_13590_gb300 import mp
from tests import gpu_common as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch  # noqa: F401
    c = mp.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def fld(ctx):
    f = I.random_box_field(4, 8, 11, seed=71, lnk_var=1.5, n_wells=2, n_inactive=2)
    fh = ctx.field(f)
    yield f, fh
    mp.mp_field_free(fh)


def _sorted(path):
    return path[np.lexsort((path["seq"], path["particle"]))]


def compare_paths(gpu, ref, f, rtol=1e-10):
    g, r = _sorted(gpu), _sorted(ref)
    assert g.size == r.size, (g.size, r.size)
    for k in ("particle", "cell", "seq", "status"):
        assert np.array_equal(g[k], r[k]), k
    ext = G.dmin(f)
    for ax, k in enumerate(("x", "y", "z")):
        e = G.rel_err(g[k], r[k], scale=G.pos_scale(ext[ax], r[k]))
        assert e.max(initial=0.0) <= rtol, k
    e = G.rel_err(g["t"], r["t"], scale=np.maximum(np.abs(r["t"]), 1e-300))
    assert e.max(initial=0.0) <= rtol


def _run(ctx, fh, cells, frac, t0=None, **kw):
    gh = mp.mp_release_group(ctx.h, fh, cell=cells, local=frac, t0=t0)
    req = ctx.track(gh, **kw)
    req.wait()
    ep, st, path = req.endpoints(), req.stats(), req.pathlines()
    ts = req.timeseries() if req.n_times else None
    req.free()
    mp.mp_group_free(gh)
    return ep, ts, st, path


@pytest.mark.parametrize("schedule,with_ts", [(mp.SCHED_STATIC, False), (mp.SCHED_DYNAMIC, False),
                                              (mp.SCHED_DYNAMIC, True), (mp.SCHED_STATIC, True)])
def test_pathlines_fp64(ctx, fld, schedule, with_ts):
    f, fh = fld
    cells, frac = I.explicit_particles(f, 2500, seed=21, cols=(1, 5))
    st0 = O.release_explicit(f, cells, frac)
    full = O.track(f, st0, arith="mirror")
    times = np.quantile(full["t"], [0.1, 0.5, 0.9]) if with_ts else None
    ref = O.track(f, st0, times=times, pathline=True, arith="mirror")
    mode = mp.MODE_ENDPOINT | mp.MODE_PATHLINE | (mp.MODE_TIMESERIES if with_ts else 0)
    ep, ts, st, path = _run(ctx, fh, cells, frac, mode=mode, times=times, schedule=schedule)
    assert st["path_points"] == ref["path"].size == int(ref["steps"].sum()) + cells.size
    compare_paths(path, ref["path"], f)
    G.compare_fp64(ep, ref, dmin=G.dmin(f))
    if with_ts:
        G.compare_timeseries_fp64(ts, ref, dmin=G.dmin(f))


def test_pathlines_stop_time_cap_and_staged_release(ctx, fld):
    f, fh = fld
    cells, frac = I.explicit_particles(f, 700, seed=22, cols=(1, 5))
    st0 = O.release_explicit(f, cells, frac)
    full = O.track(f, st0, arith="mirror")
    t0 = np.where(np.arange(cells.size) % 3 == 0, 0.4 * np.median(full["t"]), 0.0)
    st0["t"] = t0
    for t_stop, max_steps in ((float(np.median(full["t"])), 0), (np.inf, 5)):
        ref = O.track(f, st0, t_stop=t_stop, max_steps=max_steps, pathline=True, arith="mirror")
        ep, _, st, path = _run(ctx, fh, cells, frac, t0=t0, mode=mp.MODE_ENDPOINT | mp.MODE_PATHLINE,
                               t_stop=t_stop, max_steps=max_steps)
        compare_paths(path, ref["path"], f)
        G.compare_fp64(ep, ref, dmin=G.dmin(f))


def test_pathline_capacity_overflow(ctx, fld):
    f, fh = fld
    cells, frac = I.explicit_particles(f, 500, seed=23, cols=(1, 5))
    st0 = O.release_explicit(f, cells, frac)
    ref = _sorted(O.track(f, st0, pathline=True, arith="mirror")["path"])
    cap = ref.size // 3
    _, _, st, path = _run(ctx, fh, cells, frac, mode=mp.MODE_ENDPOINT | mp.MODE_PATHLINE, path_capacity=cap)
    assert st["path_points"] == ref.size and path.size == cap
    # what was kept is a set of genuine points
    key = lambda a: a["particle"].astype(np.int64) * (1 << 32) + a["seq"]
    pos = np.searchsorted(key(ref), key(path))
    assert np.array_equal(key(ref)[pos], key(path))
    assert np.array_equal(ref["cell"][pos], path["cell"]) and np.array_equal(ref["t"][pos], path["t"])


def test_pathlines_in_a_batch(ctx, fld):
    """A batch mixing pathline and endpoint-only requests: points go to their
    own request's array."""
    f, fh = fld
    groups, specs, refs = [], [], []
    for i, n in enumerate((300, 1, 977, 64)):
        cells, frac = I.explicit_particles(f, n, seed=40 + i, cols=(1, 5))
        groups.append(mp.mp_release_group(ctx.h, fh, cell=cells, local=frac))
        pl = i != 1
        specs.append(mp.make_opts(mode=mp.MODE_ENDPOINT | (mp.MODE_PATHLINE if pl else 0)))
        refs.append(O.track(f, O.release_explicit(f, cells, frac), pathline=pl, arith="mirror"))
    ids = mp.mp_track_batch(ctx.h, groups, specs)
    for i, rid in enumerate(ids):
        mp.mp_wait(ctx.h, rid)
        if i != 1:
            compare_paths(mp.mp_get_pathlines(ctx.h, rid), refs[i]["path"], f)
        else:
            assert mp.mp_get_stats(ctx.h, rid)["path_points"] == 0
        mp.mp_req_free(ctx.h, rid)
    for g in groups:
        mp.mp_group_free(g)


def test_pathlines_through_periods(ctx, fld):
    f, fh = fld
    cells, frac = I.explicit_particles(f, 1500, seed=24, cols=(1, 5))
    st0 = O.release_explicit(f, cells, frac)
    full = O.track(f, st0, arith="mirror")
    fs = I.period_fields(f, seed=9, head_scale=(1.0, 0.5, -0.6), new_wells=(0, 1, 0))
    fhs = [fh] + [ctx.field(g) for g in fs[1:]]
    T = np.quantile(full["t"], [0.3, 0.6])
    ref = O.track_periods(fs, T, st0, pathline=True, arith="mirror")
    gh = mp.mp_release_group(ctx.h, fh, cell=cells, local=frac)
    req = ctx.track_periods(gh, fhs, T, mode=mp.MODE_ENDPOINT | mp.MODE_PATHLINE)
    req.wait()
    compare_paths(req.pathlines(), ref["path"], f)
    G.compare_fp64(req.endpoints(), ref, dmin=G.dmin(f))
    req.free()
    mp.mp_group_free(gh)
    for g in fhs[1:]:
        mp.mp_field_free(g)


def test_pathlines_mixed(ctx, fld):
    f, fh = fld
    cells, frac = I.explicit_particles(f, 2000, seed=25, cols=(1, 5))
    st0 = O.release_explicit(f, cells, frac)
    ref = O.track(f, st0, pathline=True, arith="mirror")
    ep, _, st, path = _run(ctx, fh, cells, frac, mode=mp.MODE_ENDPOINT | mp.MODE_PATHLINE,
                           precision=mp.PREC_MIXED)
    same = np.nonzero(ep["hash"] == ref["hash"])[0]
    G.check_mixed(ep, field=f, state=st0, label="pathline run")
    g = _sorted(path[np.isin(path["particle"], same)])
    r = _sorted(ref["path"][np.isin(ref["path"]["particle"], same)])
    assert g.size == r.size
    assert np.array_equal(g["cell"], r["cell"]) and np.array_equal(g["seq"], r["seq"])
    fin = r["t"] > 0
    assert np.median(G.rel_err(g["t"][fin], r["t"][fin])) <= 1e-6
    cw = min(f.delr.min(), f.delc.min(), f.dz.min())
    assert np.quantile(np.abs(g["x"] - r["x"]), 0.99) <= 1e-4 * cw


def test_pathlines_cfg2_sampled(ctx):
    """2e5 particles on the 200x200x20 field (5.5e7 points, 2.6 GB kept on
    the device); the points of 2000 sampled particles are gathered on the
    device and compared with the oracle's."""
    import torch
    w = I.workload("cfg2")
    fh = ctx.field(w.field)
    n = 200_000
    gh = mp.mp_release_group(ctx.h, fh, n=n, lo=w.release.lo, hi=w.release.hi, seed=w.release.seed)
    req = ctx.track(gh, mode=mp.MODE_ENDPOINT | mp.MODE_PATHLINE, path_capacity=400 * n)
    req.wait()
    st = req.stats()
    assert st["device_error"] == 0 and st["path_points"] == st["cell_steps"] + n
    buf = torch.empty((st["path_points"], 12), dtype=torch.int32, device="cuda")
    mp.mp_get_pathlines(ctx.h, req.id, st["path_points"], out=buf, device=True)
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(6).choice(n, 2000, replace=False))
    keep = torch.isin(buf[:, 8], torch.as_tensor(idx, dtype=torch.int32, device="cuda"))
    path = buf[keep].cpu().numpy().view(mp.PATH_RECORD).reshape(-1)
    s0 = O.subset(O.release_box(w.field, n, w.release.lo, w.release.hi, w.release.seed), idx)
    ref = O.track(w.field, s0, pathline=True, arith="mirror")["path"]
    ref["particle"] = idx[ref["particle"]]
    compare_paths(path, ref, w.field)
    print(f"cfg2 pathlines: {st['path_points']:.3e} points, {st['cell_steps']:.3e} cell-steps in "
          f"{st['kernel_ms']:.1f} ms")
    req.free()
    mp.mp_group_free(gh)
    mp.mp_field_free(fh)
