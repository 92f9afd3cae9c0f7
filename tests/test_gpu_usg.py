"""Rectangular unstructured (quadtree) grids on the GPU against the oracle:
FP64 cell sequences, statuses, steps and exit faces bit-exact with its
mirror arithmetic and equal (near-ties apart) with its plain arithmetic,
positions and times within 1e-10; a rectilinear grid written as an
unstructured one gives the rectilinear GPU path's results bit for bit."""
import numpy as np
import pytest

import oracle as O
from paper_2302_13590_gb300 import inputs as I
from paper_2302_13590_gb300 import mp
from paper_2302_13590_gb300.inputs import usg as U
from tests import gpu_common as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch  # noqa: F401
    c = mp.Context(0)
    yield c
    c.close()


def _dmin(u):
    return u.extent


def _run(ctx, fh, cells, frac, t0=None, **kw):
    if kw.get("times") is not None:
        kw.setdefault("mode", mp.MODE_ENDPOINT | mp.MODE_TIMESERIES)
    gh = mp.mp_release_group(ctx.h, fh, cell=cells, local=frac, t0=t0)
    req = ctx.track(gh, **kw)
    req.wait()
    ep, st = req.endpoints(), req.stats()
    ts = req.timeseries() if req.n_times else None
    path = req.pathlines() if (kw.get("mode", 0) & mp.MODE_PATHLINE) else None
    req.free()
    mp.mp_group_free(gh)
    return ep, ts, st, path


def test_structured_as_unstructured_equals_rectilinear_path(ctx):
    f = I.random_box_field(4, 9, 12, seed=303, lnk_var=2.0, n_wells=2, n_inactive=3)
    u = U.from_structured(f)
    fs, fu = ctx.field(f), ctx.field(u)
    cells, frac = I.explicit_particles(f, 2000, seed=4, cols=(1, 6))
    full = O.track(f, O.release_explicit(f, cells, frac), arith="mirror")
    times = np.quantile(full["t"], [0.05, 0.5, 0.95])
    for sched in (mp.SCHED_STATIC, mp.SCHED_DYNAMIC):
        a = _run(ctx, fs, cells, frac, times=times, schedule=sched,
                 mode=mp.MODE_ENDPOINT | mp.MODE_TIMESERIES | mp.MODE_PATHLINE, path_capacity=400 * cells.size)
        b = _run(ctx, fu, cells, frac, times=times, schedule=sched,
                 mode=mp.MODE_ENDPOINT | mp.MODE_TIMESERIES | mp.MODE_PATHLINE, path_capacity=400 * cells.size)
        for k in a[0]:
            assert np.array_equal(a[0][k], b[0][k], equal_nan=True), k
        assert np.array_equal(a[1], b[1])
        pa, pb = (np.sort(x, order=["particle", "seq"]) for x in (a[3], b[3]))
        assert pa.tobytes() == pb.tobytes()
    mp.mp_field_free(fs)
    mp.mp_field_free(fu)


@pytest.mark.parametrize("seed,n,schedule,pass_sinks", [(5, 3000, mp.SCHED_DYNAMIC, False),
                                                        (6, 1, mp.SCHED_STATIC, False),
                                                        (7, 4099, mp.SCHED_STATIC, True)])
def test_quadtree_fp64_vs_oracle(ctx, seed, n, schedule, pass_sinks):
    u = U.quadtree_field(3, 12, 16, seed=seed, n_wells=3)
    fh = ctx.field(u)
    cells, frac = U.explicit_particles(u, n, seed=seed)
    st0 = O.release_explicit(u, cells, frac)
    full = O.track(u, st0, pass_weak_sinks=pass_sinks, arith="mirror")
    times = np.quantile(full["t"], [0.0, 0.2, 0.6, 0.99]) * 1.01
    flags = mp.TRACK_PASS_WEAK_SINKS if pass_sinks else 0
    ref = O.track(u, st0, times=times, pathline=True, pass_weak_sinks=pass_sinks, arith="mirror")
    ep, ts, st, path = _run(ctx, fh, cells, frac, times=times, schedule=schedule, flags=flags,
                            mode=mp.MODE_ENDPOINT | mp.MODE_TIMESERIES | mp.MODE_PATHLINE, path_capacity=200 * n)
    G.compare_fp64(ep, ref, dmin=_dmin(u))
    G.compare_timeseries_fp64(ts, ref, dmin=_dmin(u))
    assert st["n_status"] == np.bincount(ref["status"], minlength=8).tolist()
    # against the plain arithmetic (the reference)
    plain = O.track(u, st0, times=times, pass_weak_sinks=pass_sinks)
    G.compare_fp64_plain(ep, plain, field=u, state=st0, ts=ts, times=times, pass_weak_sinks=pass_sinks,
                         label=f"quadtree {seed}")
    assert st["cell_steps"] == int(ref["steps"].astype(np.int64).sum())
    g, r = (np.sort(x, order=["particle", "seq"]) for x in (path, ref["path"]))
    assert g.size == r.size
    for k in ("particle", "cell", "seq", "status"):
        assert np.array_equal(g[k], r[k]), k
    for k in ("x", "y", "z", "t"):
        assert np.max(G.rel_err(g[k], r[k], scale=np.maximum(np.abs(r[k]), max(u.extent)))) <= 1e-10, k
    mp.mp_field_free(fh)


def test_quadtree_periods_and_resume(ctx):
    base = I.random_box_field(3, 8, 10, seed=52, lnk_var=1.0, n_wells=1)
    fs = I.period_fields(base, seed=4)
    us = [U.from_structured(g) for g in fs]
    fhs = [ctx.field(x) for x in us]
    cells, frac = I.explicit_particles(base, 1500, seed=9, cols=(1, 4))
    st0 = O.release_explicit(us[0], cells, frac)
    full = O.track(us[0], st0, arith="mirror")
    T = np.quantile(full["t"], [0.3, 0.6])
    ref = O.track_periods(us, T, st0, arith="mirror")
    gh = mp.mp_release_group(ctx.h, fhs[0], cell=cells, local=frac)
    req = ctx.track_periods(gh, fhs, T, flags=mp.TRACK_UPDATE_GROUP, t_stop=float(T[1] * 1.2))
    req.wait()
    a = O.track_periods(us, T, st0, t_stop=float(T[1] * 1.2), arith="mirror")
    G.compare_fp64(req.endpoints(), a, dmin=_dmin(us[0]))
    r2 = ctx.track(gh)
    r2.wait()
    G.compare_fp64(r2.endpoints(), O.track(us[-1], O.resume_state(a), arith="mirror"), dmin=_dmin(us[0]))
    del ref
    for r in (req, r2):
        r.free()
    mp.mp_group_free(gh)
    for fh in fhs:
        mp.mp_field_free(fh)


def test_hand_over_moved_point_vs_oracle(ctx):
    """A refined face whose sub-faces carry opposite flows (the hand-made
    two-cell case of the oracle tests): particles reaching the face where
    its flow runs back enter the other sub-face's cell at the moved point;
    the GPU's cells, faces, times and every pathline point equal the
    oracle's."""
    from tests.test_oracle_usg import _two_cells
    for q_lo, q_hi in ((1e-4, 3e-4), (-1e-4, 5e-4), (4e-4, -1e-4)):
        u = _two_cells(q_lo, q_hi)
        fh = ctx.field(u)
        rng = np.random.default_rng(21)
        frac = np.column_stack([rng.uniform(0.02, 0.3, 97), rng.uniform(0.02, 0.98, 97), rng.uniform(0.1, 0.9, 97)])
        cells = np.zeros(97, np.int32)
        ref = O.track(u, O.release_explicit(u, cells, frac), pathline=True, arith="mirror")
        ep, _, st, path = _run(ctx, fh, cells, frac, mode=mp.MODE_ENDPOINT | mp.MODE_PATHLINE, path_capacity=20 * 97)
        G.compare_fp64(ep, ref, dmin=_dmin(u))
        g, r = (np.sort(x, order=["particle", "seq"]) for x in (path, ref["path"]))
        assert g.tobytes() == r.tobytes()
        if q_lo < 0:
            assert (ref["cell"] == 2).all()          # every particle crosses into the northern cell
        mp.mp_field_free(fh)


def test_quadtree_weak_sink_fraction_vs_oracle(ctx):
    """Weak sinks with a threshold on a quadtree (sink fractions from the
    faces' total flows): FP64 bit-exact against the oracle below, between
    and above the wells' fractions."""
    from tests.test_oracle_weak_sinks import _fractions_usg
    u = U.quadtree_field(2, 8, 12, seed=15, n_wells=3, well_rate=0.05)
    fh = ctx.field(u)
    fs = np.sort(_fractions_usg(u)[u.ibound == U.IB_SINK])
    cells, frac = U.explicit_particles(u, 2000, seed=6)
    st0 = O.release_explicit(u, cells, frac)
    for thr in [fs[0] / 2] + list((fs[:-1] + fs[1:]) / 2) + [(fs[-1] + 1) / 2]:
        ref = O.track(u, st0, pass_weak_sinks=True, weak_sink_fraction=thr, pathline=True, arith="mirror")
        ep, _, st, path = _run(ctx, fh, cells, frac, flags=mp.TRACK_PASS_WEAK_SINKS, weak_sink_fraction=thr,
                               mode=mp.MODE_ENDPOINT | mp.MODE_PATHLINE, path_capacity=200 * cells.size)
        G.compare_fp64(ep, ref, dmin=_dmin(u))
        g, r = (np.sort(x, order=["particle", "seq"]) for x in (path, ref["path"]))
        assert np.array_equal(g[["particle", "cell", "seq", "status"]], r[["particle", "cell", "seq", "status"]])
    mp.mp_field_free(fh)


def test_quadtree_balance_report(ctx):
    """The quadtree field's volume-balance report equals the sums made here
    from the face totals (sub-faces summed in list order)."""
    from tests.test_gpu_parity import _balance_np
    u = U.quadtree_field(2, 8, 12, seed=15, n_wells=3, well_rate=0.05)
    fh = ctx.field(u)
    q6 = np.zeros((u.ncell, 6))
    for c in range(u.ncell):
        for fi in range(6):
            sl = u.subfaces(c, fi)
            acc = 0.0
            for e in range(sl.start, sl.stop):
                acc = float(u.q[e]) if e == sl.start else acc + float(u.q[e])
            q6[c, fi] = acc
    assert mp.mp_field_balance(fh) == _balance_np(q6, np.asarray(u.ibound))
    mp.mp_field_free(fh)


def test_usg_rejections(ctx):
    u = U.quadtree_field(2, 6, 8, seed=3, n_wells=1)
    fh = ctx.field(u)
    with pytest.raises(mp.MPError):
        mp.mp_release_group(ctx.h, fh, n=10, lo=(0, 0, 0), hi=(1, 1, 1), seed=1)
    cells, frac = U.explicit_particles(u, 10, seed=1)
    gh = mp.mp_release_group(ctx.h, fh, cell=cells, local=frac)
    with pytest.raises(mp.MPError):
        ctx.track(gh, precision=mp.PREC_MIXED)
    bad = U.UsgField(u.box, u.porosity, u.ibound, u.face_off, np.where(u.nbr >= 0, u.nbr + u.ncell, -1).astype(
        np.int32), u.q, u.rect)
    with pytest.raises(mp.MPError) as e:
        ctx.field(bad)
    assert e.value.code == mp.ERR_SHAPE
    mp.mp_group_free(gh)
    mp.mp_field_free(fh)


def test_quadtree_larger_sampled(ctx):
    """A 40 x 60 x 4 base grid with 15 % of the columns and the wells'
    neighbourhoods refined; 2e5 particles; FP64 against the oracle on 2000."""
    u = U.quadtree_field(4, 40, 60, seed=11, n_wells=6, refine_frac=0.15)
    fh = ctx.field(u)
    n = 200_000
    cells, frac = U.explicit_particles(u, n, seed=12)
    gh = mp.mp_release_group(ctx.h, fh, cell=cells, local=frac)
    req = ctx.track(gh)
    req.wait()
    ep, st = req.endpoints(), req.stats()
    assert st["device_error"] == 0 and sum(st["n_status"]) == n
    idx = np.sort(np.random.default_rng(1).choice(n, 2000, replace=False))
    ref = O.track(u, O.release_explicit(u, cells[idx], frac[idx]), arith="mirror")
    G.compare_fp64(ep, ref, idx=idx, dmin=_dmin(u))
    print(f"quadtree {u.ncell} cells: {st['cell_steps']:.3e} cell-steps in {st['kernel_ms']:.2f} ms = "
          f"{st['cell_steps'] / st['kernel_ms'] * 1e3:.3e}/s")
    req.free()
    mp.mp_group_free(gh)
    mp.mp_field_free(fh)
