"""Piecewise-steady flow on the GPU (Methods, "MODPATH": the time-step loop
swaps the flow arrays at each step's end): one request, one launch per flow
period, against the oracle's period driver.  FP64: cell sequences,
statuses, steps, exit faces bit-exact, positions and times within 1e-10;
timeseries across the period ends likewise."""
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
def small(ctx):
    f = I.random_box_field(3, 7, 10, seed=51, lnk_var=1.0, n_wells=1)
    fs = I.period_fields(f, seed=6, head_scale=(1.0, 0.4, -0.7), new_wells=(0, 2, 1), well_scale=3.0)
    fhs = [ctx.field(g) for g in fs]
    cells, frac = I.explicit_particles(f, 3000, seed=12, cols=(1, 4))
    st0 = O.release_explicit(f, cells, frac)
    full = O.track(f, st0, arith="mirror")
    T = np.quantile(full["t"], [0.25, 0.6])
    yield f, fs, fhs, cells, frac, st0, full, T
    for fh in fhs:
        mp.mp_field_free(fh)


def _run(ctx, fhs, T, cells, frac, t0=None, **kw):
    if kw.get("times") is not None:
        kw.setdefault("mode", mp.MODE_ENDPOINT | mp.MODE_TIMESERIES)
    gh = mp.mp_release_group(ctx.h, fhs[0], cell=cells, local=frac, t0=t0)
    req = ctx.track_periods(gh, fhs, T, **kw)
    req.wait()
    ep = req.endpoints()
    ts = req.timeseries() if req.n_times else None
    st = req.stats()
    req.free()
    mp.mp_group_free(gh)
    return ep, ts, st


@pytest.mark.parametrize("schedule,pass_sinks,wsf", [(mp.SCHED_STATIC, False, 0.0), (mp.SCHED_DYNAMIC, False, 0.0),
                                                      (mp.SCHED_DYNAMIC, True, 0.0), (mp.SCHED_STATIC, True, 0.3)])
def test_periods_fp64_vs_oracle(ctx, small, schedule, pass_sinks, wsf):
    """Flow periods (and weak sinks, passed or with a threshold: each
    period's field has its own sink fractions) against the oracle."""
    f, fs, fhs, cells, frac, st0, full, T = small
    times = np.sort(np.concatenate([np.quantile(full["t"], [0.02, 0.1, 0.4, 0.8, 0.97]) * 1.01, T]))
    flags = mp.TRACK_PASS_WEAK_SINKS if pass_sinks else 0
    ref = O.track_periods(fs, T, st0, times=times, pass_weak_sinks=pass_sinks, weak_sink_fraction=wsf, arith="mirror")
    ep, ts, st = _run(ctx, fhs, T, cells, frac, times=times, schedule=schedule, flags=flags, weak_sink_fraction=wsf)
    G.compare_fp64(ep, ref, dmin=G.dmin(f))
    G.compare_timeseries_fp64(ts, ref, dmin=G.dmin(f))
    assert st["n_status"] == np.bincount(ref["status"], minlength=8).tolist()
    assert st["cell_steps"] == int(ref["steps"].astype(np.int64).sum())
    assert st["device_error"] == 0
    # the reversed last period sends particles back west
    assert np.any((ref["t"] > T[1]) & (ref["status"] == O.ST_BOUNDARY))


def test_periods_with_stop_time_and_step_cap(ctx, small):
    f, fs, fhs, cells, frac, st0, full, T = small
    for t_stop, max_steps in ((0.5 * (T[0] + T[1]), 0), (np.inf, 9)):
        ref = O.track_periods(fs, T, st0, t_stop=t_stop, max_steps=max_steps, arith="mirror")
        ep, _, st = _run(ctx, fhs, T, cells, frac, t_stop=t_stop, max_steps=max_steps)
        G.compare_fp64(ep, ref, dmin=G.dmin(f))
        assert st["n_status"] == np.bincount(ref["status"], minlength=8).tolist()


def test_identical_periods_equal_steady(ctx, small):
    f, fs, fhs, cells, frac, st0, full, T = small
    times = np.quantile(full["t"], [0.1, 0.5, 0.9])
    ep, ts, st = _run(ctx, [fhs[0]] * 3, T, cells, frac, times=times)
    ep1, ts1, st1 = G.gpu_run(ctx, fhs[0], cells=cells, frac=frac, times=times)
    for k in ("hash", "status", "cell", "exit_face"):
        assert np.array_equal(ep[k], ep1[k]), k
    np.testing.assert_allclose(ep["t"], ep1["t"], rtol=1e-12)
    pauses = sum((ep1["t"] > Tp) for Tp in T)
    assert np.array_equal(ep["steps"].astype(np.int64), ep1["steps"].astype(np.int64) + pauses)
    assert st["n_status"] == st1["n_status"]
    assert np.array_equal(ts["cell"], ts1["cell"]) and np.array_equal(ts["status"], ts1["status"])


def test_periods_update_group_then_continue(ctx, small):
    f, fs, fhs, cells, frac, st0, full, T = small
    t1 = float(T[1] + 0.3 * (T[1] - T[0]))
    gh = mp.mp_release_group(ctx.h, fhs[0], cell=cells, local=frac)
    r1 = ctx.track_periods(gh, fhs, T, t_stop=t1, flags=mp.TRACK_UPDATE_GROUP)
    r1.wait()
    # the group now sits in the last period's field: continue there
    r2 = ctx.track(gh)
    r2.wait()
    a = O.track_periods(fs, T, st0, t_stop=t1, arith="mirror")
    b = O.track(fs[-1], O.resume_state(a), arith="mirror")
    G.compare_fp64(r2.endpoints(), b, dmin=G.dmin(f))
    for r in (r1, r2):
        r.free()
    mp.mp_group_free(gh)


def test_periods_mixed(ctx, small):
    f, fs, fhs, cells, frac, st0, full, T = small
    ref = O.track_periods(fs, T, st0, arith="mirror")
    ep, _, st = _run(ctx, fhs, T, cells, frac, precision=mp.PREC_MIXED)
    same = ep["hash"] == ref["hash"]
    assert np.array_equal(ep["status"][same], ref["status"][same])
    G.check_mixed(ep, field=f, state=st0, label="flow periods",
                  oracle_run=lambda **jk: O.track_periods(fs, T, st0, **jk))
    assert sum(st["n_status"]) == len(cells)


def test_periods_argument_errors(ctx, small):
    f, fs, fhs, cells, frac, st0, full, T = small
    other = ctx.field(I.random_box_field(3, 7, 11, seed=51))
    gh = mp.mp_release_group(ctx.h, fhs[0], cell=cells[:10], local=frac[:10])
    with pytest.raises(mp.MPError) as e:
        mp.mp_track_periods(ctx.h, gh, [fhs[0], other], [1.0], mp.make_opts())
    assert e.value.code == mp.ERR_SHAPE
    with pytest.raises(mp.MPError) as e:
        mp.mp_track_periods(ctx.h, gh, fhs, [2.0, 1.0], mp.make_opts())
    assert e.value.code == mp.ERR_INVALID_ARG
    with pytest.raises(mp.MPError) as e:
        mp.mp_group_set_field(gh, other)
    assert e.value.code == mp.ERR_SHAPE
    mp.mp_group_set_field(gh, fhs[1])
    mp.mp_group_free(gh)
    mp.mp_field_free(other)


def test_periods_cfg2_sampled(ctx):
    """Three flow periods on the 200x200x20 field (the gradient halved, then
    reversed, two wells switched on), 2e5 particles; FP64 against the oracle
    on a 3000-particle sample."""
    w = I.workload("cfg2")
    fs = I.period_fields(w.field, seed=8, head_scale=(1.0, 0.5, -0.5), new_wells=(0, 2, 0), tol_abs=1e-13)
    fhs = [ctx.field(g) for g in fs]
    n = 200_000
    rel = I.Release(n, w.release.lo, w.release.hi, w.release.seed)
    T = [0.3 * w.t_adv, 0.8 * w.t_adv]
    times = w.times[::5]
    gh = mp.mp_release_group(ctx.h, fhs[0], n=n, lo=rel.lo, hi=rel.hi, seed=rel.seed)
    req = ctx.track_periods(gh, fhs, T, times=times, mode=mp.MODE_ENDPOINT | mp.MODE_TIMESERIES)
    req.wait()
    ep, ts, st = req.endpoints(), req.timeseries(), req.stats()
    assert st["device_error"] == 0 and sum(st["n_status"]) == n
    idx = np.sort(np.random.default_rng(3).choice(n, 3000, replace=False))
    s0 = O.subset(O.release_box(w.field, n, rel.lo, rel.hi, rel.seed), idx)
    ref = O.track_periods(fs, T, s0, times=times, arith="mirror")
    ndiv = G.compare_fp64(ep, ref, idx=idx, dmin=G.dmin(w.field), allow_divergent=0.002)
    keep = ep["hash"][idx] == ref["hash"]
    G.compare_timeseries_fp64(ts, ref, idx=idx, dmin=G.dmin(w.field), keep=keep)
    print(f"cfg2 periods: {st['cell_steps']:.3e} cell-steps in {st['kernel_ms']:.1f} ms; statuses {st['n_status']}; "
          f"{ndiv} of 3000 sampled sequences differ")
    req.free()
    mp.mp_group_free(gh)
    for fh in fhs:
        mp.mp_field_free(fh)


@pytest.mark.parametrize("with_periods", [False, True])
def test_staged_release_fp64(ctx, small, with_periods):
    """Staged injection (TC2: particles released from the top face of a few
    cells in stages at a fixed interval), steady or through the periods."""
    f, fs, fhs, cells, frac, st0, full, T = small
    top = np.nonzero(f.ibound.reshape(-1)[:f.nrow * f.ncol] == 1)[0]
    src = [c for c in top if (c % f.ncol) in (1, 2, 3) and all(g.ibound.reshape(-1)[c] == 1 for g in fs)][:4]
    cell, fr, t0 = I.staged_release(f, src, 50, 10, interval=float(T[1]) / 6, seed=7)
    st = O.release_explicit(f, cell, fr)
    st["t"] = t0
    times = np.linspace(0.0, 2.0 * T[1], 9)
    if with_periods:
        ref = O.track_periods(fs, T, st, times=times, arith="mirror")
        ep, ts, stats = _run(ctx, fhs, T, cell, fr, times=times, t0=t0)
    else:
        ref = O.track(f, st, times=times, arith="mirror")
        ep, ts, stats = G.gpu_run(ctx, fhs[0], cells=cell, frac=fr, t0=t0, times=times)
    G.compare_fp64(ep, ref, dmin=G.dmin(f))
    G.compare_timeseries_fp64(ts, ref, dmin=G.dmin(f))
    assert stats["n_status"] == np.bincount(ref["status"], minlength=8).tolist()
