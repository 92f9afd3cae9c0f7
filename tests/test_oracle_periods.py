"""Piecewise-steady flow on the oracle (Methods, "MODPATH": the outer loop
runs over the flow model's time steps and swaps the flow arrays at each
step's end time).

Pins that do not come from the oracle itself:
* identical fields in every period reproduce the steady run (same cell
  sequence and exit face, times to rounding, one extra step per pause);
* a reversed field for the same duration brings every particle that was
  still moving back to its start (the piecewise-linear flow is reversible);
* brute-force RK4 integration with the field switched at the period ends;
* a particle whose cell turns inactive, constant-head or sink at a period
  end stops there without a step.
"""
import numpy as np
import pytest

import oracle as O
from paper_2302_13590_gb300 import inputs as I
from tests import helpers as H

# every pin holds for both arithmetic modes of the oracle
pytestmark = pytest.mark.usefixtures("oracle_arith")


@pytest.fixture
def base(oracle_arith):
    # per test: the reference run depends on the oracle's arithmetic mode
    f = I.random_box_field(2, 5, 8, seed=40, lnk_var=0.5, n_wells=1)
    cells, frac = I.explicit_particles(f, 120, seed=9, cols=(1, 3))
    st0 = O.release_explicit(f, cells, frac)
    full = O.track(f, st0)
    return f, cells, frac, st0, full


def _kij(f, c):
    return c // (f.ncol * f.nrow), (c // f.ncol) % f.nrow, c % f.ncol


def test_identical_periods_equal_steady(base):
    f, cells, frac, st0, full = base
    T = np.quantile(full["t"], [0.15, 0.4, 0.7])
    times = np.quantile(full["t"], [0.05, 0.15, 0.3, 0.5, 0.9]) * 1.003
    times = np.sort(np.concatenate([times, T[:1]]))  # an output time exactly at a period end
    steady = O.track(f, st0, times=times)
    r = O.track_periods([f] * 4, T, st0, times=times)
    for k in ("hash", "exit_face", "status", "cell"):
        assert np.array_equal(r[k], steady[k]), k
    np.testing.assert_allclose(r["t"], steady["t"], rtol=1e-12)
    ext = max(f.delr.sum(), f.delc.sum(), f.dz.sum())
    for k in ("gx", "gy", "gz"):
        np.testing.assert_allclose(r[k], steady[k], rtol=0, atol=1e-12 * ext)
    # a particle pays one partial step for every period end it is still moving at
    pauses = sum((steady["t"] > Tp) for Tp in T)
    assert np.array_equal(r["steps"], steady["steps"] + pauses)
    for k in ("ts_x", "ts_y", "ts_z"):
        np.testing.assert_allclose(r[k], steady[k], rtol=0, atol=1e-12 * ext)
    assert np.array_equal(r["ts_cell"], steady["ts_cell"])
    assert np.array_equal(r["ts_status"], steady["ts_status"])


def test_reversed_period_returns_to_start(base):
    f, cells, frac, st0, full = base
    T = float(np.quantile(full["t"], 0.3))
    back = H.reversed_flow(f)
    r = O.track_periods([f, back], [T], st0, t_stop=2 * T)
    fwd = O.track(f, st0, t_stop=T)
    moving = fwd["status"] == O.ST_TIME
    assert moving.sum() > 50
    assert np.all(r["status"][moving] == O.ST_TIME)
    assert np.array_equal(r["cell"][moving], st0["cell"][moving])
    for k in ("px", "py", "pz"):
        np.testing.assert_allclose(r[k][moving], st0[k][moving], rtol=0, atol=1e-9)
    np.testing.assert_allclose(r["t"][moving], 2 * T, rtol=1e-15)


@pytest.mark.parametrize("pass_sinks", [False, True])
def test_periods_against_rk4(base, pass_sinks):
    f, cells, frac, st0, full = base
    fs = I.period_fields(f, seed=5, head_scale=(1.0, 0.5, -0.6), new_wells=(0, 2, 0))
    T = np.quantile(full["t"], [0.2, 0.5])
    r = O.track_periods(fs, T, st0, pass_weak_sinks=pass_sinks)
    seen = set()
    for q in range(0, len(cells), 3):
        k, i, j = _kij(f, int(cells[q]))
        p0 = [st0["px"][q], st0["py"][q], st0["pz"][q]]
        status, seq, _, p, t = H.rk4_track(f, k, i, j, p0, periods=(fs, T), pass_sinks=pass_sinks,
                                           capture_time=50 * float(np.max(full["t"])))
        assert status == r["status"][q], q
        assert H.fnv_hash(seq) == int(r["hash"][q]), q
        assert r["t"][q] == pytest.approx(t, rel=1e-7)
        seen.add(status)
    # every period matters: some particles leave west after the reversal
    assert O.ST_BOUNDARY in seen
    assert np.any((r["t"] > T[1]) & (r["status"] == O.ST_BOUNDARY))


def test_cell_class_change_at_period_end(base):
    f, cells, frac, st0, full = base
    T = float(np.quantile(full["t"], 0.3))
    a = O.track(f, st0, t_stop=T)
    q = int(np.nonzero(a["status"] == O.ST_TIME)[0][0])
    c = int(a["cell"][q])
    for ib, expect, flag in ((0, O.ST_BOUNDARY, False), (-1, O.ST_BOUNDARY, False), (2, O.ST_SINK, False)):
        g = H.SimpleField(f.nlay, f.nrow, f.ncol, f.delr, f.delc, f.dz, f.origin, f.qx, f.qy, f.qz, f.porosity,
                          f.ibound.copy())
        g.ibound.reshape(-1)[c] = ib
        r = O.track_periods([f, g], [T], st0, pass_weak_sinks=flag)
        assert r["status"][q] == expect
        assert r["cell"][q] == c and r["steps"][q] == a["steps"][q]
        assert r["t"][q] == T
    # passing weak sinks, the particle keeps moving out of the new sink cell
    g.ibound.reshape(-1)[c] = 2
    r = O.track_periods([f, g], [T], st0, pass_weak_sinks=True)
    assert r["steps"][q] > a["steps"][q]


def test_period_driver_rejects_bad_ends(base):
    f, cells, frac, st0, full = base
    with pytest.raises(ValueError):
        O.track_periods([f, f], [], st0)
    with pytest.raises(ValueError):
        O.track_periods([f, f, f], [2.0, 1.0], st0)


def test_staged_release_is_a_time_translation(base):
    """Staged injection (TC2) in steady flow: a particle released at t0
    follows the path of the same particle released at 0, shifted by t0;
    output times before t0 see the release position."""
    f, cells, frac, st0, full = base
    t0 = np.linspace(0.0, 3.0, cells.size) * float(np.median(full["t"]))
    st = dict(st0, t=t0)
    r = O.track(f, st)
    for k in ("hash", "steps", "status", "cell", "exit_face", "px", "py", "pz"):
        assert np.array_equal(r[k], full[k]), k
    np.testing.assert_allclose(r["t"] - t0, full["t"], rtol=1e-12)
    tau = np.quantile(full["t"], [0.1, 0.5])
    q = int(np.argmax(t0))
    times = np.sort(np.concatenate([tau, t0[q] + tau, [0.5 * t0[q]]]))
    rs = O.track(f, {k: v[q:q + 1] for k, v in st.items()}, times=times)
    r0 = O.track(f, {k: v[q:q + 1] for k, v in st0.items()}, times=tau)
    before = times < t0[q]
    assert np.all(rs["ts_status"][before, 0] == O.ST_ACTIVE)
    c = int(st0["cell"][q])
    k0, i0, j0 = _kij(f, c)
    x0 = float(np.sum(f.delr[:j0]) + f.origin[0] + st0["px"][q])
    assert np.all(rs["ts_x"][before, 0] == x0)
    after = np.nonzero(~before)[0][-2:]
    for k in ("ts_x", "ts_y", "ts_z"):
        np.testing.assert_allclose(rs[k][after, 0], r0[k][:, 0], rtol=1e-11)


def test_staged_release_through_periods_against_rk4(base):
    f, cells, frac, st0, full = base
    fs = I.period_fields(f, seed=5, head_scale=(1.0, 0.5, -0.6), new_wells=(0, 2, 0))
    T = np.quantile(full["t"], [0.2, 0.5])
    top = np.nonzero(f.ibound.reshape(-1)[:f.nrow * f.ncol] == 1)[0]
    src = [c for c in top if (c % f.ncol) in (1, 2) and all(g.ibound.reshape(-1)[c] == 1 for g in fs)][:4]
    cell, fr, t0 = I.staged_release(f, src, 3, 5, interval=float(T[1]) / 3, seed=4)
    st = O.release_explicit(f, cell, fr)
    st["t"] = t0
    r = O.track_periods(fs, T, st)
    for q in range(cell.size):
        k, i, j = _kij(f, int(cell[q]))
        status, seq, _, p, t = H.rk4_track(f, k, i, j, [st["px"][q], st["py"][q], st["pz"][q]],
                                           periods=(fs, T), t0=float(t0[q]))
        assert status == r["status"][q], q
        assert H.fnv_hash(seq) == int(r["hash"][q]), q
        assert r["t"][q] == pytest.approx(t, rel=1e-7)
    # stages released into the reversed last period leave west, the first stage east
    col = r["cell"] % f.ncol
    assert np.all(col[t0 > T[1]] < f.ncol // 2)
    assert np.any(col[t0 < T[0]] >= f.ncol // 2)
