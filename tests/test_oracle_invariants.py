"""Invariants of the exact piecewise-analytic solution, checked on the oracle.

* time additivity: stopping at T1 and continuing to T2 equals going to T2;
* a timeseries record at t_k equals an endpoint run with t_stop = t_k
  (bit-exact: the same step, the same arithmetic);
* reversibility: with every face flow negated, running back for the same
  time returns to the start;
* mirror symmetry across x;
* particle order does not change any particle's result.
"""
import numpy as np
import pytest

import oracle as O
from paper_2302_13590_gb300 import inputs as I
from tests import helpers as H

# every pin holds for both arithmetic modes of the oracle
pytestmark = pytest.mark.usefixtures("oracle_arith")


@pytest.fixture(scope="module")
def fld():
    return I.random_box_field(3, 5, 8, seed=31, lnk_var=1.5, n_wells=1)


@pytest.fixture(scope="module")
def rel(fld):
    cells, frac = I.explicit_particles(fld, 60, seed=3, cols=(1, 4))
    return O.release_explicit(fld, cells, frac)


def test_time_additivity(fld, rel):
    full = O.track(fld, rel)
    T2 = np.median(full["t"])
    T1 = 0.37 * T2
    a = O.track(fld, rel, t_stop=T1)
    mid = dict(cell=a["cell"], px=a["px"], py=a["py"], pz=a["pz"], t=a["t"],
               status=np.where(a["status"] == O.ST_TIME, O.ST_ACTIVE, a["status"]).astype(np.uint8))
    b = O.track(fld, mid, t_stop=T2)
    d = O.track(fld, rel, t_stop=T2)
    assert np.array_equal(b["status"], d["status"])
    assert np.array_equal(b["cell"], d["cell"])
    assert np.array_equal(a["steps"] + b["steps"] - (a["status"] == O.ST_TIME), d["steps"])
    for k in ("gx", "gy", "gz"):
        np.testing.assert_allclose(b[k], d[k], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(b["t"], d["t"], rtol=1e-13)
    # carrying the step count, hash and exit face makes resume == continue
    # for those too: the pause adds one partial step, the hash does not
    # repeat the cell the particle paused in
    c = O.track(fld, O.resume_state(a), t_stop=T2)
    assert np.array_equal(c["hash"], d["hash"])
    assert np.array_equal(c["exit_face"], d["exit_face"])
    assert np.array_equal(c["steps"], d["steps"] + (a["status"] == O.ST_TIME))
    for k in ("gx", "gy", "gz", "t", "status", "cell"):
        assert np.array_equal(c[k], b[k]), k


def test_timeseries_equals_endpoint_at_tk(fld, rel):
    full = O.track(fld, rel)
    times = np.quantile(full["t"], [0.0, 0.1, 0.3, 0.5, 0.9, 1.0]) * np.array([0.0, 1, 1, 1, 1, 1.2])
    ts = O.track(fld, rel, times=times)
    for kk, tk in enumerate(times):
        e = O.track(fld, rel, t_stop=tk)
        live = e["status"] == O.ST_TIME
        assert np.array_equal(ts["ts_x"][kk][live], e["gx"][live])
        assert np.array_equal(ts["ts_y"][kk][live], e["gy"][live])
        assert np.array_equal(ts["ts_z"][kk][live], e["gz"][live])
        assert np.array_equal(ts["ts_cell"][kk][live], e["cell"][live])
        # particles that ended before t_k report their final position and status
        done = ~live
        assert np.array_equal(ts["ts_x"][kk][done], full["gx"][done])
        assert np.array_equal(ts["ts_status"][kk][done], full["status"][done])
    # t_0 = 0: the release position
    assert np.all(ts["ts_status"][0] == O.ST_ACTIVE)


def test_reversibility(fld, rel):
    fwd_full = O.track(fld, rel)
    T = 0.5 * np.min(fwd_full["t"][fwd_full["status"] != O.ST_SINK])
    fwd = O.track(fld, rel, t_stop=T)
    assert np.all(fwd["status"] == O.ST_TIME)
    back_state = dict(cell=fwd["cell"], px=fwd["px"], py=fwd["py"], pz=fwd["pz"],
                      t=np.zeros(len(fwd["cell"])), status=np.zeros(len(fwd["cell"]), np.uint8))
    back = O.track(H.reversed_flow(fld), back_state, t_stop=T)
    assert np.array_equal(back["cell"], rel["cell"])
    for k in ("px", "py", "pz"):
        np.testing.assert_allclose(back[k], rel[k], rtol=1e-9, atol=1e-10)


def test_mirror_symmetry(fld, rel):
    m = H.mirror_x(fld)
    c = rel["cell"]
    j, rest = c % fld.ncol, c // fld.ncol
    mc = (rest * fld.ncol + (fld.ncol - 1 - j)).astype(np.int32)
    mstate = dict(cell=mc, px=fld.delr[j] - rel["px"], py=rel["py"].copy(), pz=rel["pz"].copy(),
                  t=np.zeros(len(c)), status=rel["status"].copy())
    a = O.track(fld, rel)
    b = O.track(m, mstate)
    assert np.array_equal(a["status"], b["status"])
    assert np.array_equal(a["steps"], b["steps"])
    ja = a["cell"] % fld.ncol
    assert np.array_equal(b["cell"] % fld.ncol, fld.ncol - 1 - ja)
    Lx = float(fld.delr.sum())
    np.testing.assert_allclose(b["gx"], Lx - a["gx"], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(b["gy"], a["gy"], rtol=1e-10)
    np.testing.assert_allclose(b["t"], a["t"], rtol=1e-10)


def test_particle_order_independence(fld, rel):
    a = O.track(fld, rel)
    perm = np.random.default_rng(0).permutation(len(rel["cell"]))
    b = O.track(fld, O.subset(rel, perm))
    for k in a:
        assert np.array_equal(a[k][perm], b[k])


def test_step_cap_and_stop_at_start(fld, rel):
    r = O.track(fld, rel, max_steps=3)
    assert np.all(r["steps"] <= 3)
    capped = r["status"] == O.ST_STEP_CAP
    assert capped.any() and np.all(r["steps"][capped] == 3)
    z = O.track(fld, rel, t_stop=0.0)
    assert np.all(z["steps"] == 0) and np.all(z["status"] == O.ST_TIME)
