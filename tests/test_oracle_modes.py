"""The oracle's two arithmetic modes and the divergence classifier.

The plain mode is the reference (the formulas as they read, the C library's
log1p/expm1); the mirror mode evaluates the same solution by fixed
table-driven steps.  Both are pinned by the same closed forms, brute force
and invariants (every test_oracle_* module runs in both modes); here they are
compared with each other on well-conditioned workloads, and the classifier
that explains a divergent path is checked on hand-made traces.
"""
import numpy as np
import pytest

import oracle as O
from paper_2302_13590_gb300 import inputs as I
from tests import divergence as D


def _agree(a, b, rtol):
    assert np.array_equal(a["hash"], b["hash"])
    for k in ("status", "cell", "steps", "exit_face"):
        assert np.array_equal(a[k], b[k]), k
    assert np.max(np.abs(a["t"] - b["t"]) / np.abs(b["t"])) <= rtol
    for k in ("gx", "gy", "gz"):
        assert np.max(np.abs(a[k] - b[k])) <= rtol * 1e3


def test_modes_agree_on_the_homogeneous_field():
    w = I.workload("cfg1")
    st = O.release_box(w.field, w.release.n, w.release.lo, w.release.hi, w.release.seed)
    a = O.track(w.field, st, times=w.times, arith="plain")
    b = O.track(w.field, st, times=w.times, arith="mirror")
    _agree(a, b, 1e-13)
    assert np.array_equal(a["ts_cell"], b["ts_cell"])


@pytest.mark.parametrize("seed", [3, 5])
def test_modes_agree_on_random_fields(seed):
    f = I.random_box_field(4, 9, 12, seed=300 + seed, lnk_var=2.0, n_wells=2, n_inactive=3)
    cells, frac = I.explicit_particles(f, 1000, seed=seed, cols=(1, 6))
    st = O.release_explicit(f, cells, frac)
    _agree(O.track(f, st, arith="plain"), O.track(f, st, arith="mirror"), 1e-12)


def _scaled(f, s):
    """The same field with every face flow times s: velocities scale by s,
    travel times by 1/s, paths stay the same."""
    import dataclasses
    return dataclasses.replace(f, qx=f.qx * s, qy=f.qy * s, qz=f.qz * s)


@pytest.mark.parametrize("scale", [1e-40, 1e42])
def test_modes_agree_at_extreme_velocity_scales(scale):
    """Velocities below 2^-120 and above 2^121 (the mirror's quotient falls
    back to the IEEE division there): both modes take the paths of the
    unscaled field, with travel times scaled by 1/s to rounding."""
    f = I.random_box_field(2, 5, 7, seed=321, lnk_var=1.0, n_wells=1, n_inactive=1)
    cells, frac = I.explicit_particles(f, 200, seed=4, cols=(1, 3))
    st = O.release_explicit(f, cells, frac)
    base = O.track(f, st, arith="plain")
    fs = _scaled(f, scale)
    # typical x velocity q / (n A): beyond the reciprocal's range on the scaled field
    area = np.outer(f.dz, f.delc)[:, :, None]
    v = np.abs(fs.qx[:, :, 1:-1]) / (np.asarray(f.porosity).reshape(f.qx[:, :, 1:].shape)[:, :, :-1] * area)
    vmed = float(np.median(v[v > 0]))
    assert (vmed < 2.0 ** -120) if scale < 1 else (vmed > 2.0 ** 121)
    a, b = O.track(fs, st, arith="plain"), O.track(fs, st, arith="mirror")
    _agree(a, b, 1e-12)
    assert np.array_equal(a["hash"], base["hash"])
    ok = base["t"] > 0
    assert np.max(np.abs(a["t"][ok] * scale - base["t"][ok]) / base["t"][ok]) <= 1e-12
    for k in ("gx", "gy", "gz"):
        assert np.max(np.abs(a[k] - base[k])) <= 1e-9


def test_modes_differ_by_rounding_only():
    """The two modes are distinct evaluations (not one code path twice):
    on a heterogeneous field their travel times differ in the last bits."""
    f = I.random_box_field(4, 9, 12, seed=305, lnk_var=2.0, n_wells=2, n_inactive=3)
    cells, frac = I.explicit_particles(f, 400, seed=5, cols=(1, 6))
    st = O.release_explicit(f, cells, frac)
    a, b = O.track(f, st, arith="plain"), O.track(f, st, arith="mirror")
    d = np.abs(a["t"] - b["t"]) / a["t"]
    assert np.count_nonzero(d) > 0 and d.max() <= 1e-12


def test_trace_records_every_step():
    f = I.random_box_field(2, 5, 8, seed=40, lnk_var=0.5, n_wells=1)
    cells, frac = I.explicit_particles(f, 20, seed=9, cols=(1, 3))
    st = O.release_explicit(f, cells, frac)
    for arith in ("plain", "mirror"):
        r = O.track(f, st, arith=arith, trace=True)
        tr = r["trace"]
        assert tr.size == int(r["steps"].sum())
        for q in range(cells.size):
            rows = tr[tr["particle"] == q]
            ax = rows["ax"][rows["ax"] >= 0]
            te = rows["te"][rows["ax"] >= 0]
            # the axis taken has the smallest exit time of the step
            assert np.all(te[np.arange(ax.size), ax] == te.min(axis=1))
            assert np.all(np.diff(rows["t"]) >= 0)


def _rec(te, ax, face=(1, 1, 1), vp=(1.0, 1.0, 1.0), vf=(1.0, 1.0, 1.0), t=0.0, cell=0):
    r = np.zeros((), O.TRACE_RECORD)
    r["te"], r["vp"], r["vf"], r["t"], r["cell"], r["face"], r["ax"] = te, vp, vf, t, cell, face, ax
    return r


def _trace(*recs):
    out = np.zeros(len(recs), O.TRACE_RECORD)
    for i, r in enumerate(recs):
        out[i] = r
    return out


def test_first_divergence_kinds():
    same = _rec((1.0, 2.0, 3.0), 0, t=5.0)
    # an exit-axis flip at a near-tie: gap 1e-12 against t + te = 7
    a = _trace(same, _rec((2.0, 2.0 + 1e-12, np.inf), 0, t=6.0))
    b = _trace(same, _rec((2.0, 2.0, np.inf), 1, t=6.0))
    d = D.first_divergence(a, b)
    assert (d.kind, d.step) == ("axis", 1)
    assert d.gap == pytest.approx(1e-12, rel=1e-3) and d.scale == pytest.approx(8.0)
    assert d.rel <= 1e-10
    # a far-apart choice is not a near-tie
    a2 = _trace(same, _rec((2.0, 3.0, np.inf), 0, t=6.0))
    assert D.first_divergence(a2, b).rel > 1e-2
    # opposite faces of one axis: the particle velocity against the face velocity
    c = _trace(_rec((1.0, np.inf, np.inf), 0, face=(1, 0, 0), vp=(1e-20, 0, 0), vf=(3.0, 0, 0)))
    e = _trace(_rec((1.0, np.inf, np.inf), 0, face=(-1, 0, 0), vp=(-1e-20, 0, 0), vf=(3.0, 0, 0)))
    d = D.first_divergence(c, e)
    assert d.kind == "face" and d.rel == pytest.approx(1e-20 / 3.0)
    # stop time reached in one, the face in the other
    s1 = _trace(_rec((4.0, np.inf, np.inf), -1, t=6.0))
    s2 = _trace(_rec((4.0, np.inf, np.inf), 0, t=6.0))
    d = D.first_divergence(s1, s2, t_stop=10.0 + 1e-9)
    assert d.kind == "stop" and d.gap == pytest.approx(1e-9, rel=1e-3)
    # one leaves through a face the other cannot reach (its particle
    # velocity rounded to zero): a face divergence at that velocity, not a stop
    x1 = _trace(_rec((2.8e9, np.inf, np.inf), 0, vp=(1.4e-20, 1.0, 1.0), vf=(1.06e-5, 1.0, 1.0), t=6.0))
    x2 = _trace(_rec((np.inf, np.inf, np.inf), -1, face=(0, 0, 0), vp=(0.0, 1.0, 1.0), vf=(1.06e-5, 1.0, 1.0),
                     t=6.0))
    d = D.first_divergence(x1, x2)
    assert d.kind == "face" and d.rel == pytest.approx(1.4e-20 / 1.06e-5)
    # identical steps, one trace longer: an unexplained end
    assert D.first_divergence(_trace(same), _trace(same, same)).kind == "end"
    # a different cell after the same exit (a hand-over)
    assert D.first_divergence(_trace(same, _rec((1, 1, 1), 0, cell=1)), _trace(same, _rec((1, 1, 1), 0, cell=2))).kind == "cell"
