"""Weak sinks with a threshold fraction on the oracle (Introduction: how
weak sink cells are treated is a choice of the tracking configuration;
TC2 passes them).  With pass-through and a fraction f > 0, a sink cell whose
sink extracts at least f of its inflow stops particles like a strong sink,
the others are passed.

Pins from outside the oracle:
* the extraction fractions are computed here from the field's face flows
  with numpy;
* f below every well's fraction gives the strong-sink results bit for bit,
  f above every fraction the plain pass-through results bit for bit;
* for every f between the fractions, no path leaves a cell whose fraction
  is at least f, every path that enters one ends there as SINK, and paths
  that never enter one are those of plain pass-through.
"""
import numpy as np
import pytest

import oracle as O
from paper_2302_13590_gb300 import inputs as I
from paper_2302_13590_gb300.inputs import usg as U

# every pin holds for both arithmetic modes of the oracle
pytestmark = pytest.mark.usefixtures("oracle_arith")


def _fractions_structured(f):
    nlay, nrow, ncol = f.nlay, f.nrow, f.ncol
    qx = np.asarray(f.qx).reshape(nlay, nrow, ncol + 1)
    qy = np.asarray(f.qy).reshape(nlay, nrow + 1, ncol)
    qz = np.asarray(f.qz).reshape(nlay + 1, nrow, ncol)
    lo = [qx[:, :, :-1], qy[:, :-1, :], qz[:-1, :, :]]
    hi = [qx[:, :, 1:], qy[:, 1:, :], qz[1:, :, :]]
    inflow = sum(np.maximum(a, 0) + np.maximum(-b, 0) for a, b in zip(lo, hi))
    outflow = sum(np.maximum(-a, 0) + np.maximum(b, 0) for a, b in zip(lo, hi))
    return np.where(inflow > 0, (inflow - outflow) / np.where(inflow > 0, inflow, 1), 1.0).reshape(-1)


def _fractions_usg(u):
    q = np.zeros((u.ncell, 6))
    for c in range(u.ncell):
        for fi in range(6):
            q[c, fi] = float(np.sum(u.q[u.subfaces(c, fi)]))
    inflow = sum(np.maximum(q[:, 2 * a], 0) + np.maximum(-q[:, 2 * a + 1], 0) for a in range(3))
    outflow = sum(np.maximum(-q[:, 2 * a], 0) + np.maximum(q[:, 2 * a + 1], 0) for a in range(3))
    return np.where(inflow > 0, (inflow - outflow) / np.where(inflow > 0, inflow, 1), 1.0)


def _equal(a, b):
    for k in a:
        if k == "path":
            assert a[k].tobytes() == b[k].tobytes(), k
        else:
            assert np.array_equal(a[k], b[k], equal_nan=True), k


def _check(f, fr, sinks, st, n):
    strong = O.track(f, st, pathline=True)
    passed = O.track(f, st, pass_weak_sinks=True, pathline=True)
    fs = np.sort(fr[sinks])
    assert fs[0] > 0 and fs[-1] < 1 and np.min(np.diff(fs)) > 1e-6
    _equal(O.track(f, st, pass_weak_sinks=True, pathline=True, weak_sink_fraction=fs[0] / 2), strong)
    _equal(O.track(f, st, pass_weak_sinks=True, pathline=True, weak_sink_fraction=(fs[-1] + 1) / 2), passed)
    stopped_somewhere = 0
    for thr in (fs[:-1] + fs[1:]) / 2:
        r = O.track(f, st, pass_weak_sinks=True, pathline=True, weak_sink_fraction=thr)
        stopping = set(int(c) for c in sinks[fr[sinks] >= thr])
        path = np.sort(r["path"], order=["particle", "seq"])
        ppath = np.sort(passed["path"], order=["particle", "seq"])
        for q in range(n):
            cells = path["cell"][path["particle"] == q]
            hit = [i for i, c in enumerate(cells) if int(c) in stopping]
            # a stopping sink is never entered: the path stops on its face
            assert not hit, (thr, q)
            pcells = ppath["cell"][ppath["particle"] == q]
            phit = [i for i, c in enumerate(pcells) if int(c) in stopping]
            if phit:
                # plain pass-through entered a stopping sink: here the path
                # ends as SINK on the face of the cell before it, like a
                # strong sink
                stopped_somewhere += 1
                assert r["status"][q] == O.ST_SINK
                # the same cells up to the one before the sink, then the stop
                # point on its face (in that cell)
                assert np.array_equal(cells[:-1], pcells[:phit[0]]) and cells[-1] == pcells[phit[0] - 1]
                assert int(r["cell"][q]) == int(pcells[phit[0] - 1])
            else:
                assert np.array_equal(cells, pcells) and r["status"][q] == passed["status"][q]
                assert r["t"][q] == passed["t"][q]
    assert stopped_somewhere > 0


def test_weak_sink_fraction_structured():
    f = I.random_box_field(2, 5, 8, seed=40, lnk_var=0.5, n_wells=3, well_scale=10.0)
    fr = _fractions_structured(f)
    sinks = np.nonzero(f.ibound.reshape(-1) == 2)[0]
    cells, frac = I.explicit_particles(f, 60, seed=9, cols=(1, 3))
    _check(f, fr, sinks, O.release_explicit(f, cells, frac), cells.size)


def test_weak_sink_fraction_quadtree():
    u = U.quadtree_field(2, 8, 12, seed=15, n_wells=3, well_rate=0.05)
    fr = _fractions_usg(u)
    sinks = np.nonzero(u.ibound == U.IB_SINK)[0]
    cells, frac = U.explicit_particles(u, 80, seed=5)
    _check(u, fr, sinks, O.release_explicit(u, cells, frac), cells.size)
