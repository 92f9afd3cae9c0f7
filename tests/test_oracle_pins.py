"""Pins for the CPU oracle against closed forms, brute force and published vectors.

Each test checks the oracle against something other than itself:
* Philox4x32-10 against the published known-answer vectors (tests/golden);
* uniform flow (A = 0): travel time = sum of (distance * porosity * area / Q);
* one cell with linearly varying velocity: exit time ln(v_exit/v_p)/A and
  position (v_p e^{At} - v_1)/A, the Pollock (1988) solution evaluated
  directly with libm's log/exp;
* the A -> 0 limit: continuity against the Taylor series of ln(1+z)/z;
* RK4 integration with bisection on face events on small random
  mass-conserving fields (cell sequences, times and positions).
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2302_13590_gb300 import inputs as I
from tests import helpers as H

# every pin holds for both arithmetic modes of the oracle
pytestmark = pytest.mark.usefixtures("oracle_arith")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
_RK4_CACHE = {}


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


@pytest.mark.parametrize("q_sign", [1.0, -1.0])
def test_uniform_flow_travel_time(q_sign):
    f = H.uniform_x_field(2, 3, 9, seed=11, q_sign=q_sign)
    rng = np.random.default_rng(5)
    n = 40
    cells, frac = [], []
    for _ in range(n):
        k, i, j = int(rng.integers(0, 2)), int(rng.integers(0, 3)), int(rng.integers(0, 9))
        cells.append((k * 3 + i) * 9 + j)
        frac.append(rng.random(3))
    st = O.release_explicit(f, np.array(cells, np.int32), np.array(frac))
    r = O.track(f, st)
    for q in range(n):
        c = cells[q]
        j, i, k = c % 9, (c // 9) % 3, c // 27
        area = f.delc[i] * f.dz[k]
        Q = f.qx[k, i, 0]
        p = st["px"][q]
        if q_sign > 0:
            parts = [(f.delr[j] - p) * f.porosity[k, i, j] * area / Q]
            parts += [f.delr[jj] * f.porosity[k, i, jj] * area / Q for jj in range(j + 1, 9)]
            assert r["gx"][q] == pytest.approx(f.origin[0] + f.delr.sum(), rel=1e-14)
            assert r["steps"][q] == 9 - j
            assert r["exit_face"][q] == 1
        else:
            parts = [p * f.porosity[k, i, j] * area / (-Q)]
            parts += [f.delr[jj] * f.porosity[k, i, jj] * area / (-Q) for jj in range(0, j)]
            assert r["gx"][q] == pytest.approx(f.origin[0], abs=1e-13)
            assert r["steps"][q] == j + 1
            assert r["exit_face"][q] == 0
        t_exact = math.fsum(parts)
        assert r["status"][q] == O.ST_EXIT_DOMAIN
        assert r["t"][q] == pytest.approx(t_exact, rel=1e-13)
        # straight lines: y and z untouched
        assert r["py"][q] == st["py"][q] and r["pz"][q] == st["pz"][q]


def test_uniform_flow_stop_time_position():
    f = H.uniform_x_field(1, 1, 6, seed=3)
    st = O.release_explicit(f, np.array([0], np.int32), np.array([[0.0, 0.5, 0.5]]))
    v = [f.qx[0, 0, 0] / (f.porosity[0, 0, j] * f.delc[0] * f.dz[0]) for j in range(6)]
    # time T: cell 0 fully (delr0/v0), then 0.25 of cell 1
    T = f.delr[0] / v[0] + 0.25 * f.delr[1] / v[1]
    r = O.track(f, st, t_stop=T)
    assert r["status"][0] == O.ST_TIME
    assert r["t"][0] == T
    assert r["cell"][0] == 1
    assert r["px"][0] == pytest.approx(0.25 * f.delr[1], rel=1e-13)


@pytest.mark.parametrize("v1,v2,pfrac", [(1.0, 3.0, 0.2), (2.0, 0.5, 0.7), (-1.0, -4.0, 0.6),
                                         (-3.0, -0.2, 0.1), (0.3, 10.0, 0.0), (-0.5, 0.5, 0.9)])
def test_single_cell_linear_velocity(v1, v2, pfrac):
    D = (2.0, 3.0, 1.5)
    por = 0.25
    area = D[1] * D[2]
    f = H.single_cell_field(v1 * por * area, v2 * por * area, d=D, por=por)
    A = (v2 - v1) / D[0]
    p0 = pfrac * D[0]
    vp = v1 + A * p0
    st = O.release_explicit(f, np.array([0], np.int32), np.array([[pfrac, 0.5, 0.5]]))
    r = O.track(f, st)
    if vp > 0 and v2 > 0:
        t_exit = math.log(v2 / vp) / A
        assert r["status"][0] == O.ST_EXIT_DOMAIN and r["exit_face"][0] == 1
        assert r["t"][0] == pytest.approx(t_exit, rel=1e-13)
    elif vp < 0 and v1 < 0:
        t_exit = math.log(v1 / vp) / A
        assert r["status"][0] == O.ST_EXIT_DOMAIN and r["exit_face"][0] == 0
        assert r["t"][0] == pytest.approx(t_exit, rel=1e-13)
    else:
        # divide inside the cell: no face is reachable
        assert r["status"][0] == O.ST_NO_EXIT
        t_exit = 10.0 / abs(A)
    # positions at intermediate times: p(t) = (vp e^{At} - v1) / A
    for frac_t in (0.1, 0.5, 0.9):
        tau = frac_t * t_exit
        r2 = O.track(f, st, t_stop=tau)
        p_exact = (vp * math.exp(A * tau) - v1) / A
        assert r2["status"][0] == O.ST_TIME
        assert r2["px"][0] == pytest.approx(p_exact, rel=1e-12, abs=1e-13 * D[0])


def test_exit_time_a_to_zero_limit_is_continuous():
    """ln(1+z)/z -> 1 with no jump: compare with its Taylor series for small z
    and with ln(v2/vp)/A where the ratio is far from 1."""
    D, p, v1 = 2.0, 0.4, 1.0
    prev = None
    for e in np.logspace(-18, -1, 69):
        v2 = v1 * (1.0 + e)
        A = (v2 - v1) / D
        t, face = O.exit_time(v1, v2, A, D, p)
        assert face == 1
        vp = v1 + A * p
        d = D - p
        z = A * d / vp
        t1 = d / vp
        if abs(z) < 1e-3:
            series = t1 * (1 - z / 2 + z * z / 3 - z ** 3 / 4 + z ** 4 / 5)
            assert t == pytest.approx(series, rel=2e-16 * 8)
        else:
            assert t == pytest.approx(math.log(v2 / vp) / A, rel=1e-13)
        if prev is not None:
            assert t <= prev * (1 + 1e-15)   # exit time falls as the far face speeds up
        prev = t
    # exactly uniform: the limit value d / vp
    t, face = O.exit_time(1.0, 1.0, 0.0, D, p)
    assert t == (D - p) / 1.0


def test_motion_factor_limit():
    # expm1(w)/w -> 1: moving with A tiny must match uniform motion
    for A in (0.0, 1e-300, 1e-20, -1e-20):
        pn = O.move(0.5, A, 10.0, 1.0, 3.0)
        assert pn == pytest.approx(1.0 + 0.5 * 3.0, rel=1e-15)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_oracle_matches_rk4_brute_force(seed):
    f = I.random_box_field(2, 3, 6, seed=100 + seed, lnk_var=1.0, n_wells=1 if seed == 2 else 0)
    cells, frac = I.explicit_particles(f, 8, seed=7 + seed, cols=(1, 3))
    st = O.release_explicit(f, cells, frac)
    r = O.track(f, st)
    for q in range(len(cells)):
        c = int(cells[q])
        j, i, k = c % f.ncol, (c // f.ncol) % f.nrow, c // (f.ncol * f.nrow)
        p0 = [st["px"][q], st["py"][q], st["pz"][q]]
        status, seq, (kk, ii, jj), p, t = H.rk4_track(f, k, i, j, p0)
        assert status == r["status"][q]
        assert H.fnv_hash(seq) == int(r["hash"][q])
        assert len(seq) == int(r["steps"][q])
        assert r["t"][q] == pytest.approx(t, rel=1e-8)
        for a, key in enumerate(("px", "py", "pz")):
            D = (f.delr[jj], f.delc[ii], f.dz[kk])[a]
            assert abs(r[key][q] - p[a]) <= 1e-7 * D


@pytest.mark.parametrize("seed", [4, 5])
def test_oracle_rk4_stop_time(seed):
    f = I.random_box_field(2, 4, 7, seed=200 + seed, lnk_var=2.0)
    cells, frac = I.explicit_particles(f, 6, seed=seed, cols=(1, 2))
    st = O.release_explicit(f, cells, frac)
    full = O.track(f, st)
    for q in range(len(cells)):
        T = 0.6 * float(full["t"][q])
        c = int(cells[q])
        j, i, k = c % f.ncol, (c // f.ncol) % f.nrow, c // (f.ncol * f.nrow)
        r = O.track(f, O.subset(st, [q]), t_stop=T)
        status, seq, (kk, ii, jj), p, t = H.rk4_track(f, k, i, j, [st["px"][q], st["py"][q], st["pz"][q]], t_stop=T)
        assert status == 1 and r["status"][0] == O.ST_TIME
        assert H.fnv_hash(seq) == int(r["hash"][0])
        assert r["cell"][0] == (kk * f.nrow + ii) * f.ncol + jj
        for a, key in enumerate(("px", "py", "pz")):
            D = (f.delr[jj], f.delc[ii], f.dz[kk])[a]
            assert abs(r[key][0] - p[a]) <= 1e-7 * D


def test_release_box_locates_cells():
    f = I.random_box_field(3, 4, 5, seed=9, lnk_var=0.5)
    Lx, Ly, Lz = float(f.delr.sum()), float(f.delc.sum()), float(f.dz.sum())
    st = O.release_box(f, 500, (0.0, 0.0, 0.0), (Lx, Ly, Lz), seed=1234)
    xf = np.concatenate([[0.0], np.cumsum(f.delr)])
    yf = np.concatenate([[0.0], np.cumsum(f.delc)])
    zf = np.concatenate([[0.0], np.cumsum(f.dz)])
    c = st["cell"]
    j, i, k = c % f.ncol, (c // f.ncol) % f.nrow, c // (f.ncol * f.nrow)
    assert np.all(st["px"] >= 0) and np.all(st["px"] <= f.delr[j])
    assert np.all(st["py"] >= 0) and np.all(st["py"] <= f.delc[i])
    assert np.all(st["pz"] >= 0) and np.all(st["pz"] <= f.dz[k])
    gx = xf[j] + st["px"]
    # positions are uniform over the box: mean near the centre
    assert abs(gx.mean() / Lx - 0.5) < 0.05
    assert abs((yf[i] + st["py"]).mean() / Ly - 0.5) < 0.05
    assert abs((zf[k] + st["pz"]).mean() / Lz - 0.5) < 0.05
    # constant-head columns are not valid release cells
    bad = f.ibound.reshape(-1)[c] == -1
    assert np.all(st["status"][bad] == O.ST_INVALID_RELEASE)
    assert np.all(st["status"][~bad] == O.ST_ACTIVE)
    # the stream is keyed by (seed, particle index): an offset shifts it
    st2 = O.release_box(f, 100, (0.0, 0.0, 0.0), (Lx, Ly, Lz), seed=1234, id_offset=400)
    assert np.array_equal(st2["cell"], st["cell"][400:]) and np.array_equal(st2["px"], st["px"][400:])


def test_exact_tie_goes_to_lowest_axis():
    """Equal exit times on x and y (a reading: the lowest axis wins, and only
    that face is crossed); the y coordinate lands on its face by the motion
    formula and leaves on the next step with a zero-length step."""
    por, D = 0.5, (2.0, 2.0, 1.0)
    qx = 1.0 * por * D[1] * D[2]
    qy = 1.0 * por * D[0] * D[2]
    f = H.single_cell_field(qx, qx, qy, qy, d=D, por=por)
    st = O.release_explicit(f, np.array([0], np.int32), np.array([[0.25, 0.25, 0.5]]))
    r = O.track(f, st)
    assert r["exit_face"][0] == 1          # +x, not +y
    assert r["t"][0] == 1.5
    assert r["px"][0] == 2.0 and r["py"][0] == 2.0


def test_series_log1p_expm1_against_libm():
    """The oracle's own log1p/expm1 (argument reduction, a table of correctly
    rounded constants and a short series, IEEE basic operations only) stay
    within a few ulp of the C library across the
    ranges the tracker meets, and keep the limits exact."""
    rng = np.random.default_rng(0)
    xs = np.concatenate([-np.exp(-rng.uniform(0, 40, 4000)), np.exp(rng.uniform(-60, 15, 4000)),
                         -rng.uniform(0, 1, 4000) * (1 - 1e-12), rng.uniform(-1e-3, 1e-3, 4000)])
    xs = xs[xs > -1]
    worst = max(abs(O.log1p(x) - math.log1p(x)) / np.spacing(abs(math.log1p(x))) for x in xs if x != 0)
    assert worst <= 4
    ws = np.concatenate([rng.uniform(-40, 40, 4000), rng.uniform(-0.4, 0.4, 4000), rng.uniform(-1e-5, 1e-5, 4000),
                         rng.uniform(-700, 700, 4000)])
    worst = max(abs(O.expm1(w) - math.expm1(w)) / np.spacing(abs(math.expm1(w))) for w in ws if w != 0)
    assert worst <= 4
    assert O.log1p(0.0) == 0.0 and O.expm1(0.0) == 0.0
    assert O.log1p(1e-300) == 1e-300 and O.expm1(-1e-300) == -1e-300
    assert O.expm1(800.0) == math.inf and O.expm1(-800.0) == -1.0


def test_weak_sinks_pass_through_against_rk4():
    """Pass-through of weak sinks: particles enter well cells and leave
    through faces they can reach (checked by RK4 integration); those that
    cannot are captured inside the well cell."""
    f = I.random_box_field(2, 5, 8, seed=40, lnk_var=0.5, n_wells=3, well_scale=30.0)
    wells = np.nonzero(f.ibound.reshape(-1) == 2)[0]
    cells, frac = I.explicit_particles(f, 60, seed=9, cols=(1, 3))
    st = O.release_explicit(f, cells, frac)
    strong = O.track(f, st)
    weak = O.track(f, st, pass_weak_sinks=True)
    passed = captured = 0
    # the capture horizon: ten times the longest path (the RK4 paths do
    # not depend on the oracle's arithmetic: integrated once, compared per mode)
    key = ("weak_sinks_rk4", float(np.max(O.track(f, st, arith="plain")["t"])))
    if key not in _RK4_CACHE:
        paths = []
        for q in range(len(cells)):
            c = int(cells[q])
            j, i, k = c % f.ncol, (c // f.ncol) % f.nrow, c // (f.ncol * f.nrow)
            p0 = [st["px"][q], st["py"][q], st["pz"][q]]
            paths.append(H.rk4_track(f, k, i, j, p0, pass_sinks=True, capture_time=10 * key[1]))
        _RK4_CACHE[key] = paths
    for q in range(len(cells)):
        status, seq, (kk, ii, jj), p, t = _RK4_CACHE[key][q]
        assert status == weak["status"][q]
        assert H.fnv_hash(seq) == int(weak["hash"][q])
        if status != O.ST_SINK:
            assert weak["t"][q] == pytest.approx(t, rel=1e-7)
        entered = np.isin(seq, wells)
        if entered.any() and status != O.ST_SINK:
            passed += 1
        if status == O.ST_SINK:
            captured += 1
            assert int(weak["cell"][q]) in wells
        # without the option every particle that reaches a well stops at its face
        if strong["status"][q] == O.ST_SINK:
            assert int(strong["cell"][q]) not in wells
    assert passed > 0 and captured > 0
