"""Shared GPU-test helpers: run the CUDA path through the C ABI and compare
it with the oracle."""
from __future__ import annotations

import numpy as np

from paper_2302_13590_gb300 import mp

KEYS_EXACT = ("status", "cell", "steps", "exit_face", "hash")


def gpu_run(ctx, fh, *, release=None, cells=None, frac=None, t0=None, times=None, t_stop=np.inf,
            precision=mp.PREC_FP64, schedule=mp.SCHED_DYNAMIC, max_steps=0, block=0, steps_per_fetch=0,
            mode=None, flags=0):
    """Release + track through the C ABI; returns (endpoints dict, timeseries or None, stats)."""
    if release is not None:
        gh = mp.mp_release_group(ctx.h, fh, n=release.n, lo=release.lo, hi=release.hi, seed=release.seed,
                                 id_offset=release.id_offset)
    else:
        gh = mp.mp_release_group(ctx.h, fh, cell=cells, local=frac, t0=t0)
    if mode is None:
        mode = mp.MODE_ENDPOINT | (mp.MODE_TIMESERIES if times is not None else 0)
    req = ctx.track(gh, mode=mode, precision=precision, schedule=schedule, times=times, t_stop=t_stop,
                    max_steps=max_steps, block=block, steps_per_fetch=steps_per_fetch, flags=flags)
    req.wait()
    ep = req.endpoints()
    ts = req.timeseries() if req.n_times else None
    st = req.stats()
    req.free()
    mp.mp_group_free(gh)
    return ep, ts, st


def release_state(ctx, fh, release):
    """The device release as a state dict (a zero-time run reports the release)."""
    ep, _, _ = gpu_run(ctx, fh, release=release, t_stop=0.0, schedule=mp.SCHED_STATIC)
    st = np.where(ep["status"] == mp.ST_TIME, mp.ST_ACTIVE, ep["status"]).astype(np.uint8)
    return dict(cell=ep["cell"], px=ep["px"], py=ep["py"], pz=ep["pz"], t=np.zeros(ep["cell"].size), status=st)


def rel_err(a, b, scale=None):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    d = np.abs(a - b)
    s = np.abs(b) if scale is None else scale
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(d == 0, 0.0, d / np.maximum(s, 1e-300))


def dmin(f):
    """Position scale per axis: the extent of the grid along that axis."""
    if not hasattr(f, "delr"):   # a quadtree grid
        return tuple(float(v) for v in f.extent)
    return (float(np.sum(f.delr)), float(np.sum(f.delc)), float(np.sum(f.dz)))


def pos_scale(field, b):
    """Scale for position errors along one axis: the larger of |coordinate|
    and the grid extent along that axis (a relative error of a coordinate
    near the origin says nothing)."""
    return np.maximum(np.abs(b), b * 0 + field)


def _same_bits(a, b):
    return int(np.count_nonzero(np.ascontiguousarray(a).view(np.int64) != np.ascontiguousarray(b).view(np.int64)))


def compare_fp64(ep, ref, idx=None, rtol=1e-10, dmin=(1.0, 1.0, 1.0), allow_divergent=0.0, exact=True):
    """FP64 parity: exact cell sequences and statuses; travel times within
    rtol relative; positions within rtol relative to max(|x|, grid extent);
    with ``exact`` (the reference is the oracle's mirror arithmetic or
    another run of the kernels) travel times and positions bit for bit.

    allow_divergent: fraction of particles whose cell sequence may differ
    (for strongly ill-conditioned fields, where a 1-ulp difference between
    the platforms' log1p/expm1 can flip a near-tie); the other particles
    are held to the full check.  Returns the number of divergent particles."""
    sel = slice(None) if idx is None else idx
    hsame = ep["hash"][sel] == ref["hash"]
    ndiv = int((~hsame).sum())
    assert ndiv <= allow_divergent * hsame.size, f"{ndiv} divergent cell sequences of {hsame.size}"
    keep = np.nonzero(hsame)[0]
    ep = {k: (np.asarray(v)[sel][keep]) for k, v in ep.items()}
    ref = {k: (np.asarray(v)[keep] if np.ndim(v) == 1 else v) for k, v in ref.items()}
    sel = slice(None)
    for k in KEYS_EXACT:
        a, b = ep[k][sel], ref[k]
        bad = np.nonzero(a != b)[0]
        assert bad.size == 0, f"{k}: {bad.size} mismatches, first {bad[:5]}: gpu {a[bad[:5]]} oracle {b[bad[:5]]}"
    for ax, (gk, ok) in enumerate((("x", "gx"), ("y", "gy"), ("z", "gz"), ("t", "t"))):
        a, b = ep[gk][sel], ref[ok]
        fin = np.isfinite(b)
        assert np.array_equal(np.isfinite(a), fin), gk
        scale = None if gk == "t" else pos_scale(dmin[ax], b[fin])
        e = rel_err(a[fin], b[fin], scale=scale)
        assert e.max(initial=0.0) <= rtol, f"{gk}: max rel err {e.max()}"
        if exact:
            nb = _same_bits(a[fin], b[fin])
            assert nb == 0, f"{gk}: {nb} of {int(fin.sum())} values not bit-identical (max rel err {e.max()})"
    return ndiv


def compare_timeseries_fp64(ts, ref, idx=None, rtol=1e-10, dmin=(1.0, 1.0, 1.0), keep=None, exact=True):
    """Timeseries parity; keep = boolean mask of particles (of the sample) to
    check (those whose cell sequence matches); ``exact`` as in compare_fp64."""
    sel = slice(None) if idx is None else idx
    if keep is not None:
        base = np.arange(ts.shape[1])[sel]
        sel = base[keep]
        ref = {k: (v[:, keep] if np.ndim(v) == 2 else v) for k, v in ref.items()}
    assert np.array_equal(ts["cell"][:, sel], ref["ts_cell"])
    assert np.array_equal(ts["status"][:, sel], ref["ts_status"])
    for ax, (gk, ok) in enumerate((("x", "ts_x"), ("y", "ts_y"), ("z", "ts_z"))):
        a, b = ts[gk][:, sel], ref[ok]
        fin = np.isfinite(b)
        assert np.array_equal(np.isfinite(a), fin)
        e = rel_err(a[fin], b[fin], scale=pos_scale(dmin[ax], b[fin]))
        assert e.max(initial=0.0) <= rtol, f"ts {gk}: max rel err {e.max()}"
        if exact:
            nb = _same_bits(a[fin], b[fin])
            assert nb == 0, f"ts {gk}: {nb} of {int(fin.sum())} records not bit-identical (max rel err {e.max()})"


def ts_pos_err(ts_xyz, ref, field):
    """Per particle: the largest timeseries position error (relative to
    pos_scale) of records ``ts_xyz`` = (x, y, z) arrays [n_times, n] against
    ``ref``'s ts_x/ts_y/ts_z; NaN records (before release, invalid) compare
    by finiteness."""
    err = np.zeros(ref["ts_x"].shape[1] if np.ndim(ref["ts_x"]) == 2 else 0)
    for ax, (a, ok) in enumerate(zip(ts_xyz, ("ts_x", "ts_y", "ts_z"))):
        b = ref[ok]
        fin = np.isfinite(b)
        e = np.where(fin, rel_err(np.where(fin, a, 0.0), np.where(fin, b, 0.0),
                                  scale=pos_scale(dmin(field)[ax], np.where(fin, b, 0.0))), 0.0)
        e = np.where(np.isfinite(a) == fin, e, np.inf)
        err = np.maximum(err, e.max(axis=0, initial=0.0))
    return err


# the jitter (oracle/mp_oracle.h) of about one FP64 rounding: 2^-52 relative
FP64_JITTER = 2.0 ** -52


def fp64_spread(field, state, which, *, runs=4, t_stop=np.inf, times=None, **track_kw):
    """The plain oracle's own sensitivity to rounding, per particle of
    ``which``: the largest change of the travel time (relative) and of the
    endpoint (relative to pos_scale) over ``runs`` runs with every crossing
    jittered by about one FP64 rounding; +inf where a run changes the cell
    sequence."""
    import oracle as O
    which = np.asarray(which, dtype=np.int64)
    sub = O.subset(state, which)
    ref = O.track(field, sub, t_stop=t_stop, times=times, arith="plain", **track_kw)
    s_t = np.zeros(which.size)
    s_p = np.zeros(which.size)
    for r in range(runs):
        rj = O.track(field, sub, t_stop=t_stop, times=times, arith="plain", jitter=FP64_JITTER,
                     jitter_seed=2000 + r, **track_kw)
        div = rj["hash"] != ref["hash"]
        fin = np.isfinite(ref["t"])
        jt = np.zeros(which.size)
        jt[fin] = rel_err(rj["t"][fin], ref["t"][fin])
        jp = np.zeros(which.size)
        for ax, k in enumerate(("gx", "gy", "gz")):
            f2 = np.isfinite(ref[k])
            jp[f2] = np.maximum(jp[f2], rel_err(rj[k][f2], ref[k][f2], scale=pos_scale(dmin(field)[ax], ref[k][f2])))
        if times is not None:
            jp = np.maximum(jp, ts_pos_err((rj["ts_x"], rj["ts_y"], rj["ts_z"]), ref, field))
        s_t = np.maximum(s_t, np.where(div, np.inf, jt))
        s_p = np.maximum(s_p, np.where(div, np.inf, jp))
    return s_t, s_p


def compare_fp64_plain(ep, plain, *, field, state, idx=None, ts=None, times=None, t_stop=np.inf, rtol=1e-10,
                       label="", **track_kw):
    """FP64 GPU results against the plain-arithmetic oracle (the reference).

    Particles whose cell sequence (FNV hash) matches: statuses, cells, step
    counts and exit faces equal, travel times and positions (endpoint and
    timeseries) within ``rtol``, except where an exit starts from a
    stagnation surface: a particle beyond ``rtol`` is traced in both oracle
    modes and passes only if the first step whose exit times part has a
    particle velocity within 1e-12 of zero (relative to the face velocity),
    where the exit time ln(v_exit / v_p) / A is set by the rounding of a
    vanishing v_p; any other such particle must stay within 4 times the
    plain oracle's own spread under a jitter of about one FP64 rounding per
    crossing (fp64_spread: a particle near an unstable stagnation line,
    whose transverse offset grows like e^(A t), moves by far more than an
    ulp when its crossings are perturbed by one).  Particles whose sequence
    differs are traced the same way
    (the mirror mode equals the GPU bit for bit, which the caller checks
    separately) and each must part at a near-tie: at the first step where the
    evaluations choose differently, the reference's two competing choices
    lie within ``rtol`` of each other (divergence.py), or else a
    one-rounding jitter of the plain oracle must change that particle's
    cell sequence as well (a rounding difference amplified over the steps
    before, near a stagnation line, decides).  ``state`` is the
    oracle state of the compared particles (``idx`` of the GPU arrays).
    Returns (divergent, max relative time error, max relative position
    error, stagnation exits) and prints them."""
    from tests import divergence as D
    sel = slice(None) if idx is None else idx
    g = {k: np.asarray(v)[sel] for k, v in ep.items()}
    hsame = g["hash"] == plain["hash"]
    ndiv = int((~hsame).sum())
    keep = np.nonzero(hsame)[0]
    for k in ("status", "cell", "steps", "exit_face"):
        bad = keep[g[k][keep] != plain[k][keep]]
        assert bad.size == 0, f"{k}: {bad.size} mismatches on matching cell sequences, first {bad[:5]}"
    err_t = np.zeros(plain["t"].size)
    err_p = np.zeros(plain["t"].size)
    fin = np.isfinite(plain["t"])
    assert np.array_equal(np.isfinite(g["t"][keep]), fin[keep]), "t finiteness"
    err_t[fin] = rel_err(g["t"][fin], plain["t"][fin])
    for ax, (gk, ok) in enumerate((("x", "gx"), ("y", "gy"), ("z", "gz"))):
        b = plain[ok]
        f2 = np.isfinite(b)
        assert np.array_equal(np.isfinite(g[gk][keep]), f2[keep]), gk
        err_p[f2] = np.maximum(err_p[f2], rel_err(g[gk][f2], b[f2], scale=pos_scale(dmin(field)[ax], b[f2])))
    if ts is not None:
        tsel = np.arange(ts.shape[1])[sel]
        err_ts = ts_pos_err((ts["x"][:, tsel], ts["y"][:, tsel], ts["z"][:, tsel]), plain, field)
        err_p = np.maximum(err_p, np.where(hsame, err_ts, 0.0))
    over = keep[np.maximum(err_t[keep], err_p[keep]) > rtol]
    stagn = []
    rest = []
    if over.size:
        for q, step, ratio in D.stagnation_exits(field, state, over, rtol=rtol, t_stop=t_stop, times=times, **track_kw):
            (stagn if ratio <= 1e-12 else rest).append(q)
    if rest:
        s_t, s_p = fp64_spread(field, state, rest, t_stop=t_stop, times=times, **track_kw)
        for n, q in enumerate(rest):
            assert err_t[q] <= max(rtol, 4 * s_t[n]) and err_p[q] <= max(rtol, 4 * s_p[n]), (
                f"particle {q}: time or position beyond {rtol} on the same cell sequence (t err {err_t[q]:.3g}, "
                f"pos err {err_p[q]:.3g}), not from a stagnation exit and beyond 4 x the oracle's own spread "
                f"under one-rounding jitter (t {s_t[n]:.3g}, pos {s_p[n]:.3g})")
        stagn += rest
    good = np.setdiff1d(keep, np.asarray(stagn, dtype=np.int64))
    if ts is not None:
        mask = np.zeros(hsame.size, dtype=bool)
        mask[good] = True
        compare_timeseries_fp64(ts, plain, idx=idx, rtol=rtol, dmin=dmin(field), keep=mask, exact=False)
    t_err = err_t[good].max(initial=0.0)
    p_err = err_p[good].max(initial=0.0)
    bad = []
    if ndiv:
        for d in D.analyse(field, state, np.nonzero(~hsame)[0], t_stop=t_stop, times=times, **track_kw):
            if not d.rel <= rtol:
                bad.append(d)
    n_sens = 0
    if bad:
        # a divergence that is not a near-tie where it happens is still
        # rounding's when a one-rounding jitter of the plain oracle also
        # changes that particle's cell sequence (the decision was prepared
        # by an amplified rounding difference a few steps earlier)
        s_t, _ = fp64_spread(field, state, [d.particle for d in bad], t_stop=t_stop, times=times, **track_kw)
        n_sens = int(np.isinf(s_t).sum())
        bad = [d for d, s in zip(bad, s_t) if not np.isinf(s)]
    print(f"fp64 vs plain oracle {label}: {hsame.size} particles, {ndiv} divergent "
          f"({ndiv / max(hsame.size, 1):.2e}; {n_sens} of them not at a near-tie but parted by one-rounding jitter "
          f"too), {len(stagn) - len(rest)} stagnation exits, {len(rest)} within the "
          f"oracle's rounding spread, max rel t err {t_err:.2e}, "
          f"max rel pos err {p_err:.2e}")
    assert not bad, f"{len(bad)} divergent particles that are not near-ties, first {bad[:3]}"
    return ndiv, t_err, p_err, len(stagn)


# One FP32 rounding of a local coordinate or a step time, relative: the size
# of the oracle's per-step jitter that calibrates the mixed-precision bounds.
FP32_JITTER = 1e-7


def mixed_errors(ep, ref, field, idx=None):
    """Per particle (of ``ref``'s): relative travel-time error and endpoint
    error in cell widths of ``ep`` against ``ref``, +inf where the cell
    sequence differs."""
    sel = slice(None) if idx is None else idx
    g = {k: np.asarray(ep[k])[sel] for k in ("hash", "t", "x", "y", "z")}
    c = ref["cell"]
    j, i, k = c % field.ncol, (c // field.ncol) % field.nrow, c // (field.ncol * field.nrow)
    with np.errstate(invalid="ignore", divide="ignore"):
        dt = np.abs(g["t"] - ref["t"]) / np.abs(ref["t"])
        dt = np.where(g["t"] == ref["t"], 0.0, dt)
    dx = np.maximum.reduce([np.abs(g["x"] - ref["gx"]) / field.delr[j], np.abs(g["y"] - ref["gy"]) / field.delc[i],
                            np.abs(g["z"] - ref["gz"]) / field.dz[k]])
    div = g["hash"] != ref["hash"]
    return np.where(div, np.inf, dt), np.where(div, np.inf, dx)


def check_mixed(ep, *, field, state, times=None, idx=None, t_stop=np.inf, c=4.0, runs=4, threads=8, label="",
                oracle_run=None, **track_kw):
    """Mixed precision against the FP64 oracle (plain arithmetic), particle
    by particle, calibrated by the problem's own sensitivity to rounding.

    The oracle is run ``runs`` more times with every crossing jittered by
    about one FP32 rounding (FP32_JITTER relative on the step time and the
    transverse offsets; oracle/mp_oracle.h).  s_i = the largest change of
    particle i's travel time (relative) and endpoint (cell widths) over those
    runs, +inf where a jittered run changes its cell sequence.  Every
    particle whose cell sequence matches the oracle's must satisfy
    |dt|/t <= max(1e-5, c s_i^t) and |dx| <= max(1e-4 cells, c s_i^x); the
    share of particles whose sequence differs may not exceed the jittered
    runs' mean share plus 0.5 %.  ``oracle_run(**jitter_kw)`` replaces the
    default oracle call (track_parallel over ``state``) where the run is
    another (flow periods).  Returns the report (also printed)."""
    import oracle as O
    if oracle_run is None:
        def oracle_run(**jk):
            return O.track_parallel(field, state, threads, times=times, t_stop=t_stop, **track_kw, **jk)
    ref = oracle_run()
    dt, dx = mixed_errors(ep, ref, field, idx)
    s_t = np.zeros(dt.size)
    s_x = np.zeros(dt.size)
    div_j = []
    for r in range(runs):
        rj = oracle_run(jitter=FP32_JITTER, jitter_seed=1000 + r)
        jt, jx = mixed_errors({"hash": rj["hash"], "t": rj["t"], "x": rj["gx"], "y": rj["gy"], "z": rj["gz"]},
                              ref, field)
        s_t = np.maximum(s_t, jt)
        s_x = np.maximum(s_x, jx)
        div_j.append(float(np.isinf(jt).mean()))
    same = np.isfinite(dt)
    bad_t = np.nonzero(same & ~(dt <= np.maximum(1e-5, c * s_t)))[0]
    bad_x = np.nonzero(same & ~(dx <= np.maximum(1e-4, c * s_x)))[0]
    q = lambda a, v: float(np.quantile(a, v)) if a.size else 0.0
    rep = {"particles": int(dt.size), "divergent": float(1.0 - same.mean()), "jittered_divergent": float(np.mean(div_j)),
           "t_median": q(dt[same], 0.5), "t_p99": q(dt[same], 0.99), "t_max": q(dt[same], 1.0),
           "within_1e-5": float(np.mean(dt[same] <= 1e-5)) if same.any() else 1.0,
           "x_median": q(dx[same], 0.5), "x_p99": q(dx[same], 0.99),
           "within_1e-4": float(np.mean(dx[same] <= 1e-4)) if same.any() else 1.0,
           "bound_fail_t": int(bad_t.size), "bound_fail_x": int(bad_x.size)}
    print(f"mixed vs oracle {label}: " + ", ".join(f"{k} {v:.3g}" if isinstance(v, float) else f"{k} {v}"
                                                  for k, v in rep.items()))
    assert bad_t.size == 0, f"{bad_t.size} particles beyond max(1e-5, {c} s_i) in time, first {bad_t[:5]}: " \
                            f"{dt[bad_t[:5]]} vs s_i {s_t[bad_t[:5]]}"
    assert bad_x.size == 0, f"{bad_x.size} particles beyond max(1e-4, {c} s_i) in position, first {bad_x[:5]}"
    assert rep["divergent"] <= rep["jittered_divergent"] + 0.005
    return rep
