"""The tracking entry point that allocates no device memory.

mp_track_noalloc is for callers that cannot allocate device memory where
they track: code that runs inside a memory budget it does not control (an
embedding application that hands out one fixed arena and forbids further
cudaMalloc), or code that must not let a library grow the device's memory
pool.  They pass every buffer themselves; the call's only other device
memory is a small static array inside the library.  Here its results are
compared with mp_track's on the same particles, on two calls in a row (the
second call reuses the static array the first one left behind), with and
without a wait for statistics; the device's free memory and torch's reserved
pool must not shrink across the calls.
"""
import numpy as np
import pytest

from paper_2302_13590_gb300 import inputs as I
from paper_2302_13590_gb300 import mp
from tests import gpu_common as G

pytestmark = pytest.mark.gpu


def _device_state(torch, ep):
    st = np.where(ep["status"] == mp.ST_TIME, mp.ST_ACTIVE, ep["status"]).astype(np.uint8)
    return {"cell": torch.from_numpy(ep["cell"].copy()).cuda(),
            "px": torch.from_numpy(ep["px"].copy()).cuda(),
            "py": torch.from_numpy(ep["py"].copy()).cuda(),
            "pz": torch.from_numpy(ep["pz"].copy()).cuda(),
            "t": torch.zeros(ep["cell"].size, dtype=torch.float64, device="cuda"),
            "status": torch.from_numpy(st).cuda()}


def _device_out(torch, n):
    tdt = {np.int32: torch.int32, np.float64: torch.float64, np.uint8: torch.uint8, np.uint32: torch.int32,
           np.uint64: torch.int64}
    return {k: torch.empty(n, dtype=tdt[dt], device="cuda") for k, dt in mp.ENDPOINT_DTYPES.items()}


def _host(out):
    h = {}
    for k, dt in mp.ENDPOINT_DTYPES.items():
        h[k] = out[k].cpu().numpy().view(dt)
    return h


@pytest.mark.parametrize("precision,flags,wsf", [(mp.PREC_FP64, 0, 0.0), (mp.PREC_MIXED, 0, 0.0),
                                                 (mp.PREC_FP64, mp.TRACK_PASS_WEAK_SINKS, 0.5)])
def test_noalloc_matches_track(precision, flags, wsf):
    torch = pytest.importorskip("torch")
    w = I.workload("cfg1")
    with mp.Context(0) as ctx:
        fh = ctx.field(w.field)
        gh = ctx.release_box(fh, w.release.n, w.release.lo, w.release.hi, w.release.seed)
        r0 = ctx.track(gh, t_stop=0.0, schedule=mp.SCHED_STATIC)
        ep0 = r0.endpoints()
        r0.free()
        ref_req = ctx.track(gh, mode=mp.MODE_ENDPOINT | mp.MODE_TIMESERIES, precision=precision,
                            schedule=mp.SCHED_DYNAMIC, times=w.times, flags=flags, weak_sink_fraction=wsf)
        ref = ref_req.endpoints()
        ref_ts = ref_req.timeseries()
        ref_st = ref_req.stats()
        ref_req.free()
        n, nt = w.release.n, len(w.times)
        state = _device_state(torch, ep0)
        opts = mp.make_opts(mode=mp.MODE_ENDPOINT | mp.MODE_TIMESERIES, precision=precision,
                            schedule=mp.SCHED_DYNAMIC, times=w.times, flags=flags, weak_sink_fraction=wsf)
        for call in range(2):
            out = _device_out(torch, n)
            ts = torch.empty(nt * n * 32, dtype=torch.uint8, device="cuda")
            st = mp.mp_track_noalloc(fh, state, out, ts=ts, opts=opts)
            got = _host(out)
            got_ts = ts.cpu().numpy().view(mp.TS_RECORD).reshape(nt, n)
            assert st["cell_steps"] == ref_st["cell_steps"], call
            assert st["n_status"] == ref_st["n_status"], call
            assert st["device_error"] == 0
            ref_o = dict(ref, gx=ref["x"], gy=ref["y"], gz=ref["z"])
            G.compare_fp64(got, ref_o, rtol=1e-10, dmin=G.dmin(w.field))
            ref_ts_o = {"ts_x": ref_ts["x"], "ts_y": ref_ts["y"], "ts_z": ref_ts["z"], "ts_cell": ref_ts["cell"],
                        "ts_status": ref_ts["status"]}
            G.compare_timeseries_fp64(got_ts, ref_ts_o, rtol=1e-10, dmin=G.dmin(w.field))
        mp.mp_group_free(gh)


def test_noalloc_rejects_too_many_times():
    torch = pytest.importorskip("torch")
    w = I.workload("cfg1")
    with mp.Context(0) as ctx:
        fh = ctx.field(w.field)
        n = 4
        state = {"cell": torch.zeros(n, dtype=torch.int32, device="cuda"),
                 "px": torch.zeros(n, dtype=torch.float64, device="cuda"),
                 "py": torch.zeros(n, dtype=torch.float64, device="cuda"),
                 "pz": torch.zeros(n, dtype=torch.float64, device="cuda"),
                 "t": torch.zeros(n, dtype=torch.float64, device="cuda"),
                 "status": torch.zeros(n, dtype=torch.uint8, device="cuda")}
        out = _device_out(torch, n)
        times = np.linspace(1.0, 2.0, mp.NOALLOC_MAX_TIMES + 1)
        ts = torch.empty(times.size * n * 32, dtype=torch.uint8, device="cuda")
        opts = mp.make_opts(mode=mp.MODE_TIMESERIES, times=times)
        with pytest.raises(mp.MPError) as e:
            mp.mp_track_noalloc(fh, state, out, ts=ts, opts=opts)
        assert e.value.code == -1 and "MP_NOALLOC_MAX_TIMES" in str(e.value)


def _ref_run(ctx, fh, w, precision, t_stop=np.inf, flags=0):
    gh = ctx.release_box(fh, w.release.n, w.release.lo, w.release.hi, w.release.seed)
    r0 = ctx.track(gh, t_stop=0.0, schedule=mp.SCHED_STATIC)
    ep0 = r0.endpoints()
    r0.free()
    req = ctx.track(gh, mode=mp.MODE_ENDPOINT | mp.MODE_TIMESERIES, precision=precision, schedule=mp.SCHED_DYNAMIC,
                    times=w.times, t_stop=t_stop, flags=flags)
    ref, ref_ts = req.endpoints(), req.timeseries()
    req.free()
    return gh, ep0, ref, ref_ts


def _check(got, got_ts, ref, ref_ts, field):
    G.compare_fp64(got, dict(ref, gx=ref["x"], gy=ref["y"], gz=ref["z"]), rtol=1e-10, dmin=G.dmin(field))
    G.compare_timeseries_fp64(got_ts, {"ts_x": ref_ts["x"], "ts_y": ref_ts["y"], "ts_z": ref_ts["z"],
                                       "ts_cell": ref_ts["cell"], "ts_status": ref_ts["status"]},
                              rtol=1e-10, dmin=G.dmin(field))


@pytest.mark.parametrize("precision", [mp.PREC_FP64, mp.PREC_MIXED])
def test_noalloc_enqueue_only_back_to_back(precision):
    """Two calls that only enqueue (no statistics, so no wait) on one stream,
    one right after the other: the second call clears what the first left in
    the static array only in stream order.  Nothing is allocated meanwhile."""
    torch = pytest.importorskip("torch")
    w = I.workload("cfg1")
    with mp.Context(0) as ctx:
        fh = ctx.field(w.field)
        gh, ep0, ref, ref_ts = _ref_run(ctx, fh, w, precision)
        n, nt = w.release.n, len(w.times)
        opts = mp.make_opts(mode=mp.MODE_ENDPOINT | mp.MODE_TIMESERIES, precision=precision,
                            schedule=mp.SCHED_DYNAMIC, times=w.times)
        state = _device_state(torch, ep0)
        outs = [_device_out(torch, n) for _ in range(3)]
        tss = [torch.empty(nt * n * 32, dtype=torch.uint8, device="cuda") for _ in range(3)]
        stream = torch.cuda.Stream()
        # a first call takes the static array's address (once per device)
        mp.mp_track_noalloc(fh, state, outs[2], ts=tss[2], opts=opts, stream=stream, want_stats=False)
        torch.cuda.synchronize()
        free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
        for c in range(2):
            assert mp.mp_track_noalloc(fh, state, outs[c], ts=tss[c], opts=opts, stream=stream,
                                       want_stats=False) is None
        stream.synchronize()
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] >= free0
        assert torch.cuda.memory_reserved() == reserved0
        for c in range(2):
            got = _host(outs[c])
            got_ts = tss[c].cpu().numpy().view(mp.TS_RECORD).reshape(nt, n)
            _check(got, got_ts, ref, ref_ts, w.field)
        mp.mp_group_free(gh)


def test_noalloc_update_group_writes_the_state_back():
    """MP_TRACK_UPDATE_GROUP: the caller's state arrays receive the
    endpoints (TIME turned back into ACTIVE), and a second call continues
    from them as mp_track continues a group."""
    torch = pytest.importorskip("torch")
    w = I.workload("cfg1")
    T1, T2 = 0.2 * w.t_adv, 0.7 * w.t_adv
    with mp.Context(0) as ctx:
        fh = ctx.field(w.field)
        gh = ctx.release_box(fh, w.release.n, w.release.lo, w.release.hi, w.release.seed)
        r0 = ctx.track(gh, t_stop=0.0, schedule=mp.SCHED_STATIC)
        ep0 = r0.endpoints()
        r0.free()
        ra = ctx.track(gh, t_stop=T1, flags=mp.TRACK_UPDATE_GROUP)
        ra.wait()
        rb = ctx.track(gh, t_stop=T2, flags=mp.TRACK_UPDATE_GROUP)
        ref_a, ref_b = ra.endpoints(), rb.endpoints()
        ra.free()
        rb.free()
        n = w.release.n
        state = _device_state(torch, ep0)
        for T, ref in ((T1, ref_a), (T2, ref_b)):
            out = _device_out(torch, n)
            opts = mp.make_opts(t_stop=T, flags=mp.TRACK_UPDATE_GROUP)
            st = mp.mp_track_noalloc(fh, state, out, opts=opts)
            assert st["device_error"] == 0
            got = _host(out)
            # (the caller's state carries no step count, hash or last exit
            # face, so only the first stage's exit faces are comparable)
            for k in ("cell", "status") + (("exit_face",) if T == T1 else ()):
                assert np.array_equal(got[k], ref[k]), k
            for k in ("t", "x", "y", "z"):
                assert np.max(G.rel_err(got[k], ref[k], scale=np.maximum(np.abs(ref[k]), 1.0))) <= 1e-10, k
            # the caller's state now holds the endpoints
            assert np.array_equal(state["cell"].cpu().numpy(), got["cell"])
            for k in ("px", "py", "pz", "t"):
                assert np.array_equal(state[k].cpu().numpy(), got[k]), k
            resumed = np.where(got["status"] == mp.ST_TIME, mp.ST_ACTIVE, got["status"])
            assert np.array_equal(state["status"].cpu().numpy(), resumed)
        mp.mp_group_free(gh)


def test_noalloc_refuses_a_capturing_stream():
    """The call copies host memory that does not outlive it, so it refuses a
    stream that is being captured (nothing is enqueued, nothing is replayed)."""
    torch = pytest.importorskip("torch")
    w = I.workload("cfg1")
    with mp.Context(0) as ctx:
        fh = ctx.field(w.field)
        n = 8
        state = {"cell": torch.zeros(n, dtype=torch.int32, device="cuda"),
                 "px": torch.zeros(n, dtype=torch.float64, device="cuda"),
                 "py": torch.zeros(n, dtype=torch.float64, device="cuda"),
                 "pz": torch.zeros(n, dtype=torch.float64, device="cuda"),
                 "t": torch.zeros(n, dtype=torch.float64, device="cuda"),
                 "status": torch.zeros(n, dtype=torch.uint8, device="cuda")}
        out = _device_out(torch, n)
        opts = mp.make_opts()
        stream = torch.cuda.Stream()
        torch.cuda.synchronize()
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        err = None
        with torch.cuda.stream(stream):
            g.capture_begin(capture_error_mode="relaxed")
            try:
                mp.mp_track_noalloc(fh, state, out, opts=opts, stream=stream, want_stats=False)
            except mp.MPError as e:
                err = e
            finally:
                g.capture_end()
        del g
        assert err is not None and err.code == -1 and "capturing" in str(err)



def test_noalloc_at_the_maximum_number_of_times():
    """Exactly MP_NOALLOC_MAX_TIMES output times (the largest request the
    static array holds) give mp_track's records."""
    torch = pytest.importorskip("torch")
    w = I.workload("cfg1", n_particles=97)
    times = np.linspace(0.0, 2.0 * w.t_adv, mp.NOALLOC_MAX_TIMES)
    with mp.Context(0) as ctx:
        fh = ctx.field(w.field)
        gh = ctx.release_box(fh, w.release.n, w.release.lo, w.release.hi, w.release.seed)
        r0 = ctx.track(gh, t_stop=0.0, schedule=mp.SCHED_STATIC)
        ep0 = r0.endpoints()
        r0.free()
        req = ctx.track(gh, mode=mp.MODE_ENDPOINT | mp.MODE_TIMESERIES, times=times)
        ref, ref_ts = req.endpoints(), req.timeseries()
        req.free()
        n, nt = w.release.n, times.size
        out = _device_out(torch, n)
        ts = torch.empty(nt * n * 32, dtype=torch.uint8, device="cuda")
        st = mp.mp_track_noalloc(fh, _device_state(torch, ep0), out, ts=ts,
                                 opts=mp.make_opts(mode=mp.MODE_ENDPOINT | mp.MODE_TIMESERIES, times=times))
        assert st["device_error"] == 0
        _check(_host(out), ts.cpu().numpy().view(mp.TS_RECORD).reshape(nt, n), ref, ref_ts, w.field)
        mp.mp_group_free(gh)
