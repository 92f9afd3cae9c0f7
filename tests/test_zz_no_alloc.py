"""The tracking entry point that allocates no device memory.

mp_track_noalloc is for callers that cannot allocate device memory where
they track (a fixed arena handed out by an embedding application, a CUDA
stream capture, a path that must not synchronise the device).  They pass
every buffer themselves; the call's only other device memory is a small
static array inside the library.  Here its results are compared with
mp_track's on the same particles, on two calls in a row (the second call
reuses the static array the first one left behind).
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
