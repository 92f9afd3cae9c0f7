"""Host-to-host tracking with overlapped transfers (mp_track_host): the
chunked, two-stream call gives the results of one release + track + copy
over all particles, bit for bit, for any chunk count (ragged last chunk,
more chunks than particles), both precisions, per-particle release times,
page-locked and pageable host buffers; FP64 results also match the oracle."""
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
def case(ctx):
    f = I.random_box_field(4, 10, 14, seed=91, lnk_var=1.5, n_wells=2, n_inactive=2)
    fh = ctx.field(f)
    cells, frac = I.explicit_particles(f, 3001, seed=12, cols=(1, 5))
    t0 = np.random.default_rng(3).uniform(0.0, 50.0, cells.size)
    full = O.track(f, _oracle_state(f, cells, frac, t0), arith="mirror")
    times = np.quantile(full["t"], [0.1, 0.4, 0.8, 0.97])
    yield f, fh, cells, frac, t0, times
    mp.mp_field_free(fh)


def _oracle_state(f, cells, frac, t0):
    st = O.release_explicit(f, cells, frac)
    st["t"] = np.asarray(t0, np.float64).copy()
    return st


def _one_request(ctx, fh, cells, frac, t0, opts):
    gh = mp.mp_release_group(ctx.h, fh, cell=cells, local=frac, t0=t0)
    rid = mp.mp_track(ctx.h, gh, opts)
    ep = mp.mp_get_endpoints(ctx.h, rid, cells.size)
    ts = mp.mp_get_timeseries(ctx.h, rid, cells.size, opts.n_times) if opts.n_times else None
    st = mp.mp_get_stats(ctx.h, rid)
    mp.mp_req_free(ctx.h, rid)
    mp.mp_group_free(gh)
    return ep, ts, st


@pytest.mark.parametrize("precision", [mp.PREC_FP64, mp.PREC_MIXED])
@pytest.mark.parametrize("n_chunks", [1, 2, 7, 0, 5000])
def test_host_call_equals_one_request(ctx, case, precision, n_chunks):
    f, fh, cells, frac, t0, times = case
    opts = mp.make_opts(mode=mp.MODE_ENDPOINT | mp.MODE_TIMESERIES, precision=precision, times=times)
    ref_ep, ref_ts, ref_st = _one_request(ctx, fh, cells, frac, t0, opts)
    ep, ts, st = mp.mp_track_host(ctx.h, fh, cells, frac, opts, t0=t0, n_chunks=n_chunks)
    for k in ref_ep:
        assert np.array_equal(ep[k], ref_ep[k], equal_nan=True), k
    assert ts.tobytes() == ref_ts.tobytes()
    assert st["cell_steps"] == ref_st["cell_steps"] and st["n_status"] == ref_st["n_status"]
    assert st["device_error"] == 0 and st["kernel_ms"] > 0
    if precision == mp.PREC_FP64:
        ref = O.track(f, _oracle_state(f, cells, frac, t0), times=times, arith="mirror")
        G.compare_fp64(ep, ref, dmin=G.dmin(f))
        G.compare_timeseries_fp64(ts, ref, dmin=G.dmin(f))


def test_host_call_pinned_buffers_and_endpoint_mode(ctx, case):
    import torch
    f, fh, cells, frac, t0, times = case
    n = cells.size
    opts = mp.make_opts(mode=mp.MODE_ENDPOINT, precision=mp.PREC_FP64)
    ref_ep, _, _ = _one_request(ctx, fh, cells, frac, None, opts)
    def pinned(count, dt):
        return torch.empty(count * np.dtype(dt).itemsize, dtype=torch.uint8, pin_memory=True).numpy().view(dt)

    out = {k: pinned(n, dt) for k, dt in mp.ENDPOINT_DTYPES.items()}
    cell_p = pinned(n, np.int32)
    local_p = pinned(3 * n, np.float64)
    cell_p[:] = cells
    local_p[:] = frac.reshape(-1)
    ep, ts, st = mp.mp_track_host(ctx.h, fh, cell_p, local_p, opts, n_chunks=3, out=out)
    assert ts is None and ep is out
    for k in ref_ep:
        assert np.array_equal(ep[k], ref_ep[k], equal_nan=True), k
    # a NULL endpoint array is skipped
    part = {"cell": np.empty(n, np.int32), "t": np.empty(n)}
    ep2, _, _ = mp.mp_track_host(ctx.h, fh, cells, frac, opts, n_chunks=2, out=part)
    assert np.array_equal(ep2["cell"], ref_ep["cell"]) and np.array_equal(ep2["t"], ref_ep["t"])


def test_host_call_on_a_quadtree(ctx):
    """The host call on a quadtree grid (FP64, weak sinks with a threshold):
    equal to one request bit for bit, and to the oracle."""
    from paper_2302_13590_gb300.inputs import usg as U
    u = U.quadtree_field(2, 8, 12, seed=15, n_wells=3, well_rate=0.05)
    fu = ctx.field(u)
    cells, frac = U.explicit_particles(u, 1500, seed=8)
    st0 = O.release_explicit(u, cells, frac)
    times = np.quantile(O.track(u, st0, pass_weak_sinks=True, arith="mirror")["t"], [0.3, 0.7])
    opts = mp.make_opts(mode=mp.MODE_ENDPOINT | mp.MODE_TIMESERIES, times=times, flags=mp.TRACK_PASS_WEAK_SINKS,
                        weak_sink_fraction=0.5)
    ref_ep, ref_ts, _ = _one_request(ctx, fu, cells, frac, None, opts)
    ep, ts, st = mp.mp_track_host(ctx.h, fu, cells, frac, opts, n_chunks=4)
    for k in ref_ep:
        assert np.array_equal(ep[k], ref_ep[k], equal_nan=True), k
    assert ts.tobytes() == ref_ts.tobytes()
    ref = O.track(u, st0, times=times, pass_weak_sinks=True, weak_sink_fraction=0.5, arith="mirror")
    G.compare_fp64(ep, ref, dmin=u.extent)
    G.compare_timeseries_fp64(ts, ref, dmin=u.extent)
    mp.mp_field_free(fu)


def test_host_call_rejections_and_empty(ctx, case):
    f, fh, cells, frac, t0, times = case
    with pytest.raises(mp.MPError) as e:
        mp.mp_track_host(ctx.h, fh, cells, frac, mp.make_opts(mode=mp.MODE_ENDPOINT | mp.MODE_PATHLINE,
                                                              path_capacity=1000))
    assert e.value.code == mp.ERR_INVALID_ARG
    bad = frac.copy()
    bad[5, 1] = np.nan
    with pytest.raises(mp.MPError) as e:
        mp.mp_track_host(ctx.h, fh, cells, bad, mp.make_opts())
    assert e.value.code == mp.ERR_NONFINITE
    ep, ts, st = mp.mp_track_host(ctx.h, fh, np.zeros(0, np.int32), np.zeros((0, 3)), mp.make_opts())
    assert ep["cell"].size == 0 and st["cell_steps"] == 0
    # the context stays usable after the rejected calls
    ep, _, st = mp.mp_track_host(ctx.h, fh, cells[:10], frac[:10], mp.make_opts())
    assert st["device_error"] == 0 and sum(st["n_status"]) == 10
