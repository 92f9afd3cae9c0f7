"""Batched launches: many requests in one launch give each request exactly
the result it gets alone (per-particle arithmetic does not depend on which
lane or launch carries it), and the batch matches the oracle on samples."""
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


def _opts(spec, precision, schedule):
    mode = mp.MODE_ENDPOINT | (mp.MODE_TIMESERIES if spec.timeseries else 0)
    return mp.make_opts(mode=mode, precision=precision, schedule=schedule, times=spec.times)


def _run_batch(ctx, fh, specs, precision, schedule):
    groups = [mp.mp_release_group(ctx.h, fh, n=s.release.n, lo=s.release.lo, hi=s.release.hi, seed=s.release.seed)
              for s in specs]
    opts = [_opts(s, precision, schedule) for s in specs]
    ids = mp.mp_track_batch(ctx.h, groups, opts)
    out = []
    for s, rid in zip(specs, ids):
        mp.mp_wait(ctx.h, rid)
        ep = mp.mp_get_endpoints(ctx.h, rid, s.release.n)
        ts = mp.mp_get_timeseries(ctx.h, rid, s.release.n, len(s.times)) if s.timeseries else None
        st = mp.mp_get_stats(ctx.h, rid)
        mp.mp_req_free(ctx.h, rid)
        out.append((ep, ts, st))
    for g in groups:
        mp.mp_group_free(g)
    return out


@pytest.mark.parametrize("precision,schedule", [(mp.PREC_FP64, mp.SCHED_DYNAMIC), (mp.PREC_MIXED, mp.SCHED_DYNAMIC),
                                                (mp.PREC_MIXED, mp.SCHED_STATIC)])
def test_batch_equals_alone(ctx, precision, schedule):
    specs = I.batch_workload(n_req=24, n_min=1, n_max=3e3, seed=77)
    fh = ctx.field(I.cfg2_field())
    batch = _run_batch(ctx, fh, specs, precision, schedule)
    for s, (ep, ts, st) in zip(specs, batch):
        alone = _run_batch(ctx, fh, [s], precision, schedule)[0]
        for k in ep:
            assert np.array_equal(ep[k], alone[0][k], equal_nan=True), k
        if s.timeseries:
            assert np.array_equal(ts.view(np.uint8), alone[1].view(np.uint8))
        assert st["cell_steps"] == alone[2]["cell_steps"]
        assert st["n_status"] == alone[2]["n_status"]
    mp.mp_field_free(fh)


def test_batch_mixed_precisions_and_oracle(ctx):
    """FP64 and mixed requests in one call (two launches); FP64 ones match
    the oracle exactly on their cell sequences."""
    specs = I.batch_workload(n_req=10, n_min=10, n_max=2e3, seed=78)
    f = I.cfg2_field()
    fh = ctx.field(f)
    groups = [mp.mp_release_group(ctx.h, fh, n=s.release.n, lo=s.release.lo, hi=s.release.hi, seed=s.release.seed)
              for s in specs]
    precs = [mp.PREC_FP64 if i % 3 else mp.PREC_MIXED for i in range(len(specs))]
    opts = [_opts(s, p, mp.SCHED_DYNAMIC) for s, p in zip(specs, precs)]
    ids = mp.mp_track_batch(ctx.h, groups, opts)
    for s, p, rid in zip(specs, precs, ids):
        ep = mp.mp_get_endpoints(ctx.h, rid, s.release.n)
        st0 = O.release_box(f, s.release.n, s.release.lo, s.release.hi, s.release.seed)
        ref = O.track(f, st0, times=s.times, arith="mirror")
        if p == mp.PREC_FP64:
            G.compare_fp64(ep, ref, dmin=G.dmin(f))
            if s.timeseries:
                G.compare_timeseries_fp64(mp.mp_get_timeseries(ctx.h, rid, s.release.n, len(s.times)), ref,
                                          dmin=G.dmin(f))
        else:
            G.check_mixed(ep, field=f, state=st0, times=s.times, label=f"batch request {rid}")
        mp.mp_req_free(ctx.h, rid)
    for g in groups:
        mp.mp_group_free(g)
    mp.mp_field_free(fh)


def test_batch_256_requests_full_size(ctx):
    """The 256-request workload (sizes log-uniform in 1e2..1e6, half with 20
    output times) in one persistent mixed-precision launch: every request's
    counters are consistent and sampled particles of a few requests meet the
    mixed-precision per-particle bound against the oracle."""
    specs = I.batch_workload()
    f = I.cfg2_field()
    fh = ctx.field(f)
    groups = [mp.mp_release_group(ctx.h, fh, n=s.release.n, lo=s.release.lo, hi=s.release.hi, seed=s.release.seed)
              for s in specs]
    opts = [_opts(s, mp.PREC_MIXED, mp.SCHED_DYNAMIC) for s in specs]
    ids = mp.mp_track_batch(ctx.h, groups, opts)
    total = 0
    rng = np.random.default_rng(3)
    for r, (s, rid) in enumerate(zip(specs, ids)):
        st = mp.mp_get_stats(ctx.h, rid)
        assert st["device_error"] == 0
        assert sum(st["n_status"]) == s.release.n
        total += s.release.n
        if r % 64 == 0:
            ep = mp.mp_get_endpoints(ctx.h, rid, s.release.n)
            assert int(ep["steps"].astype(np.int64).sum()) == st["cell_steps"]
            idx = np.sort(rng.choice(s.release.n, min(200, s.release.n), replace=False))
            st0 = O.release_box(f, s.release.n, s.release.lo, s.release.hi, s.release.seed)
            G.check_mixed(ep, field=f, state=O.subset(st0, idx), times=s.times, idx=idx, label=f"request {r}")
        mp.mp_req_free(ctx.h, rid)
    assert total > 1e7
    for g in groups:
        mp.mp_group_free(g)
    mp.mp_field_free(fh)
