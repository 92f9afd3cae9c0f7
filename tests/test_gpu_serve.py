"""Serving loop: requests admitted while others run give the same results as
alone and as the oracle; their batches run at the same time on the device;
admission respects the memory budget and the in-flight cap."""
import numpy as np
import pytest

import oracle as O
from paper_2302_13590_gb300 import inputs as I
from paper_2302_13590_gb300 import mp
from paper_2302_13590_gb300 import serve as S
from tests import gpu_common as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    ctx = mp.Context(0)
    fields = {"cfg1": ctx.field(I.cfg1_field()), "cfg2": ctx.field(I.cfg2_field())}
    yield torch, ctx, fields
    ctx.close()


@pytest.mark.parametrize("precision", [mp.PREC_MIXED, mp.PREC_FP64])
def test_served_results_equal_alone(setup, precision):
    torch, ctx, fields = setup
    specs = I.serving_workload(n_req=30, rate_hz=2000.0, n_min=1e2, n_max=2e4, seed=91)
    srv = S.Server(ctx, fields, precision=precision, max_inflight=6, keep_results={id(s) for s in specs})
    # the default budget is a share of the free device memory
    free, total = torch.cuda.mem_get_info()
    assert 0 < srv.budget <= total and abs(srv.budget - 0.8 * free) <= 0.05 * total
    rep = srv.run(specs, realtime=True)
    summ = rep.summary()
    assert summ["requests"] == 30 and summ["p50_ms"] <= summ["p99_ms"]
    assert rep.max_inflight <= 6 and rep.batches >= 5
    for s in specs:
        served = srv.results[id(s)]
        alone = S.Server(ctx, fields, precision=precision, keep_results={id(s)})
        alone.run([s], realtime=False)
        ref = alone.results[id(s)]
        for k in served:
            assert np.array_equal(served[k], ref[k], equal_nan=True), k
    # and against the oracle, on up to 300 particles of every request: FP64
    # bit-exact with the mirror arithmetic and within 1e-10 of the plain one,
    # mixed precision within its per-particle bound
    rng = np.random.default_rng(5)
    for s in specs:
        served = srv.results[id(s)]
        f = I.cfg1_field() if s.field_name == "cfg1" else I.cfg2_field()
        n = s.release.n
        idx = np.sort(rng.choice(n, min(n, 300), replace=False))
        st0 = O.subset(O.release_box(f, n, s.release.lo, s.release.hi, s.release.seed, s.release.id_offset), idx)
        times = s.times if s.timeseries else None
        label = f"served request ({s.field_name}, {n} particles)"
        if precision == mp.PREC_FP64:
            G.compare_fp64(served, O.track(f, st0, times=times, arith="mirror"), idx=idx, dmin=G.dmin(f))
            G.compare_fp64_plain(served, O.track(f, st0, times=times), field=f, state=st0, idx=idx, times=times,
                                 label=label)
        else:
            G.check_mixed(served, field=f, state=st0, times=times, idx=idx, label=label)


def test_memory_budget_limits_inflight(setup):
    torch, ctx, fields = setup
    specs = I.serving_workload(n_req=12, rate_hz=1e6, n_min=2e4, n_max=2e4, seed=92)
    one = max(S.Server(ctx, fields)._bytes(s) for s in specs)
    srv = S.Server(ctx, fields, memory_budget=int(2.5 * one))
    rep = srv.run(specs, realtime=False)
    summ = rep.summary()
    assert summ["peak_bytes"] <= summ["budget_bytes"]
    assert summ["requests"] == 12
    # with equal requests the budget admits two at a time
    for s in specs:
        s.timeseries, s.times = False, None
    one = S.Server(ctx, fields)._bytes(specs[0])
    rep = S.Server(ctx, fields, memory_budget=int(2.5 * one)).run(specs, realtime=False)
    assert rep.max_inflight <= 2


@pytest.mark.parametrize("precision", [mp.PREC_MIXED, mp.PREC_FP64])
def test_batches_overlap_on_the_device(setup, precision):
    """Continuous batching overlaps work on the GPU: requests arriving while
    others run go out as new batches on other streams, and their tracking
    launches execute at the same time.  Each launch records its window on the
    device's global timer (earliest block start, latest block end); at least
    two batches' windows must be open at one instant.  The requests are
    large enough (3e4 to 1e5 particles) that a batch's kernel outlasts the
    host's turn around the loop that launches the next one, in either
    precision."""
    torch, ctx, fields = setup
    specs = I.serving_workload(n_req=60, rate_hz=20000.0, n_min=3e4, n_max=1e5, seed=93)
    srv = S.Server(ctx, fields, precision=precision)
    rep = srv.run(specs, realtime=True)
    summ = rep.summary()
    print(f"served {summ['requests']} in {summ['batches']} batches: max concurrent on the device "
          f"{summ['max_concurrent_batches']}, concurrency {summ['device_concurrency']:.2f}")
    assert len(srv.windows) == summ["batches"]
    assert all(e > b for b, e in srv.windows)
    assert summ["max_concurrent_batches"] >= 2 and summ["device_concurrency"] > 1.0
