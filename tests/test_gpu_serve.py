"""Serving loop: requests admitted while others run give the same results as
alone; admission respects the memory budget and the in-flight cap."""
import numpy as np
import pytest

from paper_2302_13590_gb300 import inputs as I
from paper_2302_13590_gb300 import mp
from paper_2302_13590_gb300 import serve as S

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
