"""The serving loop's host logic on the CPU, with the library calls and the
device queries replaced by fakes: requests are admitted in arrival order,
within the memory budget and the in-flight cap (a request larger than the
whole budget still runs, alone), batched per field, and every group and
request is freed once; the report adds up."""
from collections import namedtuple

import numpy as np
import pytest

from paper_2302_13590_gb300 import inputs as I
from paper_2302_13590_gb300 import mp
from paper_2302_13590_gb300 import serve as SV

Spec = namedtuple("Spec", "release field_name timeseries times arrival_s")


class FakeTorch:
    class cuda:
        @staticmethod
        def mem_get_info():
            return (10_000_000, 20_000_000)

        class Stream:
            pass


class FakeLib:
    """Records the calls the server makes; a request completes on its
    third poll."""

    def __init__(self):
        self.released = []       # (field handle, n) in call order
        self.batches = []        # [(field handles of the batch)]
        self.polls = {}
        self.freed_req, self.freed_grp = [], []
        self.next_id = 1
        self.live_bytes = 0

    def query_bytes(self, opts, n):
        return 1000 * int(n)

    def release_group(self, ctx, fh, n=None, **kw):
        g = {"fh": fh, "n": int(n), "id": len(self.released)}
        self.released.append((fh, int(n)))
        return g

    def track_batch(self, ctx, groups, opts, stream):
        assert len({id(g["fh"]) for g in groups}) == 1     # one field per batch
        self.batches.append([g["fh"] for g in groups])
        # a launch window per batch: batch k runs on the device from 100 k to
        # 100 k + 250 (ns), so neighbouring batches overlap
        k = len(self.batches) - 1
        ids = []
        for g in groups:
            rid = self.next_id
            self.next_id += 1
            self.polls[rid] = [0, g["n"], (1000 + 100 * k, 1250 + 100 * k)]
            ids.append(rid)
        return ids

    def query(self, ctx, rid):
        self.polls[rid][0] += 1
        return self.polls[rid][0] >= 3

    def get_stats(self, ctx, rid):
        b, e = self.polls[rid][2]
        return {"device_error": 0, "cell_steps": 10 * self.polls[rid][1], "t_begin_ns": b, "t_end_ns": e}

    def req_free(self, ctx, rid):
        self.freed_req.append(rid)

    def group_free(self, g):
        self.freed_grp.append(g["id"])


@pytest.fixture()
def fake(monkeypatch):
    lib = FakeLib()
    monkeypatch.setattr(mp, "mp_query_bytes", lib.query_bytes)
    monkeypatch.setattr(mp, "mp_release_group", lib.release_group)
    monkeypatch.setattr(mp, "mp_track_batch", lib.track_batch)
    monkeypatch.setattr(mp, "mp_query", lib.query)
    monkeypatch.setattr(mp, "mp_get_stats", lib.get_stats)
    monkeypatch.setattr(mp, "mp_req_free", lib.req_free)
    monkeypatch.setattr(mp, "mp_group_free", lib.group_free)
    monkeypatch.setattr(mp, "mp_get_endpoints", lambda *a, **k: {"ok": True})
    return lib


class Ctx:
    h = object()


def _specs(ns, fields=("a", "b")):
    rng = np.random.default_rng(3)
    out = []
    for i, n in enumerate(ns):
        rel = I.Release(int(n), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), seed=i + 1)
        out.append(Spec(rel, fields[int(rng.integers(len(fields)))], bool(i % 2), [1.0, 2.0], 0.0))
    return out


def test_admission_order_budget_and_cap(fake):
    ns = [300, 200, 900, 100, 50, 400, 700, 100, 20, 600, 250, 80]
    specs = _specs(ns)
    fields = {"a": object(), "b": object()}
    budget = 1_500_000       # bytes: ~1000 B per particle + the group's share
    srv = SV.Server(Ctx(), fields, memory_budget=budget, max_inflight=3, torch_mod=FakeTorch)
    rep = srv.run(specs, realtime=False)
    # every request released once, in arrival order, on its own field
    assert [n for _, n in fake.released] == ns
    assert [fh for fh, _ in fake.released] == [fields[s.field_name] for s in specs]
    # every request and group freed once
    assert sorted(fake.freed_req) == list(range(1, len(ns) + 1))
    assert sorted(fake.freed_grp) == list(range(len(ns)))
    # the report
    assert rep.n_requests == len(ns)
    sm = rep.summary()
    assert sm["requests"] == len(ns)
    assert sm["max_inflight"] <= 3
    assert sm["peak_bytes"] <= budget
    assert sm["batches"] >= 1
    assert rep.cell_steps == 10 * sum(ns)


def test_request_larger_than_budget_runs_alone(fake):
    specs = _specs([100, 5000, 100], fields=("a",))
    srv = SV.Server(Ctx(), {"a": object()}, memory_budget=200_000, max_inflight=8, torch_mod=FakeTorch)
    rep = srv.run(specs, realtime=False)
    assert rep.summary()["requests"] == 3
    # the large one was admitted only with nothing else in flight: the
    # batches around it hold one request each
    sizes = [len(b) for b in fake.batches]
    assert sizes == [1, 1, 1]


def test_budget_defaults_to_a_share_of_free_memory():
    srv = SV.Server(Ctx(), {}, torch_mod=FakeTorch)
    assert srv.budget == int(0.8 * 10_000_000)
    srv = SV.Server(Ctx(), {}, free_share=0.5, torch_mod=FakeTorch)
    assert srv.budget == 5_000_000


def test_device_overlap_of_batch_windows(fake):
    """Per-batch launch windows (shared by a batch's requests) and their
    overlap: batch k holds [1000 + 100 k, 1250 + 100 k]."""
    specs = _specs([10] * 12, fields=("a",))
    srv = SV.Server(Ctx(), {"a": object()}, max_inflight=2, torch_mod=FakeTorch)
    rep = srv.run(specs, realtime=False)
    nb = len(fake.batches)
    assert srv.windows == [(1000 + 100 * k, 1250 + 100 * k) for k in range(nb)]
    sm = rep.summary()
    assert sm["max_concurrent_batches"] == min(3, nb)
    assert sm["device_concurrency"] == pytest.approx(250 * nb / (100 * (nb - 1) + 250))


def test_device_overlap_arithmetic():
    assert SV.device_overlap([]) == {"max_concurrent_batches": 0, "device_concurrency": 0.0}
    assert SV.device_overlap([(0, 10), (10, 20)])["max_concurrent_batches"] == 1
    r = SV.device_overlap([(0, 10), (5, 15), (20, 30), (21, 22)])
    assert r["max_concurrent_batches"] == 2 and r["device_concurrency"] == pytest.approx(31 / 25)

