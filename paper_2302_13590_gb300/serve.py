"""Serving loop: continuous batching of particle-group tracking requests.

Requests (a box release on one of the device-resident fields, endpoint or
timeseries mode) arrive over time.  The loop, on the host:

* admits waiting requests in arrival order while the device-memory budget
  (bytes of group state + request outputs, from ``mp_query_bytes``) and the
  in-flight cap allow;
* launches everything admitted at one instant as one batch per field
  (``mp_track_batch``: one kernel over all their particles) on the next
  stream of a small pool, so batches admitted later run while earlier ones
  are still on the GPU;
* polls completions (``mp_query``, an event query, never a device-wide sync),
  stamps latency = completion - arrival, frees the request's memory and
  admits more.

This is the many-groups use the paper names as future work (Conclusions:
several particle groups, each with many particles), on one GPU.  Every
request's results are the same alone and in the mix: particles never
interact and each particle's arithmetic does not depend on its lane or its
launch (tested in tests/test_gpu_serve.py).
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field as dc_field
from typing import Dict, List, Optional

import numpy as np

from . import mp

# device bytes of a group's state per particle: cell, px/py/pz, t, status,
# steps, hash, exit face (+ alignment slack in the 4096 per request)
GROUP_BYTES_PER_PARTICLE = 4 + 24 + 8 + 1 + 4 + 8 + 1


@dataclass
class Served:
    spec: object
    arrival: float
    admitted: float = 0.0
    done: float = 0.0
    rid: int = -1
    group: object = None
    bytes: int = 0
    cell_steps: int = 0
    result: Optional[dict] = None
    batch: int = -1
    window_ns: tuple = (0, 0)   # its launch's window on the device's global timer


@dataclass
class ServeReport:
    n_requests: int
    wall_s: float
    particles: int
    cell_steps: int
    latency_ms: np.ndarray
    queue_ms: np.ndarray
    batches: int
    max_inflight: int
    extra: dict = dc_field(default_factory=dict)

    def summary(self) -> dict:
        lat = self.latency_ms
        return {"requests": self.n_requests, "wall_s": self.wall_s,
                "requests_per_s": self.n_requests / self.wall_s,
                "particles_per_s": self.particles / self.wall_s,
                "cell_steps_per_s": self.cell_steps / self.wall_s,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
                "queue_p50_ms": float(np.percentile(self.queue_ms, 50)),
                "queue_p99_ms": float(np.percentile(self.queue_ms, 99)),
                "batches": self.batches, "max_inflight": self.max_inflight, **self.extra}


def batch_windows(finished) -> List[tuple]:
    """(begin, end) of every batch's tracking launch on the device's global
    timer (ns), from its requests' stats; batches without a window (nothing
    launched) are left out."""
    w: Dict[int, tuple] = {}
    for s in finished:
        b, e = s.window_ns
        if s.batch < 0 or not b or not e:
            continue
        lo, hi = w.get(s.batch, (b, e))
        w[s.batch] = (min(lo, b), max(hi, e))
    return sorted(w.values())


def device_overlap(windows: List[tuple]) -> dict:
    """How much batches ran at the same time on the device: the largest
    number of launch windows open at one instant, and the sum of the
    windows' lengths over the length of their union (1: one at a time)."""
    if not windows:
        return {"max_concurrent_batches": 0, "device_concurrency": 0.0}
    ev = sorted([(b, 1) for b, _ in windows] + [(e, -1) for _, e in windows], key=lambda x: (x[0], x[1]))
    cur = top = 0
    for _, d in ev:
        cur += d
        top = max(top, cur)
    union = 0
    lo, hi = windows[0]
    for b, e in windows[1:]:
        if b > hi:
            union += hi - lo
            lo, hi = b, e
        else:
            hi = max(hi, e)
    union += hi - lo
    total = sum(e - b for b, e in windows)
    return {"max_concurrent_batches": top, "device_concurrency": total / union if union > 0 else 0.0}


class Server:
    """Continuous-batching request loop over loaded fields.

    fields: name -> mp field handle.  precision / schedule apply to every
    request.  memory_budget: bytes that requests in flight may hold; by
    default the given share of the device memory free when the server
    starts (admission by free device memory).
    """

    def __init__(self, ctx: mp.Context, fields: Dict[str, object], precision=mp.PREC_MIXED,
                 schedule=mp.SCHED_STATIC, n_streams: int = 4, max_inflight: int = 256,
                 memory_budget: Optional[int] = None, free_share: float = 0.8,
                 keep_results: Optional[set] = None, torch_mod=None):
        self.ctx = ctx
        self.fields = fields
        self.precision = precision
        self.schedule = schedule
        self.max_inflight = max_inflight
        self.keep = keep_results or set()
        if torch_mod is None:
            import torch as torch_mod  # streams and the free-memory query only
        if memory_budget is None:
            free, _ = torch_mod.cuda.mem_get_info()
            memory_budget = int(free_share * free)
        self.budget = memory_budget
        self.streams = [torch_mod.cuda.Stream() for _ in range(n_streams)]
        self._next_stream = 0

    def _opts(self, spec):
        mode = mp.MODE_ENDPOINT | (mp.MODE_TIMESERIES if spec.timeseries else 0)
        return mp.make_opts(mode=mode, precision=self.precision, schedule=self.schedule,
                            times=spec.times if spec.timeseries else None)

    def _bytes(self, spec) -> int:
        n = spec.release.n
        return mp.mp_query_bytes(self._opts(spec), n) + GROUP_BYTES_PER_PARTICLE * n + 4096

    def run(self, specs: List, realtime: bool = True, time_scale: float = 1.0) -> ServeReport:
        """Serve the requests; arrival times are honoured on the wall clock
        (scaled by time_scale) when realtime, else all arrive at once."""
        n = len(specs)
        waiting: deque = deque()
        inflight: List[Served] = []
        finished: List[Served] = []
        held = 0
        peak_bytes = 0
        batches = 0
        peak = 0
        nxt = 0
        t0 = time.perf_counter()
        while len(finished) < n:
            now = time.perf_counter() - t0
            while nxt < n and (not realtime or specs[nxt].arrival_s * time_scale <= now):
                arr = specs[nxt].arrival_s * time_scale if realtime else 0.0
                waiting.append(Served(specs[nxt], arr))
                nxt += 1
            # completions
            still = []
            for s in inflight:
                if mp.mp_query(self.ctx.h, s.rid):
                    s.done = time.perf_counter() - t0
                    st = mp.mp_get_stats(self.ctx.h, s.rid)
                    if st["device_error"]:
                        raise RuntimeError("tracking kernel raised its error flag")
                    s.cell_steps = st["cell_steps"]
                    s.window_ns = (st["t_begin_ns"], st["t_end_ns"])
                    if id(s.spec) in self.keep:
                        s.result = mp.mp_get_endpoints(self.ctx.h, s.rid, s.spec.release.n)
                    mp.mp_req_free(self.ctx.h, s.rid)
                    mp.mp_group_free(s.group)
                    held -= s.bytes
                    finished.append(s)
                else:
                    still.append(s)
            inflight = still
            # admission: arrival order, memory budget and slot cap
            admit: List[Served] = []
            while waiting and len(inflight) + len(admit) < self.max_inflight:
                b = self._bytes(waiting[0].spec)
                if held + b > self.budget and (inflight or admit):
                    break
                s = waiting.popleft()
                s.bytes = b
                held += b
                admit.append(s)
            if admit:
                by_field: Dict[str, List[Served]] = {}
                for s in admit:
                    by_field.setdefault(s.spec.field_name, []).append(s)
                tnow = time.perf_counter() - t0
                for name, group in by_field.items():
                    # every batch on the next stream of the pool
                    stream = self.streams[self._next_stream % len(self.streams)]
                    self._next_stream += 1
                    fh = self.fields[name]
                    for s in group:
                        r = s.spec.release
                        s.group = mp.mp_release_group(self.ctx.h, fh, n=r.n, lo=r.lo, hi=r.hi, seed=r.seed,
                                                      id_offset=r.id_offset, stream=stream)
                        s.admitted = tnow
                    ids = mp.mp_track_batch(self.ctx.h, [s.group for s in group], [self._opts(s.spec) for s in group],
                                            stream)
                    for s, rid in zip(group, ids):
                        s.rid = rid
                        s.batch = batches
                    batches += 1
                inflight.extend(admit)
                peak = max(peak, len(inflight))
                peak_bytes = max(peak_bytes, held)
            elif not inflight and realtime and nxt < n:
                time.sleep(max(0.0, min(0.002, specs[nxt].arrival_s * time_scale - (time.perf_counter() - t0))))
            else:
                time.sleep(50e-6)
        wall = time.perf_counter() - t0
        lat = np.array([(s.done - s.arrival) * 1e3 for s in finished])
        qms = np.array([(s.admitted - s.arrival) * 1e3 for s in finished])
        self.results = {id(s.spec): s.result for s in finished if s.result is not None}
        self.windows = batch_windows(finished)
        return ServeReport(n, wall, int(sum(s.spec.release.n for s in finished)),
                           int(sum(s.cell_steps for s in finished)), lat, qms, batches, peak,
                           extra={"peak_bytes": peak_bytes, "budget_bytes": self.budget,
                                  **device_overlap(self.windows)})
