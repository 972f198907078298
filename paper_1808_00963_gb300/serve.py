"""Serving loop for sort requests on one GPU.

Requests (a host string set each) arrive over time.  They are admitted in
arrival order while their device footprint (characters, offsets, outputs and
workspace) fits the HBM budget.  Admission puts a request on the device at
once: its buffers are allocated and its characters and offsets copied in on a
copy stream, and they stay there until the request completes.

Continuous batching: each of several worker streams takes everything admitted
so far (up to a cap) and enqueues it as one batch (ss_batch_*; a single
request with ss_sort_ex), followed by the copies of the results back to
pinned host memory, then takes the next group without waiting: a worker keeps
up to ``depth`` groups in flight on its stream and completes the oldest one
when it has to wait (its results are on the host, its memory goes back to the
budget).  Requests that arrive while others are on the GPU are admitted as
memory frees up, and their work overlaps with the running groups on the
device.  ss_sort_ex and ss_batch_run return without waiting (the multi-block
rounds of large requests run on the device), so no request holds a worker's
thread while the GPU sorts it.  A request above ``big`` strings is sorted
alone (ss_sort_ex), by default none: batches take multi-block steps too.

``mode="plain"`` is the one-at-a-time baseline: a single worker sorts one
request after the other with ss_sort_ex and waits for each, under the same
admission rule.

The sorting itself runs in the library's CUDA kernels; this module only
schedules, allocates (through torch) and copies.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import Batch, SortError, sort, stream_status, workspace_size


@dataclass
class Request:
    rid: int
    arrival: float                 # seconds after the start of the run
    chars: object                  # pinned torch.uint8 (host)
    offsets: object                # pinned torch.int64 (host)
    max_len: int = 0
    n: int = 0
    footprint: int = 0
    start: float = -1.0
    done: float = -1.0
    batch_size: int = 0
    perm: object = None            # pinned torch.int32 result (host)
    lcp: object = None
    meta: dict = field(default_factory=dict)


def device_footprint(n: int, nchars: int, max_len: int = 0) -> int:
    """Bytes a request holds on the device while admitted."""
    return nchars + 16 + 8 * n + 8 * n + workspace_size(max(n, 1), max_len)


def make_request(rid: int, arrival: float, chars: np.ndarray, offsets: np.ndarray, max_len: int = 0) -> Request:
    import torch
    ch = torch.from_numpy(np.ascontiguousarray(chars) if chars.size else np.zeros(1, np.uint8)).pin_memory()
    of = torch.from_numpy(np.ascontiguousarray(offsets).view(np.int64)).pin_memory()
    n = int(of.numel())
    r = Request(rid, arrival, ch, of, max_len, n, device_footprint(n, int(ch.numel()), max_len))
    r.perm = torch.empty(n, dtype=torch.int32).pin_memory()
    r.lcp = torch.empty(n, dtype=torch.int32).pin_memory()
    return r


class _Resident:
    """A request's device buffers, filled on the copy stream at admission."""

    def __init__(self, r: Request, copy_stream):
        import torch
        with torch.cuda.stream(copy_stream):
            self.chars = torch.empty(r.chars.numel() + 16, dtype=torch.uint8, device="cuda")
            self.chars[r.chars.numel():].zero_()
            self.chars[: r.chars.numel()].copy_(r.chars, non_blocking=True)
            self.offsets = r.offsets.to("cuda", non_blocking=True)
            self.perm = torch.empty(r.n, dtype=torch.int32, device="cuda")
            self.lcp = torch.empty(r.n, dtype=torch.int32, device="cuda")
            self.ready = torch.cuda.Event()
            self.ready.record(copy_stream)

    def use_on(self, stream):
        """Make `stream` wait for the copies; tie the buffers' lifetime to it."""
        stream.wait_event(self.ready)
        for t in (self.chars, self.offsets, self.perm, self.lcp):
            t.record_stream(stream)


class Server:
    def __init__(self, budget_bytes: int = 30 << 30, streams: int = 4, batch_max: int = 512,
                 big: int | None = None, mode: str = "served", on_done=None, depth: int = 2):
        """on_done(request), if given, is called by the worker for every
        completed request once its results are on the host (for checks; it
        delays that worker's next group)."""
        assert mode in ("served", "plain")
        self.on_done = on_done
        self.budget = budget_bytes
        self.nstreams = 1 if mode == "plain" else streams
        self.batch_max = 1 if mode == "plain" else batch_max
        self.big = big if big is not None else (1 << 62)
        self.depth = 1 if mode == "plain" else max(1, depth)
        self.mode = mode
        self.cv = threading.Condition()
        self.pending = collections.deque()
        self.admitted = collections.deque()
        self.free = budget_bytes
        self.arrivals_done = False
        self.in_flight_peak = 0
        self.in_flight = 0
        self.errors = []
        self.copy_stream = None

    # -- scheduling (call with self.cv held) --------------------------------------------------
    def _admit(self):
        # a request larger than the whole budget is admitted alone (when
        # nothing else holds memory), so that it cannot block the queue
        while self.pending and (self.pending[0].footprint <= self.free or self.free == self.budget):
            r = self.pending.popleft()
            self.free -= r.footprint
            r.meta["dev"] = _Resident(r, self.copy_stream)
            self.admitted.append(r)

    def _take(self):
        first = self.admitted.popleft()
        group = [first]
        if self.mode == "plain" or first.n > self.big:
            return group
        while self.admitted and len(group) < self.batch_max and self.admitted[0].n <= self.big:
            group.append(self.admitted.popleft())
        return group

    # -- execution ---------------------------------------------------------------------------
    def _enqueue(self, group, stream, t0):
        """Enqueues a group's sort and result copies on `stream`; returns what
        completing it needs (its event and batch)."""
        import torch
        now = time.perf_counter() - t0
        dev = []
        for r in group:
            r.start = now
            r.batch_size = len(group)
            d = r.meta["dev"]
            d.use_on(stream)
            dev.append((d.chars, d.offsets, r.max_len, d.perm, d.lcp))
        batch = None
        with torch.cuda.stream(stream):
            if len(group) == 1:
                ch, of, ml, p, l = dev[0]
                sort(ch, of, max_len=ml, out=(p, l), stream=stream, sync=False)
            else:
                batch = Batch(dev, own_workspace=True)
                batch.run(stream)
            for r, (_, _, _, p, l) in zip(group, dev):
                r.perm.copy_(p, non_blocking=True)
                r.lcp.copy_(l, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        return ev, batch

    def _complete(self, group, ev, batch, status_stream, t0):
        """Waits for a group; checks its device status; marks it done."""
        ev.synchronize()
        try:
            if batch is not None:
                batch.status(status_stream)  # the batch's own status word (its run has finished)
        finally:
            if batch is not None:
                batch.close()
        now = time.perf_counter() - t0
        for r in group:
            r.done = now
            r.meta.pop("dev", None)
        if self.on_done is not None:
            for r in group:
                self.on_done(r)

    def _release(self, group):
        with self.cv:
            self.free += sum(r.footprint for r in group)
            self.in_flight -= 1
            self.cv.notify_all()

    def _worker(self, t0):
        import torch
        stream = torch.cuda.Stream()
        status_stream = torch.cuda.Stream()
        flight = collections.deque()  # (group, event, batch)

        def finish_oldest():
            group, ev, batch = flight.popleft()
            try:
                self._complete(group, ev, batch, status_stream, t0)
            except Exception as e:  # report, never hang the loop
                self.errors.append(repr(e))
                for r in group:
                    r.done = float("nan")
            self._release(group)

        while True:
            group = None
            with self.cv:
                while True:
                    self._admit()
                    if self.admitted and len(flight) < self.depth:
                        group = self._take()
                        self.in_flight += 1
                        self.in_flight_peak = max(self.in_flight_peak, self.in_flight)
                        break
                    if flight or (self.arrivals_done and not self.pending and not self.admitted):
                        break
                    self.cv.wait()
            if group is None:
                if not flight:
                    break
                finish_oldest()  # nothing to take now (or no room): complete the oldest group
                continue
            try:
                ev, batch = self._enqueue(group, stream, t0)
                flight.append((group, ev, batch))
            except Exception as e:
                self.errors.append(repr(e))
                for r in group:
                    r.done = float("nan")
                self._release(group)
        try:  # single-request groups report device errors through the stream's status word
            stream_status(stream)
        except SortError as e:
            self.errors.append(repr(e))

    def run(self, requests):
        """Replays the requests at their arrival times; returns per-request
        (arrival, start, done) and summary statistics."""
        import torch
        torch.cuda.synchronize()
        self.copy_stream = torch.cuda.Stream()
        t0 = time.perf_counter()
        workers = [threading.Thread(target=self._worker, args=(t0,), daemon=True) for _ in range(self.nstreams)]
        for w in workers:
            w.start()
        for r in sorted(requests, key=lambda x: x.arrival):
            delay = r.arrival - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            with self.cv:
                self.pending.append(r)
                self.cv.notify_all()
        with self.cv:
            self.arrivals_done = True
            self.cv.notify_all()
        for w in workers:
            w.join()
        return summarize(requests, self)


def summarize(requests, server=None):
    lat = np.array([r.done - r.arrival for r in requests]) * 1e3
    n = sum(r.n for r in requests)
    span = max(r.done for r in requests) - min(r.arrival for r in requests)
    out = {
        "requests": len(requests), "strings": n,
        "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
        "latency_ms_max": float(lat.max()), "strings_per_s": n / span, "span_s": span,
        "mean_batch": float(np.mean([r.batch_size for r in requests])),
    }
    if server is not None:
        out["peak_batches_in_flight"] = server.in_flight_peak
        out["errors"] = server.errors
    return out
