"""A serving loop for the scan: requests arrive over time, each naming a resident
table and carrying a DNA text; the server batches whatever has arrived into one
``pfac_match_batched`` pass per slot and keeps several slots in flight.

* Tables stay on the device for the server's lifetime (built once).
* Admission by free device memory: a request is admitted only while the bytes of
  all batches in flight (text in, ids out) stay under a budget taken from the free
  HBM at start-up (and within one slot's capacity).
* Continuous batching: whenever a slot is free, everything admitted so far goes into
  its next batch, so requests that arrive while other batches are on the GPU join
  the next one; each slot has its own stream, pinned buffers and device buffers,
  so the copies and scans of different batches overlap.
* Latency of a request = time from its arrival to the moment its ids are on the host.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import _binding as b


@dataclass
class Request:
    rid: int
    set_id: int
    text: np.ndarray          # ASCII uint8
    arrival: float            # seconds from the start of the run


# device bytes one base costs while its batch is in flight: its byte in, its int32 id out
BYTES_PER_BASE = 5


def take_batch(waiting: deque, in_flight: int, budget: int, slot_bases: int, max_reads: int) -> list:
    """Pops the next batch from the front of `waiting`, in arrival order: at most
    `max_reads` requests and `slot_bases` bases, and only while the device bytes of
    the batches in flight (`in_flight`) plus this one's stay within `budget`. With
    nothing in flight the first request is taken whatever its size, so a request
    larger than the budget still runs, alone. A request longer than `slot_bases` can
    never run: the batch before it is returned as usual, and the call that finds it at
    the front of `waiting` raises ValueError and leaves it there."""
    batch, bases = [], 0
    while waiting and len(batch) < max_reads:
        r = waiting[0]
        n = int(r.text.shape[0])
        if bases + n > slot_bases:
            if not batch:
                raise ValueError(f"request {r.rid} ({n} bases) exceeds the slot capacity")
            break
        if in_flight + BYTES_PER_BASE * (bases + n) > budget and (in_flight or batch):
            break        # admitted only when device memory frees up
        batch.append(waiting.popleft())
        bases += n
    return batch


@dataclass
class _Slot:
    stream: object
    h_in: object              # pinned uint8
    h_out: object             # pinned int32
    d_in: object
    d_out: object
    d_offs: object
    d_sets: object
    event: object = None
    requests: list = field(default_factory=list)
    starts: list = field(default_factory=list)
    bytes: int = 0


class Server:
    def __init__(self, tables, slot_bases: int = 1 << 24, n_slots: int = 3, max_reads: int = 4096,
                 hbm_fraction: float = 0.5, keep_results=False):
        """keep_results: True to keep every request's ids on the host, or a set of request
        ids to keep only those."""
        import torch
        self.torch = torch
        self.tables = list(tables)
        self.handles = [t.h for t in self.tables]
        self.slot_bases = int(slot_bases)
        self.max_reads = int(max_reads)
        free, _total = torch.cuda.mem_get_info()
        self.budget = int(free * hbm_fraction)
        self.keep_results = keep_results
        self.slots = []
        for _ in range(n_slots):
            self.slots.append(_Slot(
                stream=torch.cuda.Stream(),
                h_in=torch.empty(self.slot_bases, dtype=torch.uint8).pin_memory(),
                h_out=torch.empty(self.slot_bases, dtype=torch.int32).pin_memory(),
                d_in=torch.empty(self.slot_bases, dtype=torch.uint8, device="cuda"),
                d_out=torch.empty(self.slot_bases, dtype=torch.int32, device="cuda"),
                d_offs=torch.empty(self.max_reads + 1, dtype=torch.int64, device="cuda"),
                d_sets=torch.empty(self.max_reads, dtype=torch.int32, device="cuda")))
        # first batched call per stream: uploads the descriptors and allocates scratch
        for sl in self.slots:
            with torch.cuda.stream(sl.stream):
                sl.d_in[:1].fill_(ord("A"))
                offs = torch.tensor([0, 1], dtype=torch.int64, device="cuda")
                b.pfac_match_batched(self.handles, sl.d_in[:1], offs, sl.d_sets[:1].zero_(), sl.d_out[:1],
                                     sl.stream)
            sl.stream.synchronize()

    @staticmethod
    def request_bytes(req: Request) -> int:
        return BYTES_PER_BASE * int(req.text.shape[0])

    def _launch(self, sl: _Slot, batch: list):
        torch = self.torch
        lens = np.array([r.text.shape[0] for r in batch], dtype=np.int64)
        offs = np.zeros(len(batch) + 1, dtype=np.int64)
        np.cumsum(lens, out=offs[1:])
        total = int(offs[-1])
        hin = sl.h_in.numpy()
        for r, o in zip(batch, offs[:-1]):
            hin[o:o + r.text.shape[0]] = r.text
        sets = np.array([r.set_id for r in batch], dtype=np.int32)
        with torch.cuda.stream(sl.stream):
            sl.d_in[:total].copy_(sl.h_in[:total], non_blocking=True)
            sl.d_offs[:len(batch) + 1].copy_(torch.from_numpy(offs), non_blocking=True)
            sl.d_sets[:len(batch)].copy_(torch.from_numpy(sets), non_blocking=True)
            b.pfac_match_batched(self.handles, sl.d_in[:total], sl.d_offs[:len(batch) + 1],
                                 sl.d_sets[:len(batch)], sl.d_out[:total], sl.stream)
            sl.h_out[:total].copy_(sl.d_out[:total], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(sl.stream)
        sl.event = ev
        sl.requests = batch
        sl.starts = offs
        sl.bytes = BYTES_PER_BASE * total

    def run(self, requests, realtime: bool = True):
        """Serve `requests` (sorted by arrival). Returns (per-request latency in s,
        results by request id if keep_results, statistics)."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        waiting = deque()
        in_flight = 0
        latency = {}
        results = {}
        matches = 0
        batches = 0
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        n_total = len(pending)
        done = 0
        while done < n_total:
            t = now()
            # arrivals (all at once when not in real time)
            while pending and (not realtime or pending[0].arrival <= t):
                waiting.append(pending.popleft())
            # completions
            progressed = False
            for sl in self.slots:
                if sl.event is not None and sl.event.query():
                    tdone = now()
                    out = sl.h_out.numpy()
                    for r, o in zip(sl.requests, sl.starts[:-1]):
                        latency[r.rid] = tdone - (r.arrival if realtime else 0.0)
                        if self.keep_results is True or (self.keep_results and r.rid in self.keep_results):
                            ids = out[o:o + r.text.shape[0]]
                            matches += int(np.count_nonzero(ids))
                            results[r.rid] = ids.copy()
                    in_flight -= sl.bytes
                    done += len(sl.requests)
                    sl.event, sl.requests, sl.bytes = None, [], 0
                    progressed = True
            # admission and batching into free slots
            for sl in self.slots:
                if sl.event is not None or not waiting:
                    continue
                batch = take_batch(waiting, in_flight, self.budget, self.slot_bases, self.max_reads)
                if batch:
                    self._launch(sl, batch)
                    in_flight += sl.bytes
                    batches += 1
                    progressed = True
            if not progressed:
                # nothing to do until the next arrival or completion
                nxt = pending[0].arrival - now() if (pending and realtime) else 0.0
                time.sleep(min(max(nxt, 0.0), 0.0002) if nxt > 0 else 0.00005)
        wall = now()
        lat = np.array([latency[r.rid] for r in requests]) if requests else np.zeros(0)
        bases = int(sum(r.text.shape[0] for r in requests))
        stats = {"requests": n_total, "batches": batches, "bases": bases, "wall_s": wall,
                 "gbases_s": bases / wall / 1e9 if wall > 0 else 0.0,
                 "p50_ms": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
                 "p99_ms": float(np.percentile(lat, 99) * 1e3) if lat.size else None,
                 "matches": matches if self.keep_results is True else None}
        return lat, results, stats


def serve_per_request(tables, requests, realtime: bool = True, max_bases: int = 1 << 24,
                      keep_results=False):
    """The baseline the server is measured against: one request at a time, in arrival
    order, on one stream, with one ``pfac_match`` launch per request: its text copied in
    from pinned memory, the scan, its ids copied out, then the next request. Same
    latency definition as ``Server.run`` (arrival to ids on the host; with
    realtime=False every request arrives at time 0). Returns (latency in s, results by
    request id if keep_results, statistics)."""
    import torch
    stream = torch.cuda.Stream()
    h_in = torch.empty(max_bases, dtype=torch.uint8).pin_memory()
    h_out = torch.empty(max_bases, dtype=torch.int32).pin_memory()
    d_in = torch.empty(max_bases, dtype=torch.uint8, device="cuda")
    d_out = torch.empty(max_bases, dtype=torch.int32, device="cuda")
    # first launch on the stream: the library allocates its per-stream scratch
    with torch.cuda.stream(stream):
        d_in[:64].fill_(ord("A"))
        for t in tables:
            b.pfac_match(t.h, d_in[:64], d_out[:64], stream)
    stream.synchronize()
    order = sorted(requests, key=lambda r: r.arrival)
    latency, results = {}, {}
    hin, hout = h_in.numpy(), h_out.numpy()
    t0 = time.perf_counter()
    for r in order:
        n = int(r.text.shape[0])
        if n > max_bases:
            raise ValueError(f"request {r.rid} ({n} bases) exceeds the buffer")
        if realtime:
            wait = r.arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        hin[:n] = r.text
        with torch.cuda.stream(stream):
            d_in[:n].copy_(h_in[:n], non_blocking=True)
            b.pfac_match(tables[r.set_id].h, d_in[:n], d_out[:n], stream)
            h_out[:n].copy_(d_out[:n], non_blocking=True)
        stream.synchronize()
        latency[r.rid] = time.perf_counter() - t0 - (r.arrival if realtime else 0.0)
        if keep_results is True or (keep_results and r.rid in keep_results):
            results[r.rid] = hout[:n].copy()
    wall = time.perf_counter() - t0
    lat = np.array([latency[r.rid] for r in requests]) if requests else np.zeros(0)
    bases = int(sum(r.text.shape[0] for r in requests))
    stats = {"requests": len(requests), "launches": len(requests), "bases": bases, "wall_s": wall,
             "gbases_s": bases / wall / 1e9 if wall > 0 else 0.0,
             "p50_ms": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
             "p99_ms": float(np.percentile(lat, 99) * 1e3) if lat.size else None}
    return lat, results, stats


def requests_from_stream(stream, limit: int | None = None):
    """Request objects for a datagen RequestStream."""
    n = len(stream.arrivals) if limit is None else min(limit, len(stream.arrivals))
    return [Request(i, int(stream.set_id[i]), stream.text(i), float(stream.arrivals[i])) for i in range(n)]
