"""Batched scans: many reads against many resident tables.

``BatchedScanner`` keeps fixed-capacity device buffers for a batch (read bytes, read
offsets, read-to-table map, output) and runs ``pfac_match_batched`` on them, either
directly or by replaying a CUDA graph captured once: every replay is one launch (each
CTA plans the batch, scans the work items dealt to it and finishes its long walks) with
the inputs the caller copied into the buffers; batches of more than 8,192 reads take a
pack, a plan, a scan and a tail launch. ``tune`` picks the launch shape with the autotuner before capturing. ``scan_per_read`` is the baseline it is measured against: one
``pfac_match`` launch per read.
"""
from __future__ import annotations

import numpy as np

from . import _binding as b


class BatchedScanner:
    def __init__(self, tables, max_bases: int, max_reads: int, graph: bool = True, device: str = "cuda"):
        import torch
        self.torch = torch
        self.tables = list(tables)
        self.handles = [t.h for t in self.tables]
        self.max_bases = int(max_bases)
        self.max_reads = int(max_reads)
        self.texts = torch.zeros(self.max_bases, dtype=torch.uint8, device=device)
        self.offsets = torch.zeros(self.max_reads + 1, dtype=torch.int64, device=device)
        self.read_set = torch.zeros(self.max_reads, dtype=torch.int32, device=device)
        self.out = torch.zeros(self.max_bases, dtype=torch.int32, device=device)
        self.stream = torch.cuda.Stream(device=device)
        self.graph = None
        if graph:
            self.capture()

    def capture(self):
        """Capture one batched call into a CUDA graph, which ``run`` then replays. The
        launch shape (the configuration of the first table) is fixed at capture."""
        torch = self.torch
        # First call: uploads the table descriptors and allocates the scratch, which
        # must happen before capture.
        with torch.cuda.stream(self.stream):
            self._call()
        self.stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream):
            self._call()
        self.graph = g

    def tune(self, **kw):
        """Autotune the batched launch shape on the loaded batch (see autotune.py), then
        capture the graph. Returns the chosen configuration."""
        from . import autotune
        with self.torch.cuda.stream(self.stream):
            cfg = autotune.tune_batched(self.tables, self.texts, self.offsets, self.read_set, self.out, **kw)
        self.stream.synchronize()
        self.capture()
        return cfg

    def _call(self):
        b.pfac_match_batched(self.handles, self.texts, self.offsets, self.read_set, self.out,
                             self.torch.cuda.current_stream())

    def load(self, reads, read_offsets, read_set):
        """Copy a batch into the device buffers (reads as one uint8 array, offsets with
        n_reads + 1 entries starting at 0, one table index per read)."""
        torch = self.torch
        n_reads = len(read_set)
        total = int(read_offsets[-1])
        if n_reads > self.max_reads or total > self.max_bases:
            raise ValueError("batch larger than the scanner's capacity")
        offs = np.full(self.max_reads + 1, total, dtype=np.int64)
        offs[:n_reads + 1] = np.asarray(read_offsets, dtype=np.int64)
        rs = np.zeros(self.max_reads, dtype=np.int32)
        rs[:n_reads] = np.asarray(read_set, dtype=np.int32)
        with torch.cuda.stream(self.stream):
            if isinstance(reads, torch.Tensor):
                self.texts[:total].copy_(reads[:total], non_blocking=True)
            else:
                self.texts[:total].copy_(torch.from_numpy(np.ascontiguousarray(reads[:total])), non_blocking=True)
            self.offsets.copy_(torch.from_numpy(offs), non_blocking=True)
            self.read_set.copy_(torch.from_numpy(rs), non_blocking=True)
        return total

    def run(self):
        """Scan the loaded batch on the scanner's stream (asynchronous)."""
        with self.torch.cuda.stream(self.stream):
            if self.graph is not None:
                self.graph.replay()
            else:
                self._call()
        return self.out

    def scan(self, reads, read_offsets, read_set) -> np.ndarray:
        total = self.load(reads, read_offsets, read_set)
        self.run()
        self.stream.synchronize()
        return self.out[:total].cpu().numpy()


def scan_per_read(tables, d_texts, read_offsets, read_set, d_out, stream=None):
    """The baseline: one pfac_match launch per read (read_offsets, read_set on the host)."""
    for r in range(len(read_set)):
        lo, hi = int(read_offsets[r]), int(read_offsets[r + 1])
        if hi > lo:
            b.pfac_match(tables[int(read_set[r])].h, d_texts[lo:hi], d_out[lo:hi], stream)


class PerReadGraph:
    """The per-read baseline as device work alone: the pfac_match launches of
    ``scan_per_read`` (one per read, each a scan and a tail kernel), captured once into
    a CUDA graph on one stream and replayed, so that timing a replay measures the
    launches on the GPU without the host's cost of issuing them one by one."""

    def __init__(self, tables, d_texts, read_offsets, read_set, d_out):
        import torch
        self.torch = torch
        self.stream = torch.cuda.Stream()
        args = (tables, d_texts, read_offsets, read_set, d_out)
        # first launches on the stream: the library allocates its per-stream scratch
        with torch.cuda.stream(self.stream):
            scan_per_read(*args, stream=self.stream)
        self.stream.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            scan_per_read(*args, stream=self.stream)
        self.launches = 2 * sum(1 for r in range(len(read_set)) if read_offsets[r + 1] > read_offsets[r])

    def run(self):
        with self.torch.cuda.stream(self.stream):
            self.graph.replay()
