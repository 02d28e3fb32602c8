"""Scan a text that lives in host memory, with the copies overlapped with the scan.

``scan_host`` cuts the text into chunks and runs three CUDA streams side by side: the
host-to-device copy of chunk i+1, the pack and scan of chunk i, and the device-to-host
copy of the ids of chunk i-1. A chunk is scanned on its own together with the first
max_len - 1 bases of the next chunk, so every walk that starts inside the chunk sees all
the bases it can use; only the chunk's own ids are copied back. Two sets of device
buffers alternate between chunks; events keep each buffer from being refilled before
the stream that reads it is done. The scan itself is the library's ``pfac_pack`` and
``pfac_match_packed`` (or ``pfac_match`` on the ASCII bytes, for texts that hold bytes
outside A/C/G/T such as newline-separated reads); Python only orders the calls.
"""
from __future__ import annotations

from . import _binding as b


def chunk_spans(n: int, chunk: int, max_len: int):
    """(lo, hi, ext) for each chunk of a text of `n` bases: the chunk's own offsets are
    [lo, hi), and it is scanned over [lo, ext), which adds the first max_len - 1 bases
    after it (fewer at the end of the text). A walk from an offset below hi reads at
    most max_len bases, so it never needs a base at or past ext."""
    if chunk <= 0 or max_len <= 0:
        raise ValueError("chunk and max_len must be positive")
    return [(lo, min(n, lo + chunk), min(n, lo + chunk + max_len - 1)) for lo in range(0, n, chunk)]


class HostScanner:
    """Device buffers and streams for chunked scans of host texts with one table."""

    def __init__(self, table, chunk_bases: int = 1 << 26, device="cuda", ascii: bool = False):
        """ascii: scan the ASCII bytes with pfac_match (any byte allowed; bytes outside
        A/C/G/T end walks) instead of packing them first."""
        import torch
        self.torch = torch
        self.table = table
        self.ascii = bool(ascii)
        self.max_len = int(table.info["max_len"])
        self.chunk = max(16, (int(chunk_bases) + 15) // 16 * 16)
        span = self.chunk + self.max_len + 16
        self.d_text = [torch.empty(span, dtype=torch.uint8, device=device) for _ in range(2)]
        self.d_packed = [torch.empty((span + 15) // 16, dtype=torch.int32, device=device) for _ in range(2)]
        self.d_out = [torch.empty(span, dtype=torch.int32, device=device) for _ in range(2)]
        self.s_in = torch.cuda.Stream(device=device)
        self.s_scan = torch.cuda.Stream(device=device)
        self.s_out = torch.cuda.Stream(device=device)
        self.ev_in = [torch.cuda.Event() for _ in range(2)]
        self.ev_scan = [torch.cuda.Event() for _ in range(2)]
        self.ev_out = [torch.cuda.Event() for _ in range(2)]
        for k in range(2):           # every buffer starts out free
            self.ev_scan[k].record(self.s_scan)
            self.ev_out[k].record(self.s_out)

    def scan(self, h_text, h_out):
        """Longest-pattern ids of the ASCII host tensor ``h_text`` (uint8, ideally pinned)
        into the host tensor ``h_out`` (int32, same length, ideally pinned). Returns when
        the last copy is queued; ``synchronize()`` waits for it. Unless the scanner was made
        with ascii=True, bytes that are not A, C, G or T are rejected by the pack step
        (status checked at the end)."""
        torch = self.torch
        n = int(h_text.numel())
        if h_out.numel() != n:
            raise ValueError("h_out must have one entry per base")
        n_chunks = (n + self.chunk - 1) // self.chunk
        status = torch.zeros(max(1, n_chunks), dtype=torch.int32, device=self.d_text[0].device)
        for i, (lo, hi, ext) in enumerate(chunk_spans(n, self.chunk, self.max_len)):
            k = i & 1
            m = ext - lo
            # input buffer k is free once the scan of chunk i-2 has read it
            self.s_in.wait_event(self.ev_scan[k])
            with torch.cuda.stream(self.s_in):
                self.d_text[k][:m].copy_(h_text[lo:ext], non_blocking=True)
                self.ev_in[k].record(self.s_in)
            # output buffer k is free once chunk i-2's ids have been copied out
            self.s_scan.wait_event(self.ev_in[k])
            self.s_scan.wait_event(self.ev_out[k])
            with torch.cuda.stream(self.s_scan):
                if self.ascii:
                    b.pfac_match(self.table.h, self.d_text[k], self.d_out[k], self.s_scan, length=m)
                else:
                    b.pfac_pack(self.d_text[k][:m], self.d_packed[k], status[i:i + 1], None, self.s_scan)
                    b.pfac_match_packed(self.table.h, self.d_packed[k], m, self.d_out[k], self.s_scan)
                self.ev_scan[k].record(self.s_scan)
            self.s_out.wait_event(self.ev_scan[k])
            with torch.cuda.stream(self.s_out):
                h_out[lo:hi].copy_(self.d_out[k][:hi - lo], non_blocking=True)
                self.ev_out[k].record(self.s_out)
        self._status = status
        return h_out

    def synchronize(self) -> int:
        """Wait for the last scan's copies; returns PFAC_OK or PFAC_ERR_BAD_SYMBOL."""
        self.s_out.synchronize()
        self.s_scan.synchronize()
        st = getattr(self, "_status", None)
        return int(st.max().item()) if st is not None else 0


def scan_host(table, h_text, h_out=None, chunk_bases: int = 1 << 26, ascii: bool = False):
    """One-shot form of ``HostScanner``: returns the host int32 ids of ``h_text``."""
    import torch
    if h_out is None:
        h_out = torch.empty(h_text.numel(), dtype=torch.int32, pin_memory=True)
    sc = HostScanner(table, chunk_bases, device="cuda", ascii=ascii)
    sc.scan(h_text, h_out)
    rc = sc.synchronize()
    if rc != 0:
        raise b.PfacError(rc, "scan_host")
    return h_out
