"""Scan a text that lives in host memory, with the copies overlapped with the scan.

``scan_host`` cuts the text into chunks and runs three CUDA streams side by side: the
host-to-device copy of chunk i+1, the pack and scan of chunk i, and the device-to-host
copy of the ids of chunk i-1 (or, with ``HostScanner.scan_matches``, of its match list). A chunk is scanned on its own together with the first
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

    def scan_matches(self, h_text, h_offsets, h_ids):
        """The match list of the ASCII host tensor ``h_text`` instead of one id per base:
        every offset with a pattern, ascending, with the longest pattern's id, into the
        host tensors ``h_offsets`` (int64) and ``h_ids`` (int32, ideally pinned), whose
        length bounds the number of matches. Each chunk is scanned into a device match list
        (``pfac_match_compact``) whose count is copied out first; the chunk's pairs are
        copied out while the next chunk is scanned, so only the matches cross the host
        link. Returns the number of matches (after synchronising); raises PfacError with
        PFAC_ERR_OVERFLOW when they do not fit."""
        torch = self.torch
        n = int(h_text.numel())
        cap_total = int(h_offsets.numel())
        if h_ids.numel() != cap_total:
            raise ValueError("h_offsets and h_ids must have the same length")
        spans = chunk_spans(n, self.chunk, self.max_len)
        if not hasattr(self, "d_moff"):
            span = self.chunk + self.max_len + 16
            dev = self.d_text[0].device
            self.d_moff = [torch.empty(span, dtype=torch.int64, device=dev) for _ in range(2)]
            self.d_mids = [torch.empty(span, dtype=torch.int32, device=dev) for _ in range(2)]
            self.d_mcnt = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(2)]
        h_cnt = torch.zeros(max(1, len(spans)), dtype=torch.int64).pin_memory()
        status = torch.zeros(max(1, len(spans)), dtype=torch.int32, device=self.d_text[0].device)
        placed = []                          # (chunk index, first slot, count)
        pos = 0

        def copy_out(i):
            # chunk i's count is on the host once its scan has finished
            nonlocal pos
            k = i & 1
            self.ev_scan[k].synchronize()
            c = int(h_cnt[i])
            if pos + c > cap_total:
                self.s_scan.synchronize()    # nothing of this call stays in flight
                self.s_out.synchronize()
                raise b.PfacError(b.CODE["PFAC_ERR_OVERFLOW"], "scan_matches")
            self.s_out.wait_event(self.ev_scan[k])
            with torch.cuda.stream(self.s_out):
                if c:
                    h_offsets[pos:pos + c].copy_(self.d_moff[k][:c], non_blocking=True)
                    h_ids[pos:pos + c].copy_(self.d_mids[k][:c], non_blocking=True)
                self.ev_out[k].record(self.s_out)
            placed.append((i, pos, c))
            pos += c

        for i, (lo, hi, ext) in enumerate(spans):
            k = i & 1
            m = ext - lo
            self.s_in.wait_event(self.ev_scan[k])
            with torch.cuda.stream(self.s_in):
                self.d_text[k][:m].copy_(h_text[lo:ext], non_blocking=True)
                self.ev_in[k].record(self.s_in)
            self.s_scan.wait_event(self.ev_in[k])
            self.s_scan.wait_event(self.ev_out[k])
            with torch.cuda.stream(self.s_scan):
                b.pfac_pack(self.d_text[k][:m], self.d_packed[k], status[i:i + 1], None, self.s_scan)
                b.pfac_match_compact(self.table.h, self.d_packed[k], m, self.d_moff[k], self.d_mids[k],
                                     self.d_mcnt[k], self.s_scan)
                h_cnt[i:i + 1].copy_(self.d_mcnt[k], non_blocking=True)
                self.ev_scan[k].record(self.s_scan)
            if i >= 1:
                copy_out(i - 1)
        if spans:
            copy_out(len(spans) - 1)
        self.s_out.synchronize()
        self._status = status
        st = int(status.max().item())
        if st:
            raise b.PfacError(st, "scan_matches")
        # chunk-relative offsets -> text offsets; the pairs of a chunk's halo belong to the
        # next chunk (which lists them itself) and are dropped; chunks are in text order
        out = 0
        offs_np, ids_np = h_offsets.numpy(), h_ids.numpy()
        for i, p0, c in placed:
            lo, hi, _ = spans[i]
            o = offs_np[p0:p0 + c] + lo
            keep = o < hi
            o, d = o[keep], ids_np[p0:p0 + c][keep]
            order = o.argsort(kind="stable")
            kk = o.size
            offs_np[out:out + kk] = o[order]
            ids_np[out:out + kk] = d[order]
            out += kk
        return out

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
