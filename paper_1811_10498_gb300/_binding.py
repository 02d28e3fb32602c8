"""ctypes binding of ``libpfac.so`` (include/pfac.h).

Argument marshalling only: every step of the scan runs in the CUDA library. Device
buffers are torch CUDA tensors (torch provides memory and streams); streams default
to torch's current stream. If the library has not been built, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build_ext

P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64

PFAC_OK = 0
STATUS = {
    0: "PFAC_OK", 1: "PFAC_ERR_INVALID_ARG", 2: "PFAC_ERR_EMPTY_PATTERN", 3: "PFAC_ERR_BAD_SYMBOL",
    4: "PFAC_ERR_TOO_MANY_STATES", 5: "PFAC_ERR_OOM", 6: "PFAC_ERR_CUDA", 7: "PFAC_ERR_OVERFLOW",
    8: "PFAC_ERR_TIMEOUT", 9: "PFAC_ERR_HOST_ONLY", 10: "PFAC_ERR_UNSUPPORTED", 11: "PFAC_ERR_SCRATCH_LIMIT",
    12: "PFAC_ERR_IO",
}
CODE = {v: k for k, v in STATUS.items()}


class PfacError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = f"{where}: {STATUS.get(code, code)}"
        if code == CODE["PFAC_ERR_CUDA"] and _lib is not None:
            msg += f" ({_lib.pfac_last_cuda_error().decode()})"
        super().__init__(msg)


class pfac_build_opts(C.Structure):
    _fields_ = [("host_only", I32), ("filter_b", I32), ("sample", I32)]


class pfac_table_info(C.Structure):
    _fields_ = [("n_states", I64), ("n_patterns", I32), ("max_len", I32), ("min_len", I32),
                ("filter_b", I32), ("n_duplicates", I64), ("table_bytes", I64), ("rows_bytes", I64),
                ("skip_bytes", I64), ("filter_set", I64), ("has_skip", I32), ("rank_wide", I32),
                ("device", I32), ("sample_q", I32), ("sample_s", I32), ("pad", I32)]


class pfac_config(C.Structure):
    _fields_ = [("kernel", I32), ("threads", I32), ("ctas_per_sm", I32), ("stages", I32), ("rank_in_smem", I32),
                ("l2_persist", I32), ("walk_loads", I32), ("lane_offsets", I32), ("table_layout", I32),
                ("row_loads", I32), ("text_smem", I32), ("zero_writer", I32), ("screen", I32), ("reserved", I32)]


_lib = None
_lock = threading.Lock()

_SIGS = {
    "pfac_build": (P, [P, P, I32]),
    "pfac_build_ex": (P, [P, P, I32, P]),
    "pfac_build_file": (P, [C.c_char_p, P]),
    "pfac_build_device": (P, [P, P, I32, P, P]),
    "pfac_read_text_file": (C.c_int, [C.c_char_p, I32, P, I64, P]),
    "pfac_last_error": (C.c_int, []),
    "pfac_error_string": (C.c_char_p, [C.c_int]),
    "pfac_last_cuda_error": (C.c_char_p, []),
    "pfac_destroy": (C.c_int, [P]),
    "pfac_info": (C.c_int, [P, P, P, P]),
    "pfac_info_ex": (C.c_int, [P, P]),
    "pfac_export": (C.c_int, [P, P, P, P]),
    "pfac_export_shortcuts": (C.c_int, [P, P, I64, P, I64, P, I64]),
    "pfac_export_sample": (C.c_int, [P, P, I64]),
    "pfac_set_config": (C.c_int, [P, P]),
    "pfac_get_config": (C.c_int, [P, I64, P]),
    "pfac_pack": (C.c_int, [P, I64, P, P, P, P]),
    "pfac_match": (C.c_int, [P, P, I64, P, P]),
    "pfac_match_packed": (C.c_int, [P, P, I64, P, P]),
    "pfac_match_compact": (C.c_int, [P, P, I64, P, P, I64, P, P]),
    "pfac_match_all": (C.c_int, [P, P, I64, P, P, I64, P, P]),
    "pfac_match_batched": (C.c_int, [P, I32, P, I64, P, P, I32, P, P]),
    "pfac_device_status": (C.c_int, [P, P, P]),
    "pfac_debug_timeout_probe": (C.c_int, [P, I64, P]),
    "pfac_match_packed_noalloc": (C.c_int, [P, P, I64, P, P]),
}


def lib_path() -> str:
    return build_ext.LIB


def lib() -> C.CDLL:
    """The loaded CUDA library. Raises if it has not been built: there is no fallback."""
    global _lib
    with _lock:
        if _lib is None:
            path = lib_path()
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with paper_1811_10498_gb300.build_ext.build() "
                                   "(the scan runs only in the CUDA library)")
            L = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
        return _lib


def _check(rc: int, where: str):
    if rc != PFAC_OK:
        raise PfacError(rc, where)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dptr(t):
    """Device pointer of a CUDA tensor (None for None)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor: the scan has no CPU path")
    return t.data_ptr()


def _patterns(patterns):
    if isinstance(patterns, tuple):
        blob, offsets = patterns
        blob = np.ascontiguousarray(blob, dtype=np.uint8)
        offsets = np.asarray(offsets, dtype=np.int64)
    else:
        lens = np.array([len(p) for p in patterns], dtype=np.int64)
        offsets = np.zeros(len(patterns) + 1, dtype=np.int64)
        np.cumsum(lens, out=offsets[1:])
        blob = np.frombuffer(b"".join(bytes(p) for p in patterns), dtype=np.uint8).copy()
    if blob.size == 0:
        blob = np.zeros(1, dtype=np.uint8)
    n = offsets.shape[0] - 1
    ptrs = (blob.ctypes.data + offsets[:-1]).astype(np.uint64) if n > 0 else np.zeros(1, np.uint64)
    lengths = np.diff(offsets).astype(np.int32) if n > 0 else np.zeros(1, np.int32)
    return blob, ptrs, lengths, n


# ---------------------------------------------------------------------------
# Calls with the C names.
# ---------------------------------------------------------------------------

def pfac_build(patterns, host_only: bool = False, filter_b: int = 0, sample: int = 0) -> int:
    """Build a table from ``(blob, offsets)`` or a list of byte strings; returns the handle."""
    L = lib()
    blob, ptrs, lengths, n = _patterns(patterns)
    opts = pfac_build_opts(int(host_only), int(filter_b), int(sample))
    h = L.pfac_build_ex(ptrs.ctypes.data, lengths.ctypes.data, n, C.byref(opts))
    if not h:
        raise PfacError(L.pfac_last_error(), "pfac_build")
    return h


def pfac_build_device(d_blob, d_offsets, filter_b: int = 0, sample: int = 0, stream=None) -> int:
    """Build a table on the GPU from device tensors: the patterns' bytes concatenated
    (uint8) and int64 offsets (n + 1 entries)."""
    n = int(d_offsets.numel()) - 1
    opts = pfac_build_opts(0, int(filter_b), int(sample))
    h = lib().pfac_build_device(_dptr(d_blob), _dptr(d_offsets), n, C.byref(opts), _stream(stream))
    if not h:
        raise PfacError(lib().pfac_last_error(), "pfac_build_device")
    return h


def pfac_build_file(path: str, host_only: bool = False, filter_b: int = 0) -> int:
    """Build from a pattern file (one pattern per line, or FASTA records)."""
    opts = pfac_build_opts(1 if host_only else 0, int(filter_b))
    h = lib().pfac_build_file(os.fsencode(path), C.byref(opts))
    if not h:
        raise PfacError(lib().pfac_last_error(), "pfac_build_file")
    return h


def read_text_file(path: str, fasta: bool = False) -> np.ndarray:
    """A text file as ASCII uint8 (as it is, or FASTA records joined with one newline
    between records)."""
    n = I64(0)
    _check(lib().pfac_read_text_file(os.fsencode(path), 1 if fasta else 0, None, 0, C.byref(n)),
           "pfac_read_text_file")
    buf = np.empty(max(1, n.value), dtype=np.uint8)
    got = I64(0)
    _check(lib().pfac_read_text_file(os.fsencode(path), 1 if fasta else 0, buf.ctypes.data, n.value, C.byref(got)),
           "pfac_read_text_file")
    return buf[:min(n.value, got.value)]


def pfac_destroy(h: int):
    _check(lib().pfac_destroy(h), "pfac_destroy")


def pfac_info(h: int):
    n_states, max_len, tb = I64(), I32(), I64()
    _check(lib().pfac_info(h, C.byref(n_states), C.byref(max_len), C.byref(tb)), "pfac_info")
    return n_states.value, max_len.value, tb.value


def pfac_info_ex(h: int) -> dict:
    i = pfac_table_info()
    _check(lib().pfac_info_ex(h, C.byref(i)), "pfac_info_ex")
    return {f: getattr(i, f) for f, _ in pfac_table_info._fields_}


def pfac_export(h: int):
    info = pfac_info_ex(h)
    S, Lm = info["n_states"], info["max_len"]
    rows = np.zeros((S, 4), dtype=np.int32)
    out_id = np.zeros(S, dtype=np.int32)
    level = np.zeros(Lm + 2, dtype=np.int64)
    _check(lib().pfac_export(h, rows.ctypes.data, out_id.ctypes.data, level.ctypes.data), "pfac_export")
    return rows, out_id, level


def pfac_export_shortcuts(h: int):
    """(skip entries [S, 4], filter words, dense entries [F, 4]) of a host-only handle."""
    info = pfac_info_ex(h)
    S, b, F = info["n_states"], info["filter_b"], info["filter_set"]
    skip = np.zeros((S if info["has_skip"] else 0, 4), dtype=np.uint32)
    filt = np.zeros(max(1, (1 << (2 * b)) // 32) if b else 0, dtype=np.uint32)
    dense = np.zeros((F, 4), dtype=np.uint32)
    ptr = lambda a: a.ctypes.data if a.size else None
    _check(lib().pfac_export_shortcuts(h, ptr(skip), skip.size, ptr(filt), filt.size, ptr(dense), dense.size),
           "pfac_export_shortcuts")
    return skip, filt, dense


def pfac_export_sample(h: int):
    """(q, s, q-gram bit words) of a host-only handle's sampled screen; (0, 0, empty)
    when it has none."""
    info = pfac_info_ex(h)
    q, s = info["sample_q"], info["sample_s"]
    g = np.zeros(((1 << (2 * q)) // 32) if q else 0, dtype=np.uint32)
    _check(lib().pfac_export_sample(h, g.ctypes.data if g.size else None, g.size), "pfac_export_sample")
    return q, s, g


def pfac_set_config(h: int, cfg: dict | None):
    if cfg is None:
        _check(lib().pfac_set_config(h, None), "pfac_set_config")
        return
    c = pfac_config(**{k: int(v) for k, v in cfg.items()})
    _check(lib().pfac_set_config(h, C.byref(c)), "pfac_set_config")


def pfac_get_config(h: int, n_bases: int = 0) -> dict:
    c = pfac_config()
    _check(lib().pfac_get_config(h, n_bases, C.byref(c)), "pfac_get_config")
    return {f: getattr(c, f) for f, _ in pfac_config._fields_}


def pfac_pack(d_text, d_packed, d_status=None, d_bad=None, stream=None):
    _check(lib().pfac_pack(_dptr(d_text), d_text.numel(), _dptr(d_packed), _dptr(d_status), _dptr(d_bad),
                           _stream(stream)), "pfac_pack")


def pfac_match(h: int, d_text, d_out_ids, stream=None, length: int | None = None):
    n = d_text.numel() if length is None else length
    _check(lib().pfac_match(h, _dptr(d_text), n, _dptr(d_out_ids), _stream(stream)), "pfac_match")


def pfac_match_packed(h: int, d_packed, n_bases: int, d_out_ids, stream=None):
    _check(lib().pfac_match_packed(h, _dptr(d_packed), n_bases, _dptr(d_out_ids), _stream(stream)),
           "pfac_match_packed")


def pfac_match_compact(h: int, d_packed, n_bases: int, d_offsets, d_ids, d_count, stream=None):
    cap = 0 if d_offsets is None else d_offsets.numel()
    _check(lib().pfac_match_compact(h, _dptr(d_packed), n_bases, _dptr(d_offsets), _dptr(d_ids), cap,
                                    _dptr(d_count), _stream(stream)), "pfac_match_compact")


def pfac_match_all(h: int, d_packed, n_bases: int, d_offsets, d_ids, d_count, stream=None):
    """Every (offset, id) occurrence, sub-patterns included (see include/pfac.h)."""
    cap = 0 if d_offsets is None else d_offsets.numel()
    _check(lib().pfac_match_all(h, _dptr(d_packed), n_bases, _dptr(d_offsets), _dptr(d_ids), cap,
                                _dptr(d_count), _stream(stream)), "pfac_match_all")


def pfac_match_batched(handles, d_texts, d_read_offsets, d_read_set, d_out_ids, stream=None):
    """Scan every read (``d_texts[off[r]:off[r+1]]``) with the table ``handles[d_read_set[r]]``."""
    arr = (C.c_void_p * max(1, len(handles)))(*handles)
    n_reads = d_read_set.numel()
    _check(lib().pfac_match_batched(arr, len(handles), _dptr(d_texts), d_texts.numel(), _dptr(d_read_offsets),
                                    _dptr(d_read_set), n_reads, _dptr(d_out_ids), _stream(stream)),
           "pfac_match_batched")


def pfac_match_packed_noalloc(h: int, d_packed, n_bases: int, d_out_ids, stream=None):
    """pfac_match_packed with the library's fixed scratch buffer: no device allocation."""
    _check(lib().pfac_match_packed_noalloc(h, _dptr(d_packed), n_bases, _dptr(d_out_ids), _stream(stream)),
           "pfac_match_packed_noalloc")


def pfac_device_status(h: int, stream=None) -> int:
    s = I32()
    _check(lib().pfac_device_status(h, C.byref(s), _stream(stream)), "pfac_device_status")
    return s.value


def pfac_debug_timeout_probe(d_status, limit_ns: int, stream=None):
    _check(lib().pfac_debug_timeout_probe(_dptr(d_status), limit_ns, _stream(stream)), "pfac_debug_timeout_probe")


# ---------------------------------------------------------------------------
# Convenience owner of a handle.
# ---------------------------------------------------------------------------

class Table:
    """Owns one table handle; destroys it when collected or closed."""

    def __init__(self, patterns, host_only: bool = False, filter_b: int = 0, sample: int = 0):
        self.h = pfac_build(patterns, host_only=host_only, filter_b=filter_b, sample=sample)

    @classmethod
    def from_device(cls, d_blob, d_offsets, filter_b: int = 0, sample: int = 0, stream=None) -> "Table":
        """A table built on the GPU (pfac_build_device) from device tensors."""
        t = cls.__new__(cls)
        t.h = pfac_build_device(d_blob, d_offsets, filter_b=filter_b, sample=sample, stream=stream)
        return t

    @classmethod
    def from_file(cls, path: str, host_only: bool = False, filter_b: int = 0) -> "Table":
        t = cls.__new__(cls)
        t.h = pfac_build_file(path, host_only=host_only, filter_b=filter_b)
        return t

    def close(self):
        """Destroy the handle (no launch using it may still be in flight); a second call
        does nothing, and calls on a closed table raise PfacError."""
        h, self.h = getattr(self, "h", None), None
        if h:
            lib().pfac_destroy(h)

    def __enter__(self) -> "Table":
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def info(self) -> dict:
        return pfac_info_ex(self.h)

    def set_config(self, **cfg):
        pfac_set_config(self.h, cfg or None)

    def match(self, d_text, d_out=None, stream=None):
        import torch
        if d_out is None:
            d_out = torch.empty(d_text.numel(), dtype=torch.int32, device=d_text.device)
        pfac_match(self.h, d_text, d_out, stream)
        return d_out

    def match_packed(self, d_packed, n_bases: int, d_out=None, stream=None):
        import torch
        if d_out is None:
            d_out = torch.empty(n_bases, dtype=torch.int32, device=d_packed.device)
        pfac_match_packed(self.h, d_packed, n_bases, d_out, stream)
        return d_out


def pack(d_text, stream=None):
    """Pack an ASCII CUDA uint8 tensor; returns (packed words, status, first bad offset)."""
    import torch
    n = d_text.numel()
    packed = torch.empty((n + 15) // 16, dtype=torch.int32, device=d_text.device)
    status = torch.empty(1, dtype=torch.int32, device=d_text.device)
    bad = torch.empty(1, dtype=torch.int64, device=d_text.device)
    pfac_pack(d_text, packed, status, bad, stream)
    return packed, status, bad
