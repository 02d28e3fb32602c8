"""CPU oracle for the PFAC scan — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package. The CUDA library never calls it, and it imports nothing
from the CUDA library or its Python binding.

Contents:
  * ``pfac_oracle.c`` (built into ``liboracle.so`` with the host C compiler): the
    insertion-order goto trie (Section V-A; Section III, Fig. 1), the failure-less
    per-offset scan (Section IV), and a classic Aho-Corasick machine with failure
    links (Section III, Fig. 2) used only as a cross-check;
  * ``brute.py``: pure-Python brute force and a regular-expression restatement for
    tiny inputs;
  * ``pack`` and ``compact`` below: the plain definitions of the 2-bit text packing
    and of the (offset, id) match list that the CUDA library produces;
  * ``all_matches``: every pattern occurrence keyed by its start, from the classic
    Aho-Corasick machine's occurrence list (the reference for the all-matches scan).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pfac_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

_lock = threading.Lock()
_libs: dict[str, C.CDLL] = {}


def build(force: bool = False, src: str = SRC, out: str = LIB) -> str:
    """Compile the C oracle with the host compiler (gcc)."""
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", src, "-o", tmp],
                       check=True)
        os.replace(tmp, out)
    return out


def load(path: str | None = None) -> C.CDLL:
    """Load (building if needed) the oracle library; ``path`` selects another build
    of the same source, which the mutation tests use."""
    with _lock:
        if path is None:
            path = build()
        lib = _libs.get(path)
        if lib is None:
            lib = C.CDLL(path)
            P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
            lib.oracle_trie_build.restype = P
            lib.oracle_trie_build.argtypes = [P, P, I32, P]
            lib.oracle_trie_free.argtypes = [P]
            lib.oracle_trie_states.restype = I64
            lib.oracle_trie_states.argtypes = [P]
            lib.oracle_trie_export.argtypes = [P, P, P]
            lib.oracle_pfac_scan.argtypes = [P, P, I64, I64, I64, P]
            lib.oracle_ac_build.restype = P
            lib.oracle_ac_build.argtypes = [P, P, I32, P]
            lib.oracle_ac_free.argtypes = [P]
            lib.oracle_ac_states.restype = I64
            lib.oracle_ac_states.argtypes = [P]
            lib.oracle_ac_export_fail.argtypes = [P, P]
            lib.oracle_ac_output.restype = I64
            lib.oracle_ac_output.argtypes = [P, I32, P, I64]
            lib.oracle_ac_scan.restype = I64
            lib.oracle_ac_scan.argtypes = [P, P, I64, P, P, P, I64]
            _libs[path] = lib
        return lib


class OracleError(RuntimeError):
    CODES = {1: "bad argument", 2: "empty pattern", 3: "pattern byte outside ACGT", 4: "out of memory"}

    def __init__(self, code: int):
        super().__init__(self.CODES.get(code, f"error {code}"))
        self.code = code


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _as_patterns(patterns):
    """Accept ``(blob, offsets)`` or a list of byte strings."""
    if isinstance(patterns, tuple):
        blob, offsets = patterns
    else:
        lens = np.array([len(p) for p in patterns], dtype=np.int64)
        offsets = np.zeros(len(patterns) + 1, dtype=np.int64)
        np.cumsum(lens, out=offsets[1:])
        blob = np.frombuffer(b"".join(bytes(p) for p in patterns) or b"\0", dtype=np.uint8)
    blob = np.ascontiguousarray(blob, dtype=np.uint8)
    if blob.size == 0:
        blob = np.zeros(1, dtype=np.uint8)
    return blob, np.ascontiguousarray(offsets, dtype=np.int64)


def _as_text(text) -> np.ndarray:
    if isinstance(text, (bytes, bytearray)):
        text = np.frombuffer(bytes(text), dtype=np.uint8)
    return np.ascontiguousarray(text, dtype=np.uint8)


class Trie:
    """Insertion-order goto trie (states numbered as they are created)."""

    def __init__(self, patterns, lib: C.CDLL | None = None):
        self.lib = lib or load()
        blob, offsets = _as_patterns(patterns)
        err = C.c_int32(0)
        self.h = self.lib.oracle_trie_build(_ptr(blob), _ptr(offsets), offsets.shape[0] - 1,
                                            C.byref(err))
        if not self.h:
            raise OracleError(err.value)
        self.n_patterns = offsets.shape[0] - 1

    def __del__(self):
        h, self.h = getattr(self, "h", None), None
        if h:
            self.lib.oracle_trie_free(h)

    @property
    def n_states(self) -> int:
        return int(self.lib.oracle_trie_states(self.h))

    def export(self):
        """``(go[S, 4], term[S])``: next state per column A, C, G, T (0 = none) and the
        id of the pattern ending at each state (0 = none)."""
        S = self.n_states
        go = np.zeros((S, 4), dtype=np.int32)
        term = np.zeros(S, dtype=np.int32)
        self.lib.oracle_trie_export(self.h, _ptr(go), _ptr(term))
        return go, term

    def scan(self, text, begin: int = 0, end: int | None = None,
             out: np.ndarray | None = None) -> np.ndarray:
        """Longest-pattern id for each offset in ``[begin, end)`` (``out`` is indexed
        by text offset)."""
        t = _as_text(text)
        n = t.shape[0]
        end = n if end is None else end
        if out is None:
            out = np.zeros(n, dtype=np.int32)
        if end > begin:
            self.lib.oracle_pfac_scan(self.h, _ptr(t) if n else None, n, begin, end, _ptr(out))
        return out

    def scan_threads(self, text, threads: int, begin: int = 0, end: int | None = None) -> np.ndarray:
        """The same scan with the offsets split into ``threads`` contiguous ranges run
        on host threads (the C call releases the interpreter lock)."""
        t = _as_text(text)
        n = t.shape[0]
        end = n if end is None else end
        out = np.zeros(n, dtype=np.int32)
        step = max(1, -(-(end - begin) // max(1, threads)))
        ranges = [(lo, min(end, lo + step)) for lo in range(begin, end, step)]
        with ThreadPoolExecutor(max_workers=max(1, threads)) as ex:
            list(ex.map(lambda r: self.lib.oracle_pfac_scan(self.h, _ptr(t), n, r[0], r[1],
                                                            _ptr(out)), ranges))
        return out


class AhoCorasick:
    """Classic Aho-Corasick machine with failure links (Section III, Fig. 2)."""

    def __init__(self, patterns, lib: C.CDLL | None = None):
        self.lib = lib or load()
        blob, offsets = _as_patterns(patterns)
        err = C.c_int32(0)
        self.h = self.lib.oracle_ac_build(_ptr(blob), _ptr(offsets), offsets.shape[0] - 1,
                                          C.byref(err))
        if not self.h:
            raise OracleError(err.value)

    def __del__(self):
        h, self.h = getattr(self, "h", None), None
        if h:
            self.lib.oracle_ac_free(h)

    @property
    def n_states(self) -> int:
        return int(self.lib.oracle_ac_states(self.h))

    def failure(self) -> np.ndarray:
        f = np.zeros(self.n_states, dtype=np.int32)
        self.lib.oracle_ac_export_fail(self.h, _ptr(f))
        return f

    def output(self, s: int) -> list[int]:
        buf = np.zeros(4096, dtype=np.int32)
        k = self.lib.oracle_ac_output(self.h, s, _ptr(buf), buf.shape[0])
        return sorted(buf[:min(k, buf.shape[0])].tolist())

    def longest(self, text) -> np.ndarray:
        """For each start, the longest pattern found there by the sequential machine."""
        t = _as_text(text)
        out = np.zeros(t.shape[0], dtype=np.int32)
        if t.shape[0]:
            self.lib.oracle_ac_scan(self.h, _ptr(t), t.shape[0], _ptr(out), None, None, 0)
        return out

    def occurrences(self, text, cap: int = 1 << 20):
        """All (end position, pattern id) occurrences, in text order."""
        t = _as_text(text)
        ends = np.zeros(cap, dtype=np.int64)
        ids = np.zeros(cap, dtype=np.int32)
        total = self.lib.oracle_ac_scan(self.h, _ptr(t) if t.shape[0] else None, t.shape[0],
                                        None, _ptr(ends), _ptr(ids), cap)
        if total > cap:
            raise ValueError(f"{total} occurrences exceed cap {cap}")
        return ends[:total], ids[:total]


def pfac_scan(text, patterns, threads: int = 1) -> np.ndarray:
    """Longest-pattern id per offset of ``text`` (0 = none)."""
    trie = Trie(patterns)
    return trie.scan_threads(text, threads) if threads > 1 else trie.scan(text)


def pfac_scan_reads(reads, read_offsets, read_set, sets) -> np.ndarray:
    """Batched form: each read is scanned on its own (a walk never crosses the read's
    end) with the trie of its pattern set; outputs keep the reads' layout."""
    reads = _as_text(reads)
    out = np.zeros(reads.shape[0], dtype=np.int32)
    tries = {}
    for r in range(read_set.shape[0]):
        k = int(read_set[r])
        if k not in tries:
            tries[k] = Trie(sets[k])
        lo, hi = int(read_offsets[r]), int(read_offsets[r + 1])
        out[lo:hi] = tries[k].scan(reads[lo:hi])
    return out


# 2-bit codes of the packed text: A=0, C=1, G=2, T=3.
_CODE = np.full(256, 255, dtype=np.uint8)
for _b, _c in zip(b"ACGT", range(4)):
    _CODE[_b] = _c


def pack(text):
    """Packed layout of a text over {A,C,G,T}: base p occupies bits 2*(p mod 16) ..
    2*(p mod 16)+1 of 32-bit word p // 16; bases past the end are 0. Returns
    ``(words, first_bad)`` with ``first_bad`` the first offset holding a byte
    outside {A,C,G,T}, or -1."""
    t = _as_text(text)
    codes = _CODE[t]
    bad = np.flatnonzero(codes == 255)
    first_bad = int(bad[0]) if bad.size else -1
    n_words = -(-t.shape[0] // 16)
    padded = np.zeros(n_words * 16, dtype=np.uint32)
    padded[:t.shape[0]] = np.where(codes == 255, 0, codes)
    shifts = (2 * np.arange(16, dtype=np.uint32))
    words = (padded.reshape(n_words, 16) << shifts).sum(axis=1, dtype=np.uint64).astype(np.uint32)
    return words, first_bad


def compact(out_ids: np.ndarray):
    """The match list: every offset with a non-zero id, ascending, with its id."""
    offs = np.flatnonzero(out_ids).astype(np.int64)
    return offs, out_ids[offs].astype(np.int32)


def all_matches(patterns, text, cap: int = 1 << 24, lib: C.CDLL | None = None):
    """Every pattern occurrence, as the walk that reports each terminal state it passes
    would list it (not only the last one, as the PFAC scan of Section IV does): one
    ``(start, id)`` per start offset and distinct pattern string occurring there, with
    the lowest id of that string, sorted by start and then by length. Computed from the
    classic Aho-Corasick machine's occurrence list (Section III), whose (end, id) pairs
    are turned into starts. Returns ``(starts int64, ids int32)``."""
    blob, offsets = _as_patterns(patterns)
    lengths = np.diff(offsets)
    ends, ids = AhoCorasick((blob, offsets), lib).occurrences(text, cap)
    if ends.size == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int32)
    lens = lengths[ids - 1]
    starts = ends - lens + 1
    # equal strings at one start: keep the lowest id
    order = np.lexsort((ids, lens, starts))
    starts, lens, ids = starts[order], lens[order], ids[order]
    keep = np.ones(starts.size, dtype=bool)
    keep[1:] = (starts[1:] != starts[:-1]) | (lens[1:] != lens[:-1])
    return starts[keep].astype(np.int64), ids[keep].astype(np.int32)
