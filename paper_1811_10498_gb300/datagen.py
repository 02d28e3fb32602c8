"""Seeded synthetic inputs for the PFAC scan: DNA texts, pattern sets, read batches
and request streams.

This module only *makes inputs*. It holds none of the matching arithmetic (no trie,
no packing, no walk), so both the CUDA path and the CPU oracle can take their
inputs from it without sharing any of the method.

The paper's own pattern files and input data sets are not available (Table III lists
1,000-5,000 patterns of about 100 bases; Table IV lists 0.75M-3.75M newline-separated
reads of about 100 bases). Every generator here is a seeded stand-in with the
shapes, sizes and base composition of the five workloads below. All randomness
comes from ``numpy.random.Generator(PCG64(seed))``.

Texts are ASCII ``uint8`` arrays over ``b"ACGT"``. A pattern set is returned as a
pair ``(blob, offsets)``: ``blob`` is every pattern concatenated (``uint8``) and
pattern ``j`` (0-based; its id is ``j + 1``) is ``blob[offsets[j]:offsets[j+1]]``.
"""
from __future__ import annotations

import functools
import hashlib
import math
from dataclasses import dataclass, field

import numpy as np

ALPHABET = np.frombuffer(b"ACGT", dtype=np.uint8)
# Base composition at 41 % GC (A = T, C = G).
GC41 = (0.295, 0.205, 0.205, 0.295)
UNIFORM = (0.25, 0.25, 0.25, 0.25)

_CHUNK = 1 << 26  # bases generated per chunk, bounds temporary memory


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def sha256(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).view(np.uint8)).hexdigest()


def _lut16(probs) -> np.ndarray:
    """Table that maps a uniform 16-bit draw to a base with the given probabilities."""
    cum = np.cumsum(np.asarray(probs, dtype=np.float64))
    cum[-1] = 1.0
    cuts = np.round(cum * 65536.0).astype(np.int64)
    lut = np.empty(65536, dtype=np.uint8)
    lo = 0
    for b, hi in enumerate(cuts):
        lut[lo:hi] = ALPHABET[b]
        lo = hi
    return lut


def iid_text(n: int, rng: np.random.Generator, probs=UNIFORM) -> np.ndarray:
    """``n`` i.i.d. bases (probabilities quantised to 1/65536)."""
    lut = _lut16(probs)
    out = np.empty(n, dtype=np.uint8)
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        out[lo:hi] = lut[rng.integers(0, 65536, hi - lo, dtype=np.uint16)]
    return out


# ----------------------------------------------------------------------------
# Order-2 Markov chain with 41 % stationary GC.
#
# P(x_t | x_{t-2}, x_{t-1}) is proportional to w[x_t] * m(x_{t-2}, x_{t-1}, x_t) with
#   w = (a, c, c, a), a + c = 1/2                    (strand-symmetric base weights)
#   m = 0.25 when x_{t-1} = C and x_t = G            (CpG depletion)
#   m = 1.25 when x_{t-2} = x_{t-1} = x_t in {A, T}  (A/T homopolymer runs)
#   m = 1 otherwise.
# ``c`` is set by bisection so that the chain's stationary G+C fraction is 0.41. The
# stationary composition is then A = T = 29.5 %, C = 22.75 %, G = 18.25 %: the mass
# taken from G after C goes to the other bases, so C and G differ.
# ----------------------------------------------------------------------------

def _markov2_matrix(c: float) -> np.ndarray:
    w = np.array([0.5 - c, c, c, 0.5 - c])
    P = np.empty((16, 4))
    for ctx in range(16):
        p2, p1 = divmod(ctx, 4)
        row = w.copy()
        if p1 == 1:
            row[2] *= 0.25
        if p2 == p1 and p1 in (0, 3):
            row[p1] *= 1.25
        P[ctx] = row / row.sum()
    return P


def _stationary_pairs(P: np.ndarray) -> np.ndarray:
    T = np.zeros((16, 16))
    for ctx in range(16):
        p1 = ctx % 4
        for b in range(4):
            T[ctx, p1 * 4 + b] = P[ctx, b]
    pi = np.full(16, 1.0 / 16)
    for _ in range(2000):
        pi = pi @ T
    return pi / pi.sum()


def _gc_of(P: np.ndarray) -> float:
    pi = _stationary_pairs(P)
    last = pi.reshape(4, 4).sum(axis=0)
    return float(last[1] + last[2])


@functools.lru_cache(maxsize=None)
def _chain(gc: float):
    """For a stationary G+C fraction ``gc``: the transition matrix (found by bisection
    on ``c``), its sampling table (16 contexts x 65536 uniform 16-bit draws) and its
    stationary pair distribution. Computed once per ``gc``; callers must not modify
    the arrays."""
    lo, hi = 0.01, 0.49
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if _gc_of(_markov2_matrix(mid)) < gc:
            lo = mid
        else:
            hi = mid
    P = _markov2_matrix(0.5 * (lo + hi))
    cum = np.cumsum(P, axis=1)
    cum[:, -1] = 1.0
    lut = np.empty((16, 65536), dtype=np.uint8)
    for ctx in range(16):
        cuts = np.round(cum[ctx] * 65536.0).astype(np.int64)
        lo_i = 0
        for b, hi_i in enumerate(cuts):
            lut[ctx, lo_i:hi_i] = b
            lo_i = hi_i
    return P, lut, _stationary_pairs(P)


def markov2_matrix(gc: float = 0.41) -> np.ndarray:
    return _chain(float(gc))[0].copy()


def markov2_text(n: int, rng: np.random.Generator, gc: float = 0.41,
                 segment: int = 4096) -> np.ndarray:
    """``n`` bases of the order-2 chain above.

    The text is a concatenation of independent stationary segments of ``segment``
    bases, generated side by side so the loop runs over positions, not bases.
    Each segment starts from the stationary pair distribution, so every base has
    the chain's stationary statistics; only the ``n / segment`` seams are not
    conditioned on the base before them.
    """
    if n == 0:
        return np.empty(0, dtype=np.uint8)
    _, lut, pairs = _chain(float(gc))
    n_seg = (n + segment - 1) // segment
    out = np.empty((segment, n_seg), dtype=np.uint8)  # position-major
    first = rng.choice(16, size=n_seg, p=pairs)
    out[0] = first // 4
    if segment > 1:
        out[1] = first % 4
    ctx = first.astype(np.int64)
    for t in range(2, segment):
        r = rng.integers(0, 65536, n_seg, dtype=np.uint16)
        nxt = lut[ctx, r]
        out[t] = nxt
        ctx = (ctx % 4) * 4 + nxt
    codes = np.ascontiguousarray(out.T).reshape(-1)[:n]
    return ALPHABET[codes]


def plant_repeats(text: np.ndarray, rng: np.random.Generator, frac: float = 0.05,
                  n_units: int = 200, len_range=(300, 6000), gc: float = 0.41) -> int:
    """Overwrite about ``frac`` of ``text`` (in place) with exact copies of
    ``n_units`` repeat units whose lengths are uniform in ``len_range``, drawn from
    the same chain. Copies land at uniform positions. Returns the bases planted."""
    n = text.shape[0]
    lo, hi = len_range
    if n < hi:
        return 0
    lengths = rng.integers(lo, hi + 1, n_units)
    units = [markov2_text(int(L), rng, gc) for L in lengths]
    target = int(frac * n)
    planted = 0
    while planted < target:
        u = units[int(rng.integers(0, n_units))]
        pos = int(rng.integers(0, n - u.shape[0] + 1))
        text[pos:pos + u.shape[0]] = u
        planted += u.shape[0]
    return planted


def mutate(seq: np.ndarray, rng: np.random.Generator, rate: float) -> np.ndarray:
    """Independent point substitutions: each base, with probability ``rate``, becomes
    one of the other three bases uniformly."""
    seq = seq.copy()
    hit = rng.random(seq.shape[0]) < rate
    if hit.any():
        code = np.searchsorted(ALPHABET, seq[hit])
        code = (code + rng.integers(1, 4, code.shape[0])) % 4
        seq[hit] = ALPHABET[code]
    return seq


def pattern_set(text: np.ndarray, rng: np.random.Generator, n: int, len_range,
                frac_substr: float, random_probs=UNIFORM, mutation: float = 0.0):
    """``n`` patterns with lengths uniform in ``len_range`` (inclusive). The first
    ``round(frac_substr * n)`` are copies of ``text`` at uniform offsets (each base
    then mutated with probability ``mutation``); the rest are i.i.d. with
    ``random_probs``. Returned as ``(blob, offsets)``."""
    lo, hi = len_range
    lengths = rng.integers(lo, hi + 1, n).astype(np.int64)
    n_sub = int(round(frac_substr * n))
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    blob = np.empty(int(offsets[-1]), dtype=np.uint8)
    if n_sub:
        ln = lengths[:n_sub]
        starts = (rng.random(n_sub) * (text.shape[0] - ln + 1)).astype(np.int64)
        idx = np.repeat(starts - offsets[:n_sub], ln) + np.arange(int(offsets[n_sub]))
        sub = text[idx]
        if mutation > 0.0:
            sub = mutate(sub, rng, mutation)
        blob[:offsets[n_sub]] = sub
    if n_sub < n:
        blob[offsets[n_sub]:] = iid_text(int(offsets[-1] - offsets[n_sub]), rng, random_probs)
    return blob, offsets


def pattern_list(blob: np.ndarray, offsets: np.ndarray) -> list[bytes]:
    raw = blob.tobytes()
    return [raw[offsets[j]:offsets[j + 1]] for j in range(offsets.shape[0] - 1)]


def patterns_from_list(pats) -> tuple[np.ndarray, np.ndarray]:
    lens = np.array([len(p) for p in pats], dtype=np.int64)
    offsets = np.zeros(len(pats) + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    blob = np.frombuffer(b"".join(bytes(p) for p in pats), dtype=np.uint8).copy()
    return blob, offsets


# ----------------------------------------------------------------------------
# The five workloads.
# ----------------------------------------------------------------------------

@dataclass
class SingleScan:
    name: str
    text: np.ndarray          # ASCII uint8
    blob: np.ndarray          # patterns, concatenated
    offsets: np.ndarray       # n + 1 pattern offsets into blob
    meta: dict = field(default_factory=dict)

    @property
    def n_patterns(self) -> int:
        return int(self.offsets.shape[0] - 1)


def small_scan(seed: int = 1, n_bases: int = 1_000_000, n_patterns: int = 1000) -> SingleScan:
    """Plain PFAC, small: ``n_bases`` i.i.d. uniform bases; ``n_patterns`` patterns of
    length U[8, 32], half text substrings at uniform offsets, half uniform random."""
    rng = rng_for(seed)
    text = iid_text(n_bases, rng, UNIFORM)
    blob, offsets = pattern_set(text, rng, n_patterns, (8, 32), 0.5, UNIFORM)
    return SingleScan(f"small uniform text {n_bases} bases, {n_patterns} patterns len 8-32",
                      text, blob, offsets, {"seed": seed})


def genome_scan(seed: int = 2, n_bases: int = 256 << 20, n_patterns: int = 20_000) -> SingleScan:
    """Genome-scale scan: ``n_bases`` of the 41 %-GC order-2 chain with 5 % of its length
    overwritten by copies of 200 repeat units of 300-6,000 bases; ``n_patterns``
    patterns of length U[20, 100], 70 % text substrings with 1 % point mutations,
    30 % i.i.d. at 41 % GC."""
    rng = rng_for(seed)
    text = markov2_text(n_bases, rng, 0.41)
    planted = plant_repeats(text, rng, 0.05, 200, (300, 6000), 0.41)
    blob, offsets = pattern_set(text, rng, n_patterns, (20, 100), 0.7, GC41, mutation=0.01)
    return SingleScan(f"genome-scale order-2 Markov 41% GC text {n_bases} bases + 5% repeats, "
                      f"{n_patterns} patterns len 20-100",
                      text, blob, offsets, {"seed": seed, "planted": planted})


def large_dict_scan(seed: int = 3, n_bases: int = 1 << 30, n_patterns: int = 1_000_000) -> SingleScan:
    """Large dictionary: ``n_bases`` i.i.d. at 41 % GC; ``n_patterns`` patterns of length
    U[16, 64], half text substrings, half i.i.d. at 41 % GC."""
    rng = rng_for(seed)
    text = iid_text(n_bases, rng, GC41)
    blob, offsets = pattern_set(text, rng, n_patterns, (16, 64), 0.5, GC41)
    return SingleScan(f"large dictionary i.i.d. 41% GC text {n_bases} bases, "
                      f"{n_patterns} patterns len 16-64",
                      text, blob, offsets, {"seed": seed})


@dataclass
class ReadBatch:
    name: str
    reads: np.ndarray          # all reads concatenated (ASCII uint8)
    read_offsets: np.ndarray   # n_reads + 1 (int64)
    read_set: np.ndarray       # n_reads (int32): index of the pattern set for each read
    sets: list                 # [(blob, offsets)]
    meta: dict = field(default_factory=dict)


def _log_uniform_int(rng, lo, hi, size):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size)).astype(np.int64)


def read_batch(seed: int = 4, n_reads: int = 4096, n_sets: int = 64, source_bases: int = 64 << 20,
               median: float = 1500.0, sigma: float = 1.0, len_clip=(100, 100_000),
               set_range=(100, 50_000), pat_len=(12, 64)) -> ReadBatch:
    """Batched workload: ``n_reads`` reads with log-normal lengths (median ``median``,
    sigma ``sigma``, clipped to ``len_clip``) cut at uniform offsets from a
    ``source_bases`` order-2 Markov source at 41 % GC; ``n_sets`` pattern sets of
    log-uniform size in ``set_range`` with lengths U[``pat_len``], half source
    substrings and half i.i.d.; each read assigned a set uniformly."""
    rng = rng_for(seed)
    src_n = max(source_bases, len_clip[1] + 1)
    source = markov2_text(src_n, rng, 0.41)
    lens = np.clip(np.round(rng.lognormal(math.log(median), sigma, n_reads)),
                   len_clip[0], len_clip[1]).astype(np.int64)
    read_offsets = np.zeros(n_reads + 1, dtype=np.int64)
    np.cumsum(lens, out=read_offsets[1:])
    starts = (rng.random(n_reads) * (src_n - lens + 1)).astype(np.int64)
    idx = np.repeat(starts - read_offsets[:-1], lens) + np.arange(int(read_offsets[-1]))
    reads = source[idx]
    sizes = _log_uniform_int(rng, set_range[0], set_range[1], n_sets)
    sets = [pattern_set(source, rng, int(s), pat_len, 0.5, GC41) for s in sizes]
    read_set = rng.integers(0, n_sets, n_reads).astype(np.int32)
    return ReadBatch(f"{n_reads} reads log-normal median {int(median)} vs {n_sets} sets "
                     f"of {set_range[0]}-{set_range[1]} patterns len {pat_len[0]}-{pat_len[1]}",
                     reads, read_offsets, read_set, sets,
                     {"seed": seed, "set_sizes": sizes.tolist()})


@dataclass
class RequestStream:
    name: str
    arrivals: np.ndarray       # seconds from start, increasing
    set_id: np.ndarray         # pattern set per request
    starts: np.ndarray         # window start in ``source`` per request
    lengths: np.ndarray        # text length per request
    source: np.ndarray         # ASCII source the request texts are cut from
    sets: list                 # [(blob, offsets)]
    meta: dict = field(default_factory=dict)

    def text(self, r: int) -> np.ndarray:
        s = int(self.starts[r])
        return self.source[s:s + int(self.lengths[r])]


def request_stream(seed: int = 5, rate: float = 2000.0, duration: float = 2.0, n_sets: int = 16,
                   set_range=(1000, 200_000), pat_len=(16, 64), text_range=(1000, 10_000_000),
                   source_bases: int = 32 << 20) -> RequestStream:
    """Serving workload: Poisson arrivals at ``rate`` per second for ``duration``
    seconds; each request names one of ``n_sets`` resident sets (log-uniform sizes in
    ``set_range``, lengths U[``pat_len``], half source substrings) and a text whose
    length is log-uniform in ``text_range``, cut from a 41 %-GC order-2 source."""
    rng = rng_for(seed)
    src_n = max(source_bases, text_range[1] + 1)
    source = markov2_text(src_n, rng, 0.41)
    sizes = _log_uniform_int(rng, set_range[0], set_range[1], n_sets)
    sets = [pattern_set(source, rng, int(s), pat_len, 0.5, GC41) for s in sizes]
    gaps = rng.exponential(1.0 / rate, int(rate * duration * 1.5) + 16)
    arrivals = np.cumsum(gaps)
    arrivals = arrivals[arrivals < duration]
    n = arrivals.shape[0]
    lengths = _log_uniform_int(rng, text_range[0], text_range[1], n)
    starts = (rng.random(n) * (src_n - lengths + 1)).astype(np.int64)
    set_id = rng.integers(0, n_sets, n).astype(np.int32)
    return RequestStream(f"Poisson {rate:g} req/s for {duration:g} s, {n_sets} sets of "
                         f"{set_range[0]}-{set_range[1]} patterns, texts "
                         f"{text_range[0]}-{text_range[1]} bases",
                         arrivals, set_id, starts, lengths, source, sets,
                         {"seed": seed, "set_sizes": sizes.tolist()})


# ----------------------------------------------------------------------------
# The paper's own workload shape (Tables III and IV), standing in for its files:
# pattern sets of 1,000-5,000 patterns of about 100 bases, and input data sets of
# 0.75-3.75 million newline-separated lines of about 100 bases (about 101 bytes per
# line with its newline: 76-380 MB).
# ----------------------------------------------------------------------------

PAPER_LINE = 100          # bases per line of an input data set
PAPER_PATTERN = 100       # bases per pattern


def paper_source(seed: int = 6, n_bases: int = 64 << 20) -> np.ndarray:
    """The genome-like source that lines and patterns are cut from (41 %-GC order-2
    chain)."""
    return markov2_text(n_bases, rng_for(seed), 0.41)


def paper_input(source: np.ndarray, n_lines: int, seed: int = 7, line: int = PAPER_LINE) -> np.ndarray:
    """``n_lines`` lines of ``line`` bases cut at uniform offsets of ``source``, each
    followed by a newline (ASCII uint8). A newline has no edge in the trie, so no walk
    crosses from one line into the next."""
    rng = rng_for(seed)
    starts = (rng.random(n_lines) * (source.shape[0] - line + 1)).astype(np.int64)
    out = np.empty((n_lines, line + 1), dtype=np.uint8)
    idx = starts[:, None] + np.arange(line)[None, :]
    out[:, :line] = source[idx]
    out[:, line] = ord("\n")
    return out.reshape(-1)


def paper_patterns(source: np.ndarray, n: int, seed: int = 8, length: int = PAPER_PATTERN):
    """``n`` patterns of ``length`` bases: half copies of ``source`` at uniform offsets,
    half i.i.d. at 41 % GC. Returned as ``(blob, offsets)``."""
    return pattern_set(source, rng_for(seed), n, (length, length), 0.5, GC41)
