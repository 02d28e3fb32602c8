"""Pure-Python checkers for tiny inputs — TEST INFRASTRUCTURE ONLY.

Two restatements of what the PFAC scan returns (Section IV: the id of the longest
pattern that starts at each offset), written without any automaton:

* ``brute_longest``: compare every pattern at every offset;
* ``regex_longest``: a regular-expression lookahead over the patterns sorted by
  decreasing length. Patterns that match at one offset are prefixes of one another,
  so the first alternative that matches there is the longest one.

Ids are 1-based in input order; 0 = no match; a repeated string keeps its lowest id.
"""
from __future__ import annotations

import re


def brute_longest(text: bytes, patterns: list[bytes]) -> list[int]:
    out = [0] * len(text)
    for i in range(len(text)):
        best_len = 0
        for j, p in enumerate(patterns):
            if len(p) > best_len and text.startswith(p, i):
                best_len = len(p)
                out[i] = j + 1
    return out


def regex_longest(text: bytes, patterns: list[bytes]) -> list[int]:
    lowest = {}
    for j, p in enumerate(patterns):
        lowest.setdefault(bytes(p), j + 1)
    alts = sorted(lowest, key=len, reverse=True)
    rx = re.compile(b"(?=(" + b"|".join(re.escape(p) for p in alts) + b"))")
    out = [0] * len(text)
    for m in rx.finditer(text):
        out[m.start()] = lowest[m.group(1)]
    return out


def occurrences(text: bytes, patterns: list[bytes]) -> list[tuple[int, int]]:
    """Every (end position, id) with ``text[end-len+1 .. end] == pattern``, sorted."""
    occ = []
    for j, p in enumerate(patterns):
        start = text.find(p)
        while start >= 0:
            occ.append((start + len(p) - 1, j + 1))
            start = text.find(p, start + 1)
    return sorted(occ)


def brute_all(text: bytes, patterns: list[bytes]) -> list[tuple[int, int]]:
    """Every (start, id) with ``text[start:start+len] == pattern``, one per start and
    distinct string (its lowest id), sorted by start then length."""
    lowest = {}
    for j, p in enumerate(patterns):
        lowest.setdefault(bytes(p), j + 1)
    out = []
    for i in range(len(text)):
        for p, pid in sorted(lowest.items(), key=lambda kv: len(kv[0])):
            if text.startswith(p, i):
                out.append((i, pid))
    return out
