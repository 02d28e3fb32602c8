"""Checks that pin the CPU oracle to the paper and to the mathematics.

Each check takes an oracle library handle so that the same checks can be run against
deliberately broken builds of the oracle (see test_oracle_mutants.py). A check raises
AssertionError when the oracle disagrees with the pinned fact.
"""
from __future__ import annotations

import os
import random

import numpy as np

import oracle
from oracle import brute

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _patterns(rows):
    for r in rows:
        if r[0] == "patterns":
            return [p.encode() for p in r[1:]]
    raise KeyError("patterns")


def check_fig1_numbering(lib):
    """Section III, Fig. 1: AC, ACG, CTGT, TG end in states 2, 3, 7, 9 (10 states)."""
    rows = _golden("fig1_goto.txt")
    pats = _patterns(rows)
    trie = oracle.Trie(pats, lib)
    go, term = trie.export()
    want_states = int(next(r[1] for r in rows if r[0] == "states"))
    assert trie.n_states == want_states, (trie.n_states, want_states)
    want = {int(r[2]): pats.index(r[1].encode()) + 1 for r in rows if r[0] == "terminal"}
    got = {int(s): int(term[s]) for s in np.flatnonzero(term)}
    assert got == want, (got, want)


def leaf_elided_view(go, term):
    """Section V-A, Table I convention: a pattern's last symbol creates no state.

    From a trie that allocates every node, drop the terminal leaves, renumber the
    other states consecutively in creation order, and point every edge at
    new(target) = the number of kept states created before the target (for a leaf
    this is the value of the state counter when the edge was written). Each cell
    carries (new(target), id of the pattern ending at the target). Rows run from 0
    to the largest value referenced; rows past the kept states are empty."""
    S = go.shape[0]
    is_leaf = (term != 0) & (go.max(axis=1) == 0)
    kept_before = np.concatenate([[0], np.cumsum(~is_leaf)])  # kept states with index < x
    cells = {}
    for s in range(S):
        if is_leaf[s]:
            continue
        row = []
        for c in range(4):
            t = int(go[s, c])
            row.append((int(kept_before[t]), int(term[t])) if t else (0, 0))
        cells[int(kept_before[s])] = row
    n_rows = 1 + max(max(v for v, _ in row) for row in cells.values())
    return [cells.get(r, [(0, 0)] * 4) for r in range(n_rows)]


def check_table1(lib):
    """Section V-A, Table I: 13 rows, columns A, T, C, G, cell by cell."""
    rows = _golden("table1.txt")
    pats = _patterns(rows)
    cols = next(r[1:] for r in rows if r[0] == "columns")
    trie = oracle.Trie(pats, lib)
    go, term = trie.export()
    view = leaf_elided_view(go, term)
    ours_col = {"A": 0, "C": 1, "G": 2, "T": 3}
    table = [r for r in rows if r[0].isdigit()]
    assert len(view) == len(table), (len(view), len(table))
    for r in table:
        i = int(r[0])
        for k, col in enumerate(cols):
            nxt, pid = (int(v) for v in r[1 + k].split(","))
            assert view[i][ours_col[col]] == (nxt, pid), (i, col, view[i][ours_col[col]], (nxt, pid))


def check_fig2_failure(lib):
    """Section III, Fig. 2: failure links and output sets derived by hand."""
    rows = _golden("fig2_failure.txt")
    pats = _patterns(rows)
    ac = oracle.AhoCorasick(pats, lib)
    f = ac.failure()
    for r in rows:
        if r[0] == "fail":
            assert f[int(r[1])] == int(r[2]), (r, f.tolist())
    outs = {}
    for r in rows:
        if r[0] == "output":
            outs.setdefault(int(r[1]), []).append(int(r[2]))
    for s in range(ac.n_states):
        assert ac.output(s) == sorted(outs.get(s, [])), (s, ac.output(s), outs.get(s))


def check_fig1_scans(lib):
    """Hand-worked failure-less scans (Section IV rule) on the Fig. 1 patterns."""
    rows = _golden("fig1_scan.txt")
    pats = _patterns(rows)
    trie = oracle.Trie(pats, lib)
    ac = oracle.AhoCorasick(pats, lib)
    for r in rows:
        if r[0] == "scan":
            text = r[1].encode()
            want = [int(v) for v in r[2:]]
            assert trie.scan(text).tolist() == want, (r[1], trie.scan(text).tolist(), want)
            assert ac.longest(text).tolist() == want, (r[1], ac.longest(text).tolist(), want)


def random_case(rng: random.Random, alphabet=b"ACGTN\n", max_len=64, max_pats=8, max_plen=6):
    n = rng.randint(0, max_len)
    text = bytes(rng.choice(alphabet) for _ in range(n))
    pats = []
    for _ in range(rng.randint(1, max_pats)):
        L = rng.randint(1, max_plen)
        if n >= L and rng.random() < 0.6:
            s = rng.randint(0, n - L)
            cand = text[s:s + L]
            if all(b in b"ACGT" for b in cand):
                pats.append(cand)
                continue
        pats.append(bytes(rng.choice(b"ACGT") for _ in range(L)))
    if rng.random() < 0.2:
        pats.append(rng.choice(pats))                # a repeated string
    return text, pats


def check_random_tiny(lib, cases: int = 400, seed: int = 7):
    """Oracle scan == brute force == regex lookahead == classic AC on tiny cases."""
    rng = random.Random(seed)
    for _ in range(cases):
        text, pats = random_case(rng)
        want = brute.brute_longest(text, pats)
        assert brute.regex_longest(text, pats) == want, (text, pats)
        got = oracle.Trie(pats, lib).scan(text).tolist()
        assert got == want, (text, pats, got, want)
        ac = oracle.AhoCorasick(pats, lib)
        assert ac.longest(text).tolist() == want, (text, pats)
        e, i = ac.occurrences(text)
        assert sorted(zip(e.tolist(), i.tolist())) == brute.occurrences(text, pats), (text, pats)


def check_special_cases(lib):
    """Cases that reduce to textbook operations."""
    T = oracle.Trie
    # Empty text; text shorter than every pattern.
    assert T([b"ACG"], lib).scan(b"").tolist() == []
    assert T([b"ACGT", b"TTTT"], lib).scan(b"ACG").tolist() == [0, 0, 0]
    # A pattern equal to the whole text.
    assert T([b"GATTACA"], lib).scan(b"GATTACA").tolist() == [1, 0, 0, 0, 0, 0, 0]
    # Nested prefixes: the longest one that fits before the text end wins.
    assert T([b"A", b"AC", b"ACG", b"ACGT"], lib).scan(b"ACGTACG").tolist() == [4, 0, 0, 0, 3, 0, 0]
    # A repeated string keeps its lowest id.
    assert T([b"CAT", b"GG", b"CAT", b"GG"], lib).scan(b"CATGG").tolist() == [1, 0, 0, 2, 0]
    # Bytes outside ACGT end a walk (lowercase is not folded).
    assert T([b"AC", b"ACGT"], lib).scan(b"ACgTACGN").tolist() == [1, 0, 0, 0, 1, 0, 0, 0]
    # Patterns of length 1: the scan is a per-byte lookup.
    rng = np.random.default_rng(0)
    text = rng.choice(np.frombuffer(b"ACGTN", dtype=np.uint8), 500)
    got = T([b"G", b"T"], lib).scan(text)
    want = np.where(text == ord("G"), 1, np.where(text == ord("T"), 2, 0))
    assert np.array_equal(got, want)
    # One pattern: naive substring search.
    text = rng.choice(np.frombuffer(b"ACGT", dtype=np.uint8), 4000).tobytes()
    p = text[1234:1240]
    want = [0] * len(text)
    k = text.find(p)
    while k >= 0:
        want[k] = 1
        k = text.find(p, k + 1)
    assert T([p], lib).scan(text).tolist() == want
    # All patterns of one length k: k-mer set membership (lowest id of the k-mer).
    k = 5
    pats = [bytes(rng.choice(np.frombuffer(b"ACGT", dtype=np.uint8), k)) for _ in range(300)]
    first = {}
    for j, q in enumerate(pats):
        first.setdefault(q, j + 1)
    want = [first.get(text[i:i + k], 0) if i + k <= len(text) else 0 for i in range(len(text))]
    assert T(pats, lib).scan(text).tolist() == want


def check_invariants(lib, n_bases: int = 30000, n_pats: int = 300, seed: int = 11):
    """(i) a reported pattern occurs at its offset; (ii) no longer pattern occurs
    there; (iii) an offset reported 0 has no pattern occurring at it."""
    from paper_1811_10498_gb300 import datagen
    rng = datagen.rng_for(seed)
    text = datagen.iid_text(n_bases, rng)
    blob, offs = datagen.pattern_set(text, rng, n_pats, (3, 12), 0.5)
    pats = datagen.pattern_list(blob, offs)
    out = oracle.Trie((blob, offs), lib).scan(text)
    raw = text.tobytes()
    by_len = {}
    for q in pats:
        by_len.setdefault(len(q), set()).add(q)
    lens = sorted(by_len)
    for i in range(len(raw)):
        pid = int(out[i])
        if pid:
            q = pats[pid - 1]
            assert raw.startswith(q, i), i
            assert pats.index(q) + 1 == pid, i                  # lowest id of the string
            longer = [L for L in lens if L > len(q)]
        else:
            longer = lens
        for L in longer:
            assert raw[i:i + L] not in by_len[L], (i, L)


def check_fig1_all(lib):
    """Hand-worked all-match lists with the Fig. 1 patterns: every pattern occurrence,
    sub-patterns included, at its start offset."""
    rows = _golden("fig1_all.txt")
    pats = _patterns(rows)
    for r in rows:
        if r[0] != "all":
            continue
        want = [tuple(int(v) for v in pair.split(":")) for pair in r[2:]]
        s, i = oracle.all_matches(pats, r[1].encode(), lib=lib)
        assert list(zip(s.tolist(), i.tolist())) == want, (r[1], want)


def check_all_matches_random_tiny(lib, cases: int = 300, seed: int = 17):
    """The all-match list == brute force over every start and pattern; its longest
    entry per start == the PFAC scan."""
    rng = random.Random(seed)
    for _ in range(cases):
        text, pats = random_case(rng)
        s, i = oracle.all_matches(pats, text, lib=lib)
        got = list(zip(s.tolist(), i.tolist()))
        assert got == brute.brute_all(text, pats), (text, pats)
        longest = [0] * len(text)
        for start, pid in got:            # sorted by length within a start
            longest[start] = pid
        assert longest == brute.brute_longest(text, pats), (text, pats)


def check_pack_layout(lib=None):
    """Hand-packed words: base p of the text in bits 2(p mod 16)..2(p mod 16)+1 of word
    p / 16 with A=0, C=1, G=2, T=3, bases past the end 0; the first byte outside
    A/C/G/T is reported by its offset."""
    words, bad = oracle.pack(b"ACGT")
    assert bad == -1 and words.tolist() == [0b11100100]
    words, bad = oracle.pack(b"T" * 16 + b"C")
    assert words.tolist() == [0xFFFFFFFF, 1]
    words, bad = oracle.pack(b"A" * 15 + b"G")
    assert words.tolist() == [2 << 30]
    assert oracle.pack(b"ACGTnA")[1] == 4
    assert oracle.pack(b"NACGT")[1] == 0
    assert oracle.pack(b"")[0].shape == (0,)


def check_compact_definition(lib=None):
    """The match list holds exactly the offsets with a non-zero id, ascending."""
    offs, ids = oracle.compact(np.array([0, 3, 0, 0, 7, 1], dtype=np.int32))
    assert offs.tolist() == [1, 4, 5] and ids.tolist() == [3, 7, 1]
    offs, ids = oracle.compact(np.zeros(5, dtype=np.int32))
    assert offs.size == 0 and ids.size == 0


def check_reads_scan(lib=None):
    """Per-read scans: a walk ends at its read's end, and each read uses its own set's
    trie and ids. Worked by hand."""
    reads = np.frombuffer(b"ACGTACG", dtype=np.uint8)
    offs = np.array([0, 2, 7])
    # read 0 = "AC" with {ACG}: ACG does not fit in the read.
    # read 1 = "GTACG" with {ACG, AC}: ACG at its offset 2 (text offset 4).
    out = oracle.pfac_scan_reads(reads, offs, np.array([0, 1], dtype=np.int32), [[b"ACG"], [b"ACG", b"AC"]])
    assert out.tolist() == [0, 0, 0, 0, 1, 0, 0]
    # read 1 with {GT, ACG}: GT (id 1) at text offset 2, ACG (id 2) at 4.
    out = oracle.pfac_scan_reads(reads, offs, np.array([0, 1], dtype=np.int32), [[b"ACG"], [b"GT", b"ACG"]])
    assert out.tolist() == [0, 0, 1, 0, 2, 0, 0]


ALL_PINS = [check_fig1_numbering, check_table1, check_fig2_failure, check_fig1_scans,
            check_random_tiny, check_special_cases, check_invariants, check_fig1_all,
            check_all_matches_random_tiny, check_pack_layout, check_compact_definition,
            check_reads_scan]
