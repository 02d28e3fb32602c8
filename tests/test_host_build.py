"""Host-side table construction of the CUDA library (host-only handles, no GPU):
the breadth-first tables encode exactly the oracle's insertion-order trie."""
import numpy as np
import pytest

import oracle
from paper_1811_10498_gb300 import _binding as b
from paper_1811_10498_gb300 import _binding as b_
from paper_1811_10498_gb300 import datagen


def bfs_relabel(go):
    """Breadth-first order of an insertion-order trie, children in A, C, G, T order."""
    order = [0]
    head = 0
    while head < len(order):
        s = order[head]
        head += 1
        for c in range(4):
            if go[s, c]:
                order.append(int(go[s, c]))
    return order


def check_same_trie(patterns):
    go, term = oracle.Trie(patterns).export()
    h = b.pfac_build(patterns, host_only=True)
    try:
        rows, out_id, level = b.pfac_export(h)
        info = b.pfac_info_ex(h)
    finally:
        b.pfac_destroy(h)
    S = go.shape[0]
    assert info["n_states"] == S == rows.shape[0]
    order = bfs_relabel(go)
    new = np.empty(S, dtype=np.int64)
    new[np.array(order)] = np.arange(S)
    # same edges, same terminal flags, same ids
    for old in range(S):
        s = new[old]
        assert out_id[s] == term[old]
        for c in range(4):
            e = int(rows[s, c]) & 0xFFFFFFFF
            if go[old, c] == 0:
                assert e == 0
            else:
                child = int(go[old, c])
                assert (e & 0x7FFFFFFF) == new[child]
                assert bool(e >> 31) == bool(term[child])
    # depth levels are contiguous ranges
    depth = np.zeros(S, dtype=np.int64)
    for s in range(S):
        for c in range(4):
            e = int(rows[s, c]) & 0x7FFFFFFF
            if e:
                depth[e] = depth[s] + 1
    assert np.all(np.diff(depth) >= 0)
    for d in range(info["max_len"] + 1):
        assert np.all(depth[level[d]:level[d + 1]] == d)
    assert level[info["max_len"] + 1] == S
    return info


def test_fig1_example_breadth_first():
    info = check_same_trie([b"AC", b"ACG", b"CTGT", b"TG"])
    assert info["n_states"] == 10 and info["max_len"] == 4 and info["min_len"] == 2


def test_duplicates_and_prefixes():
    info = check_same_trie([b"CAT", b"CA", b"CAT", b"C", b"CATTAG", b"CA"])
    assert info["n_duplicates"] == 2


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_sets(seed):
    rng = datagen.rng_for(seed)
    text = datagen.iid_text(5000, rng)
    blob, offs = datagen.pattern_set(text, rng, 200, (1, 12), 0.5)
    check_same_trie((blob, offs))


def test_small_workload_set():
    w = datagen.small_scan(n_bases=100_000)
    info = check_same_trie((w.blob, w.offsets))
    assert info["has_skip"] == 1 and info["filter_b"] == 8


def reference_shortcuts(go, term, b):
    """Filter bits and the depth-b state of each b-mer (None for a clear bit, "special"
    when a pattern ends within it), by walking the oracle's insertion-order trie."""
    bits, state = [], []
    for code in range(1 << (2 * b)):
        s, seen = 0, False
        for j in range(b):
            nxt = int(go[s, (code >> (2 * j)) & 3])
            if nxt == 0:
                s = None
                break
            s = nxt
            seen = seen or bool(term[s])
        on = seen or s is not None
        bits.append(1 if on else 0)
        state.append(("special" if seen else s) if on else None)
    return bits, state


def check_skip_entry(e, s_old, go, term, new):
    """A skip entry of (breadth-first) state new[s_old] follows the single-child chain
    of the oracle's trie below s_old."""
    label, meta, last, node = (int(v) for v in e)
    L = meta & 31
    assert bool(meta & (1 << 8)) == bool(term[s_old])
    children = [c for c in range(4) if go[s_old, c]]
    mask = sum(1 << c for c in children)
    assert node & 15 == mask and bool(node & 16) == bool(term[s_old])
    if children:
        assert node >> 5 == new[int(go[s_old, children[0]])]
    cur = s_old
    for i in range(L):
        kids = [c for c in range(4) if go[cur, c]]
        assert len(kids) == 1, "a chain only follows single-child states"
        assert (label >> (2 * i)) & 3 == kids[0]
        cur = int(go[cur, kids[0]])
        if i < L - 1:
            assert not term[cur], "no terminal strictly inside a chain"
    if L:
        assert last == new[cur] and bool(meta & (1 << 10)) == bool(term[cur])
        stop = term[cur] or L == 16 or len([c for c in range(4) if go[cur, c]]) != 1
        assert stop, "a chain stops only at 16 bases, a terminal, or a branch or leaf"
    else:
        assert len(children) != 1


@pytest.mark.parametrize("seed,b", [(1, 4), (2, 3), (3, 5), (4, 6), (5, 1), (6, 2)])
def test_skip_filter_dense_definition(seed, b):
    rng = datagen.rng_for(seed)
    text = datagen.iid_text(3000, rng)
    blob, offs = datagen.pattern_set(text, rng, 60, (1, 30), 0.6)
    go, term = oracle.Trie((blob, offs)).export()
    order = bfs_relabel(go)
    new = np.empty(go.shape[0], dtype=np.int64)
    new[np.array(order)] = np.arange(go.shape[0])
    h = b_.pfac_build((blob, offs), host_only=True, filter_b=b)
    try:
        skip, filt, dense = b_.pfac_export_shortcuts(h)
        info = b_.pfac_info_ex(h)
    finally:
        b_.pfac_destroy(h)
    assert info["filter_b"] == b and skip.shape[0] == go.shape[0]
    for s_old in range(go.shape[0]):
        check_skip_entry(skip[new[s_old]], s_old, go, term, new)
    bits, state = reference_shortcuts(go, term, b)
    got = [(int(filt[w >> 5]) >> (w & 31)) & 1 for w in range(1 << (2 * b))]
    assert got == bits
    on = [st for st in state if st is not None]
    assert dense.shape[0] == len(on) == info["filter_set"]
    for r, st in enumerate(on):
        if st == "special":
            assert dense[r, 1] & (1 << 9)
        else:
            assert not dense[r, 1] & (1 << 9)
            assert np.array_equal(dense[r], skip[new[st]])


@pytest.mark.parametrize("seed,b", [(7, 4), (8, 6), (9, 7)])
def test_filter_when_no_pattern_ends_inside_a_bmer(seed, b):
    """Patterns no shorter than b (the builder's path without range fills): filter bits,
    dense entries in b-mer order and skip entries against their definitions."""
    rng = datagen.rng_for(seed)
    text = datagen.iid_text(4000, rng)
    blob, offs = datagen.pattern_set(text, rng, 120, (b, b + 20), 0.6)
    go, term = oracle.Trie((blob, offs)).export()
    order = bfs_relabel(go)
    new = np.empty(go.shape[0], dtype=np.int64)
    new[np.array(order)] = np.arange(go.shape[0])
    h = b_.pfac_build((blob, offs), host_only=True, filter_b=b)
    try:
        skip, filt, dense = b_.pfac_export_shortcuts(h)
        info = b_.pfac_info_ex(h)
    finally:
        b_.pfac_destroy(h)
    assert info["min_len"] >= b and info["filter_b"] == b
    bits, state = reference_shortcuts(go, term, b)
    got = [(int(filt[w >> 5]) >> (w & 31)) & 1 for w in range(1 << (2 * b))]
    assert got == bits
    on = [st for st in state if st is not None]
    assert dense.shape[0] == len(on) == info["filter_set"]
    for r, st in enumerate(on):
        if st == "special":                      # a pattern of exactly b bases ends there
            assert dense[r, 1] & (1 << 9)
        else:
            assert np.array_equal(dense[r], skip[new[st]])


def qgram_codes(pats, q, start):
    """Code of each pattern's q-gram at position `start` (base j in bits 2j..2j+1)."""
    lut = np.zeros(256, dtype=np.uint64)
    for i, ch in enumerate(b"ACGT"):
        lut[ch] = i
    codes = []
    for p in pats:
        a = lut[np.frombuffer(p[start:start + q], dtype=np.uint8)]
        codes.append(int((a << (2 * np.arange(q, dtype=np.uint64))).sum()))
    return codes


def set_bits(words):
    """Indices of the set bits of a little-endian bit array held in uint32 words."""
    nz = np.flatnonzero(words)
    out = [int(w) * 32 + j for w in nz for j in range(32) if (int(words[w]) >> j) & 1]
    return np.array(out, dtype=np.int64)


@pytest.mark.parametrize("seed", [11, 12])
def test_sampled_screen_definition(seed):
    """The sampled screen of a table whose filter lives in global memory and whose
    patterns have 16 bases or more: exactly the 13-grams at positions 0..3 of every
    pattern; of a table with an order-10 filter and patterns of 13 bases or more: the
    10-grams at positions 0..3. Tables with a shorter pattern, a filter of order 9 or
    less, or the option off have none."""
    rng = datagen.rng_for(seed)
    text = datagen.iid_text(20000, rng)
    blob, offs = datagen.pattern_set(text, rng, 400, (16, 40), 0.5)
    pats = datagen.pattern_list(blob, offs)
    h = b_.pfac_build(pats, host_only=True, filter_b=11)
    try:
        q, smp, g = b_.pfac_export_sample(h)
    finally:
        b_.pfac_destroy(h)
    assert (q, smp) == (13, 4) and g.size == (1 << 26) // 32
    want = sorted({c for d in range(smp) for c in qgram_codes(pats, q, d)})
    assert set_bits(g).tolist() == want
    # an order-10 filter (it fits in shared memory) gets a screen of 10-grams instead,
    # when asked for
    h = b_.pfac_build(pats, host_only=True, filter_b=10, sample=1)
    try:
        q, smp, g = b_.pfac_export_sample(h)
    finally:
        b_.pfac_destroy(h)
    assert (q, smp) == (10, 4) and g.size == (1 << 20) // 32
    want = sorted({c for d in range(smp) for c in qgram_codes(pats, q, d)})
    assert set_bits(g).tolist() == want
    short13 = [p for p in pats if len(p) >= 13] + [pats[0][:12]]
    for kw, ps in [(dict(filter_b=11), pats + [pats[0][:15]]), (dict(filter_b=10, sample=1), short13),
                   (dict(filter_b=10), pats), (dict(filter_b=9, sample=1), pats), (dict(filter_b=11, sample=-1), pats)]:
        h = b_.pfac_build(ps, host_only=True, **kw)
        try:
            assert b_.pfac_export_sample(h)[0] == 0, kw
        finally:
            b_.pfac_destroy(h)


def test_order_14_filter_of_long_patterns():
    """An order-14 filter (the automatic order for large sets without short patterns) of
    a set with patterns of 14-40 bases: its set bits are the codes of the patterns'
    14-base prefixes, and dense entry r is the skip entry of the state that the r-th of
    them (in code order) reaches, or the special entry when a 14-base pattern ends
    there."""
    rng = datagen.rng_for(21)
    text = datagen.iid_text(50000, rng)
    blob, offs = datagen.pattern_set(text, rng, 3000, (14, 40), 0.5)
    pats = datagen.pattern_list(blob, offs)
    h = b_.pfac_build(pats, host_only=True, filter_b=14)
    try:
        rows, out_id, _ = b_.pfac_export(h)
        skip, filt, dense = b_.pfac_export_shortcuts(h)
        info = b_.pfac_info_ex(h)
    finally:
        b_.pfac_destroy(h)
    assert info["filter_b"] == 14
    lut = {ch: i for i, ch in enumerate(b"ACGT")}
    by_code = {}
    for p in pats:
        s, code = 0, 0
        for j in range(14):
            c = lut[p[j]]
            code |= c << (2 * j)
            s = int(rows[s, c]) & 0x7FFFFFFF
        by_code[code] = s
    codes = sorted(by_code)
    assert set_bits(filt).tolist() == codes
    assert dense.shape[0] == len(codes) == info["filter_set"]
    assert any(len(p) == 14 for p in pats)
    for r, code in enumerate(codes):
        if out_id[by_code[code]]:
            assert dense[r, 1] & (1 << 9)
        else:
            assert np.array_equal(dense[r], skip[by_code[code]])


@pytest.mark.parametrize("cuts", [(15, 16, 17, 33), (16, 32, 48), (1, 17, 34, 40), (31, 32, 47), ()])
def test_skip_entries_at_the_chain_cap(cuts):
    """Single-child chains far longer than the 16-base cap, with pattern ends just
    before, at and after the cap's multiples and a branch deep inside the chain: every
    state's entry (cut at 16 bases, at a terminal or at the branch) follows its
    definition."""
    rng = datagen.rng_for(100 + sum(cuts))
    long = datagen.iid_text(70, rng).tobytes()
    other = b"A" if long[20:21] != b"A" else b"C"
    pats = [long] + [long[:k] for k in cuts] + [long[:20] + other + long[21:45]]
    go, term = oracle.Trie(pats).export()
    order = bfs_relabel(go)
    new = np.empty(go.shape[0], dtype=np.int64)
    new[np.array(order)] = np.arange(go.shape[0])
    h = b_.pfac_build(pats, host_only=True, filter_b=3)
    try:
        skip, _, _ = b_.pfac_export_shortcuts(h)
    finally:
        b_.pfac_destroy(h)
    assert skip.shape[0] == go.shape[0]
    lengths = set()
    for s_old in range(go.shape[0]):
        check_skip_entry(skip[new[s_old]], s_old, go, term, new)
        lengths.add(int(skip[new[s_old]][1]) & 31)
    assert 16 in lengths and 1 in lengths


def test_threaded_build_numbers_prefixes_by_length_then_lexicographically():
    """A set big enough for the builder to spread its sub-tries over several threads,
    checked against an independent definition of the breadth-first numbering: the
    distinct prefixes of the patterns (the empty one included) sorted by length and then
    lexicographically in A < C < G < T order. A row entry is the id of the prefix
    extended by that base, and a state's pattern id is the lowest 1-based index of a
    pattern equal to its prefix."""
    rng = datagen.rng_for(11)
    text = datagen.iid_text(1 << 20, rng)
    blob, offs = datagen.pattern_set(text, rng, 300_000, (1, 28), 0.7)
    lens = np.diff(offs)
    n = lens.size
    assert int(lens.sum()) >= 4 << 20          # four threads' worth of bases
    base = np.searchsorted(np.frombuffer(b"ACGT", dtype=np.uint8), blob).astype(np.uint64)
    # key of a prefix of d bases: d << 56 | its code, first base most significant
    # (lengths up to 28, so a code fits in 56 bits)
    sh = np.uint64(56)
    code = np.zeros(n, dtype=np.uint64)
    full = np.zeros(n, dtype=np.uint64)
    keys = [np.zeros(1, dtype=np.uint64)]
    for d in range(1, 29):
        live = lens >= d
        code[live] = code[live] * np.uint64(4) + base[offs[:-1][live] + d - 1]
        keys.append((np.uint64(d) << sh) | code[live])
        ends = lens == d
        full[ends] = (np.uint64(d) << sh) | code[ends]
    keys = np.unique(np.concatenate(keys))
    depth = (keys >> sh).astype(np.int64)
    kcode = keys & np.uint64((1 << 56) - 1)

    first = np.full(keys.size, n + 1, dtype=np.int64)
    np.minimum.at(first, np.searchsorted(keys, full), np.arange(1, n + 1))
    want_out = np.where(first == n + 1, 0, first)

    h = b.pfac_build((blob, offs), host_only=True, filter_b=-1)
    try:
        rows, out_id, level = b.pfac_export(h)
        info = b.pfac_info_ex(h)
    finally:
        b.pfac_destroy(h)
    assert info["n_states"] == keys.size
    assert info["n_duplicates"] == n - np.unique(full).size
    assert np.array_equal(out_id, want_out)
    assert np.array_equal(level, np.searchsorted(depth, np.arange(info["max_len"] + 2)))
    urows = rows.view(np.uint32)
    for c in range(4):
        inner = depth < 28
        child = ((depth[inner].astype(np.uint64) + np.uint64(1)) << sh) | (kcode[inner] * np.uint64(4) + np.uint64(c))
        pos = np.minimum(np.searchsorted(keys, child), keys.size - 1)
        exists = keys[pos] == child
        want = np.zeros(keys.size, dtype=np.uint32)
        want[inner] = np.where(exists, pos, 0).astype(np.uint32)
        want[inner] |= np.where(exists & (want_out[pos] != 0), np.uint32(1 << 31), np.uint32(0))
        assert np.array_equal(urows[:, c], want)
