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
    assert info["has_nodes"] == 1 and info["jump_k"] == 10 and info["filter_b"] == 10


def shortcut_reference(go, term, order_new, k, b):
    """Jump entries and filter bits defined by walking the oracle's insertion-order trie
    over every k-mer / b-mer (base j of a k-mer in bits 2j..2j+1)."""
    def walk(code, length):
        s, term_seen = 0, False
        for j in range(length):
            c = (code >> (2 * j)) & 3
            nxt = int(go[s, c])
            if nxt == 0:
                return None, term_seen
            s = nxt
            term_seen = term_seen or bool(term[s])
        return s, term_seen

    jump = []
    for code in range(1 << (2 * k)):
        s, t = walk(code, k)
        if t:
            jump.append(1)
        elif s is None:
            jump.append(0)
        else:
            jump.append(("state", int(order_new[s])))
    bits = []
    for code in range(1 << (2 * b)):
        s, t = walk(code, b)
        bits.append(1 if (t or s is not None) else 0)
    return jump, bits


@pytest.mark.parametrize("seed,k,b", [(1, 3, 4), (2, 4, 3), (3, 5, 5), (4, 2, 6), (5, 1, 1)])
def test_jump_and_filter_definition(seed, k, b):
    rng = datagen.rng_for(seed)
    text = datagen.iid_text(3000, rng)
    blob, offs = datagen.pattern_set(text, rng, 60, (1, 9), 0.6)
    go, term = oracle.Trie((blob, offs)).export()
    order = bfs_relabel(go)
    new = np.empty(go.shape[0], dtype=np.int64)
    new[np.array(order)] = np.arange(go.shape[0])
    h = b_.pfac_build((blob, offs), host_only=True, jump_k=k, filter_b=b)
    try:
        rows, out_id, level = b_.pfac_export(h)
        jump, filt = b_.pfac_export_shortcuts(h)
        info = b_.pfac_info_ex(h)
    finally:
        b_.pfac_destroy(h)
    kk = info["jump_k"]
    ref_jump, ref_bits = shortcut_reference(go, term, new, kk, b)
    for code, want in enumerate(ref_jump):
        v = int(jump[code])
        if isinstance(want, tuple):
            assert v >= 2 and level[kk] + v - 2 == want[1], (code, v, want)
        else:
            assert v == want, (code, v, want)
    got_bits = [(int(filt[w >> 5]) >> (w & 31)) & 1 for w in range(1 << (2 * b))]
    assert got_bits == ref_bits
