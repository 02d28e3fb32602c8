"""Host-side table construction of the CUDA library (host-only handles, no GPU):
the breadth-first tables encode exactly the oracle's insertion-order trie."""
import numpy as np
import pytest

import oracle
from paper_1811_10498_gb300 import _binding as b
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
    assert info["has_nodes"] == 1 and info["jump_k"] == 8
