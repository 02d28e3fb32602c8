"""The chunk plan of the host-text scanner (host logic, no GPU): chunks scanned on
their own with a halo of max_len - 1 bases give the scan of the whole text."""
import numpy as np
import pytest

import oracle
from paper_1811_10498_gb300 import datagen
from paper_1811_10498_gb300.hoststream import chunk_spans


def scan_by_chunks(trie, text, spans):
    """Each chunk scanned as a text of its own (walks end at ext), own offsets kept."""
    out = np.zeros(text.size, dtype=np.int32)
    for lo, hi, ext in spans:
        out[lo:hi] = trie.scan(text[lo:ext])[:hi - lo]
    return out


@pytest.mark.parametrize("n,chunk,max_len", [(0, 16, 5), (1, 16, 1), (100, 16, 1), (100, 16, 30),
                                              (96, 16, 17), (1000, 1000, 64), (1001, 1000, 64)])
def test_spans_tile_the_text(n, chunk, max_len):
    spans = chunk_spans(n, chunk, max_len)
    assert [lo for lo, _, _ in spans] == list(range(0, n, chunk))
    assert all(hi - lo == chunk or hi == n for lo, hi, _ in spans)
    assert all(ext == min(n, hi + max_len - 1) for _, hi, ext in spans)
    assert sum(hi - lo for lo, hi, _ in spans) == n


def test_bad_arguments():
    with pytest.raises(ValueError):
        chunk_spans(10, 0, 4)
    with pytest.raises(ValueError):
        chunk_spans(10, 4, 0)


@pytest.mark.parametrize("seed,chunk", [(1, 16), (2, 64), (3, 100), (4, 1000)])
def test_chunked_scan_equals_the_whole_scan(seed, chunk):
    rng = datagen.rng_for(seed)
    text = datagen.iid_text(3000, rng)
    # patterns cut from the text, so matches straddle chunk edges
    blob, offs = datagen.pattern_set(text, rng, 300, (1, 40), 0.8)
    trie = oracle.Trie((blob, offs))
    max_len = int(np.diff(offs).max())
    want = trie.scan(text)
    assert np.count_nonzero(want) > 100
    got = scan_by_chunks(trie, text, chunk_spans(text.size, chunk, max_len))
    assert np.array_equal(got, want)


def test_a_shorter_halo_misses_the_longest_match_at_a_chunk_edge():
    """A pattern of max_len bases starting at the last offset of a chunk needs all
    max_len - 1 bases of the halo."""
    rng = datagen.rng_for(7)
    text = datagen.iid_text(64, rng)
    L, chunk = 12, 16
    pat = text[chunk - 1:chunk - 1 + L].tobytes()
    trie = oracle.Trie([pat, pat[:1]])
    want = trie.scan(text)
    assert want[chunk - 1] == 1
    assert np.array_equal(scan_by_chunks(trie, text, chunk_spans(text.size, chunk, L)), want)
    short = [(lo, hi, min(text.size, hi + L - 2)) for lo, hi, _ in chunk_spans(text.size, chunk, L)]
    assert scan_by_chunks(trie, text, short)[chunk - 1] != 1
