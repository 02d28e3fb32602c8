"""Chunked scans of host-resident texts with overlapped copies (hoststream.py)."""
import numpy as np
import pytest

import oracle
from gpu_util import first_diff, host_threads, require_cuda
from paper_1811_10498_gb300 import _binding as b
from paper_1811_10498_gb300 import datagen
from paper_1811_10498_gb300.hoststream import HostScanner, scan_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def genome():
    torch = require_cuda()
    w = datagen.genome_scan(n_bases=(5 << 20) + 4321, n_patterns=4000)
    t = b.Table((w.blob, w.offsets))
    want = oracle.Trie((w.blob, w.offsets)).scan_threads(w.text, host_threads())
    yield torch, w, t, want
    t.close()


@pytest.mark.parametrize("chunk", [1 << 16, (1 << 20) + 48, 1 << 26])
def test_chunks_equal_the_oracle(genome, chunk):
    """Walks that start near a chunk's end read into the next chunk's bases."""
    torch, w, t, want = genome
    h_text = torch.from_numpy(w.text).pin_memory()
    got = scan_host(t, h_text, chunk_bases=chunk).numpy()
    assert np.array_equal(got, want), first_diff(got, want)


@pytest.mark.parametrize("chunk", [1 << 16, (1 << 18) + 48, 1 << 22])
def test_match_list_equals_the_oracle(genome, chunk):
    """The match list of a host text (only the matches cross the host link): every offset
    with a pattern, ascending, with its id; a chunk's halo adds nothing twice."""
    torch, w, t, want = genome
    sc = HostScanner(t, chunk_bases=chunk)
    h_text = torch.from_numpy(w.text).pin_memory()
    offs_w, ids_w = oracle.compact(want)
    h_off = torch.full((offs_w.size + 10,), -1, dtype=torch.int64).pin_memory()
    h_ids = torch.zeros(offs_w.size + 10, dtype=torch.int32).pin_memory()
    c = sc.scan_matches(h_text, h_off, h_ids)
    assert c == offs_w.size
    assert np.array_equal(h_off.numpy()[:c], offs_w) and np.array_equal(h_ids.numpy()[:c], ids_w)
    # too small an output: an overflow error, not a truncated list
    small_off = torch.zeros(max(1, c // 2), dtype=torch.int64).pin_memory()
    small_ids = torch.zeros(max(1, c // 2), dtype=torch.int32).pin_memory()
    with pytest.raises(b.PfacError) as e:
        sc.scan_matches(h_text, small_off, small_ids)
    assert e.value.code == b.CODE["PFAC_ERR_OVERFLOW"]


def test_scanner_reuse_and_short_texts(genome):
    torch, w, t, want = genome
    sc = HostScanner(t, chunk_bases=1 << 18)
    for n in (w.text.size, 1, 99, (1 << 18) + 1):
        h_text = torch.from_numpy(np.ascontiguousarray(w.text[:n])).pin_memory()
        h_out = torch.full((n,), -3, dtype=torch.int32).pin_memory()
        sc.scan(h_text, h_out)
        assert sc.synchronize() == 0
        ref = oracle.Trie((w.blob, w.offsets)).scan(w.text[:n])
        assert np.array_equal(h_out.numpy(), ref), (n, first_diff(h_out.numpy(), ref))


def test_bad_symbol_is_reported(genome):
    torch, w, t, _ = genome
    text = w.text[:300_000].copy()
    text[250_000] = ord("N")
    with pytest.raises(b.PfacError):
        scan_host(t, torch.from_numpy(text), chunk_bases=1 << 16)


def test_ascii_chunks_with_newline_separated_reads():
    """The paper's input shape: lines of 100 bases, each ending in a newline, scanned as
    ASCII (a newline ends every walk)."""
    torch = require_cuda()
    src = datagen.paper_source(n_bases=1 << 16)     # lines overlap, so patterns recur
    text = datagen.paper_input(src, 20_000)
    blob, offs = datagen.paper_patterns(src, 1000)
    t = b.Table((blob, offs))
    want = oracle.Trie((blob, offs)).scan(text)
    got = scan_host(t, torch.from_numpy(text), chunk_bases=(1 << 18) + 16, ascii=True).numpy()
    assert np.array_equal(got, want), first_diff(got, want)
    assert (want != 0).sum() > 100
    t.close()


def test_files_to_ids(tmp_path):
    """The paper's host program end to end: patterns and newline-separated reads from
    files, the table built from the file, the text scanned from host memory."""
    torch = require_cuda()
    src = datagen.paper_source(n_bases=1 << 16)
    text = datagen.paper_input(src, 5000)
    blob, offs = datagen.paper_patterns(src, 300, length=40)
    pats = datagen.pattern_list(blob, offs)
    (tmp_path / "patterns.txt").write_bytes(b"\n".join(pats) + b"\n")
    (tmp_path / "reads.txt").write_bytes(text.tobytes())
    t = b.Table.from_file(str(tmp_path / "patterns.txt"))
    h_text = torch.from_numpy(b.read_text_file(str(tmp_path / "reads.txt")))
    got = scan_host(t, h_text, chunk_bases=1 << 17, ascii=True).numpy()
    want = oracle.Trie(pats).scan(text)
    assert np.array_equal(got, want), first_diff(got, want)
    assert (want != 0).sum() > 100
    t.close()
