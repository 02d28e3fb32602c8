"""The paper's memory-placement experiments (Section V-C; Section VII, Figs. 6-8) on the
one-thread-per-offset kernel: every combination of table layout (16-byte rows, the
paper's two arrays nextState / matchedPatternId, the two merged into pairs), table load
path (read-only/texture, default L1-cached, L1 bypassed) and text placement (global
memory, staged per block in shared memory) gives the oracle's ids, on the paper's
workload shape (newline-separated 100-base lines, 100-base patterns) and on a
genome-like text with patterns of 20-100 bases, ASCII and packed."""
import itertools

import numpy as np
import pytest

import oracle
from gpu_util import first_diff, gpu_match, gpu_match_packed, host_threads, require_cuda
from paper_1811_10498_gb300 import _binding as b
from paper_1811_10498_gb300 import datagen

pytestmark = pytest.mark.gpu

PLACEMENTS = [dict(table_layout=l, row_loads=ld, text_smem=ts)
              for l, ld, ts in itertools.product((0, 1, 2), (0, 1, 2), (0, 1))]


@pytest.fixture(scope="module")
def paper_shape():
    require_cuda()
    # a short source, so that many of the lines start where a pattern was copied from
    src = datagen.paper_source(n_bases=1 << 16)
    text = datagen.paper_input(src, 20_000)
    blob, offs = datagen.paper_patterns(src, 1000)
    want = oracle.Trie((blob, offs)).scan_threads(text, host_threads())
    assert (want != 0).sum() > 100
    return text, (blob, offs), want


@pytest.fixture(scope="module")
def genome():
    require_cuda()
    w = datagen.genome_scan(n_bases=(1 << 20) + 4321, n_patterns=5000)
    want = oracle.Trie((w.blob, w.offsets)).scan_threads(w.text, host_threads())
    assert (want != 0).sum() > 100
    return w.text, (w.blob, w.offsets), want


@pytest.mark.parametrize("cfg", PLACEMENTS, ids=lambda c: "layout{table_layout}-loads{row_loads}-smem{text_smem}".format(**c))
def test_paper_shape_placements(paper_shape, cfg):
    text, pats, want = paper_shape
    t = b.Table(pats)
    got = gpu_match(t, text, kernel=1, **cfg)
    assert np.array_equal(got, want), first_diff(got, want)
    t.close()


@pytest.mark.parametrize("packed", [False, True])
@pytest.mark.parametrize("cfg", PLACEMENTS, ids=lambda c: "layout{table_layout}-loads{row_loads}-smem{text_smem}".format(**c))
def test_genome_placements(genome, cfg, packed):
    text, pats, want = genome
    t = b.Table(pats)
    got = (gpu_match_packed if packed else gpu_match)(t, text, kernel=1, **cfg)
    assert np.array_equal(got, want), first_diff(got, want)
    t.close()


def test_layouts_describe_the_same_table():
    """The two-array and merged layouts hold, for every state and base, the state the
    edge leads to and the id of the pattern ending there, i.e. what the exported rows
    and ids say: checked through scans of every single-pattern walk of a small set
    (each pattern, scanned alone, must be found at offset 0 with every layout)."""
    pats = [b"ACGT", b"ACG", b"A", b"GATTACA", b"TTTT", b"ACGTACGT", b"CC"]
    t = b.Table(pats)
    want = oracle.Trie(pats)
    for cfg in PLACEMENTS:
        for p in pats:
            text = np.frombuffer(p + b"N" + p, dtype=np.uint8)
            got = gpu_match(t, text, kernel=1, **cfg)
            assert np.array_equal(got, want.scan(text)), (cfg, p)
    t.close()


def test_text_smem_falls_back_for_very_long_patterns():
    """A table whose per-block text tile would exceed 48 KB (a 60,000-base pattern)
    scans with the text in global memory instead, with the same ids."""
    rng = datagen.rng_for(11)
    text = datagen.iid_text(200_000, rng, datagen.GC41)
    pats = [text[1000:61000].tobytes(), text[5:40].tobytes(), b"ACGTACGTAC"]
    t = b.Table(pats)
    want = oracle.Trie(pats).scan(text)
    got = gpu_match(t, text, kernel=1, table_layout=2, text_smem=1)
    assert np.array_equal(got, want), first_diff(got, want)
    assert got[1000] == 1
    t.close()
