"""pfac_match_all: every pattern occurrence, sub-patterns included, against the oracle's
all-match list (the classic Aho-Corasick occurrences keyed by their start)."""
import random

import numpy as np
import pytest

import oracle
import pins
from gpu_util import require_cuda, to_dev
from paper_1811_10498_gb300 import _binding as b
from paper_1811_10498_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()


def gpu_all(table, text: np.ndarray, cap: int | None = None, **cfg):
    import torch
    if cfg:
        b.pfac_set_config(table.h, cfg)
    packed, status, _ = b.pack(to_dev(text))
    cap = cap if cap is not None else 4 * text.size + 16
    d_off = torch.full((max(1, cap),), -1, dtype=torch.int64, device="cuda")
    d_ids = torch.zeros(max(1, cap), dtype=torch.int32, device="cuda")
    d_cnt = torch.full((1,), 77, dtype=torch.int64, device="cuda")
    b.pfac_match_all(table.h, packed, text.size, d_off[:cap], d_ids[:cap], d_cnt)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    c = int(d_cnt.item())
    k = min(c, cap)
    return c, d_off[:k].cpu().numpy(), d_ids[:k].cpu().numpy()


def canonical(offs, ids, pattern_lengths):
    """Sort by start, then by pattern length (as oracle.all_matches lists them)."""
    order = np.lexsort((pattern_lengths[ids - 1], offs))
    return offs[order], ids[order]


@pytest.mark.parametrize("cfg", [dict(kernel=1), dict(kernel=2), dict(kernel=2, lane_offsets=16, walk_loads=1),
                                 dict(kernel=2, threads=64)], ids=lambda c: ",".join(f"{k}={v}" for k, v in c.items()))
def test_random_nested_sets(cfg):
    """Tiny random cases over ACGT with short, nested and repeated patterns, so that many
    walks pass several terminal states, some inside the filter's prefix."""
    rng = random.Random(23)
    for _ in range(40):
        text, pats = pins.random_case(rng, alphabet=b"ACGT", max_len=400, max_pats=12, max_plen=9)
        if not text:
            continue
        a = np.frombuffer(text, dtype=np.uint8)
        lens = np.array([len(p) for p in pats])
        ws, wi = oracle.all_matches(pats, a)
        for fb in (0, 2, 9, 12):     # 12: main filter in global memory behind a first level
            t = b.Table(pats, filter_b=fb)
            c, o, i = gpu_all(t, a, **cfg)
            assert c == ws.size, (text, pats, fb)
            o, i = canonical(o, i, lens)
            assert np.array_equal(o, ws) and np.array_equal(i, wi), (text, pats, fb)
            t.close()


def test_genome_text_all_matches():
    """Markov text with planted repeats and patterns cut from it: many nested hits along
    long walks that go through the deferred list."""
    w = datagen.genome_scan(n_bases=(2 << 20) + 99, n_patterns=3000)
    # add prefixes of some patterns, so that one walk meets several terminals
    pats = datagen.pattern_list(w.blob, w.offsets)
    pats += [p[:len(p) // 2] for p in pats[:500]] + [p[:12] for p in pats[500:800]]
    lens = np.array([len(p) for p in pats])
    ws, wi = oracle.all_matches(pats, w.text)
    longest = oracle.Trie(pats).scan(w.text)
    assert ws.size > np.count_nonzero(longest) > 1000     # sub-patterns add occurrences
    t = b.Table(pats)
    for cfg in (dict(kernel=2), dict(kernel=2, walk_loads=1, lane_offsets=16), dict(kernel=1)):
        c, o, i = gpu_all(t, w.text, **cfg)
        assert c == ws.size, cfg
        o, i = canonical(o, i, lens)
        assert np.array_equal(o, ws) and np.array_equal(i, wi), cfg
    t.close()


def test_overflow_reports_true_count():
    w = datagen.genome_scan(n_bases=1 << 20, n_patterns=2000)
    pats = datagen.pattern_list(w.blob, w.offsets)
    pats += [p[:10] for p in pats[:400]]
    ws, wi = oracle.all_matches(pats, w.text)
    t = b.Table(pats)
    cap = ws.size // 4
    c, o, i = gpu_all(t, w.text, cap=cap)
    assert c == ws.size
    assert o.size == cap
    have = set(zip(ws.tolist(), wi.tolist()))
    assert all((int(x), int(y)) in have for x, y in zip(o, i))   # each written pair is real
    assert len(set(zip(o.tolist(), i.tolist()))) == cap           # and written once
    assert b.pfac_device_status(t.h) == b.CODE["PFAC_ERR_OVERFLOW"]
    t.close()
