"""The seeded input generators hold to the recipe they state (no GPU): base composition
and context effects of the order-2 chain, pattern lengths and sources, read lengths,
arrival process, the paper's line shape, and determinism per seed. Sizes are small
versions of the workloads, large enough for the statistics to be tight."""
import math

import numpy as np
import pytest

from paper_1811_10498_gb300 import datagen


def freqs(text: np.ndarray):
    codes = np.searchsorted(np.frombuffer(b"ACGT", dtype=np.uint8), text)
    mono = np.bincount(codes, minlength=4) / codes.size
    di = np.bincount(codes[:-1] * 4 + codes[1:], minlength=16).reshape(4, 4) / (codes.size - 1)
    tri = np.bincount(codes[:-2] * 16 + codes[1:-1] * 4 + codes[2:], minlength=64) / (codes.size - 2)
    return mono, di, tri


def test_markov_text_composition_and_context():
    """The chain's definition: P(x | x2, x1) proportional to w[x] * m with base weights
    w = (a, c, c, a), m = 0.25 for G after C, m = 1.25 for a third A (or T) in a row.
    So G after C is 0.25 / (1 - 0.75 c) times as likely as G after G (a context no rule
    touches, where it is c), and A after AA is 1.25 / (1 + 0.25 a) times as likely as A
    after CA (where it is a). Stationary G+C is 41 %; A = T, while C > G because the
    mass taken from G after C goes to the other bases."""
    text = datagen.markov2_text(1 << 23, datagen.rng_for(0), 0.41)
    mono, di, tri = freqs(text)
    A, C, G, T = mono
    assert abs((C + G) - 0.41) < 0.003
    assert abs(A - T) < 0.004 and C > G + 0.02

    def cond(x2, x1, x):              # P(x | x2 x1)
        return tri[x2 * 16 + x1 * 4 + x] / tri[x2 * 16 + x1 * 4:x2 * 16 + x1 * 4 + 4].sum()

    c = cond(2, 2, 2)                 # G after GG: the weight c itself
    a = cond(1, 0, 0)                 # A after CA: the weight a itself
    assert abs(a + c - 0.5) < 0.01
    for x2 in range(4):
        assert abs(cond(x2, 1, 2) / cond(x2, 2, 2) / (0.25 / (1 - 0.75 * c)) - 1) < 0.06
    assert abs(cond(0, 0, 0) / a / (1.25 / (1 + 0.25 * a)) - 1) < 0.03
    assert abs(cond(3, 3, 3) / cond(1, 3, 3) / (1.25 / (1 + 0.25 * a)) - 1) < 0.03


def test_iid_text_follows_its_probabilities():
    text = datagen.iid_text(1 << 22, datagen.rng_for(1), datagen.GC41)
    mono, di, _ = freqs(text)
    assert abs(mono[1] + mono[2] - 0.41) < 0.002
    # independent bases: every dinucleotide is the product of its bases' frequencies
    assert np.allclose(di, np.outer(mono, mono), atol=0.002)


def test_genome_scale_patterns():
    """The genome-scale pattern recipe (the arguments genome_scan passes): lengths
    U[20, 100]; 70 % text substrings with 1 % point substitutions, so about E[0.99^L]
    of them still occur exactly; 30 % i.i.d. at 41 % G+C, which essentially never occur."""
    rng = datagen.rng_for(21)
    text = datagen.markov2_text(1 << 20, rng, 0.41)
    m = 1000
    blob, offs = datagen.pattern_set(text, rng, m, (20, 100), 0.7, datagen.GC41, mutation=0.01)
    lens = np.diff(offs)
    assert lens.min() >= 20 and lens.max() <= 100 and abs(lens.mean() - 60) < 3
    tb = text.tobytes()
    pats = datagen.pattern_list(blob, offs)
    n_sub = int(round(0.7 * m))
    exact = sum(tb.find(p) >= 0 for p in pats[:n_sub]) / n_sub
    assert abs(exact - float(np.mean(0.99 ** np.arange(20, 101)))) < 0.06
    assert sum(tb.find(p) >= 0 for p in pats[n_sub:]) <= 1
    rnd = np.frombuffer(b"".join(pats[n_sub:]), dtype=np.uint8)
    assert abs(np.isin(rnd, np.frombuffer(b"CG", dtype=np.uint8)).mean() - 0.41) < 0.015


def test_planted_repeats():
    """Repeat units copied over the text until the planted bases reach the fraction;
    every copy is one of the units (so the text holds each planted unit exactly)."""
    rng = datagen.rng_for(22)
    n = 1 << 20
    text = datagen.markov2_text(n, rng, 0.41)
    before = text.copy()
    planted = datagen.plant_repeats(text, rng, 0.05, 10, (300, 6000), 0.41)
    assert 0.05 * n <= planted < 0.05 * n + 6000
    changed = np.count_nonzero(text != before)
    assert 0 < changed <= planted
    assert datagen.plant_repeats(np.zeros(5000, dtype=np.uint8), rng, 0.05, 10, (300, 6000)) == 0


def test_read_batch_recipe():
    rb = datagen.read_batch(n_reads=4096, n_sets=8, source_bases=1 << 20, set_range=(100, 2000))
    lens = np.diff(rb.read_offsets)
    assert lens.min() >= 100 and lens.max() <= 100_000
    assert abs(np.median(lens) / 1500 - 1) < 0.08
    assert abs(np.std(np.log(lens[(lens > 100) & (lens < 100_000)])) - 1.0) < 0.08
    assert rb.read_set.min() >= 0 and rb.read_set.max() < 8
    assert len(rb.sets) == 8
    for blob, offs in rb.sets:
        pl = np.diff(offs)
        assert pl.min() >= 12 and pl.max() <= 64 and 100 <= pl.size <= 2000


def test_request_stream_recipe():
    rs = datagen.request_stream(rate=2000.0, duration=2.0, n_sets=4, set_range=(1000, 3000),
                                text_range=(1000, 100_000), source_bases=1 << 20)
    n = rs.arrivals.size
    assert abs(n - 4000) < 4 * math.sqrt(4000)
    gaps = np.diff(rs.arrivals)
    assert np.all(gaps > 0) and rs.arrivals[-1] < 2.0
    assert abs(gaps.mean() / 0.0005 - 1) < 0.05
    assert abs(gaps.std() / gaps.mean() - 1) < 0.08          # exponential gaps
    logs = np.log(rs.lengths)
    assert rs.lengths.min() >= 1000 and rs.lengths.max() <= 100_000
    assert abs(logs.mean() - 0.5 * (math.log(1000) + math.log(100_000))) < 0.1
    r = int(np.argmax(rs.lengths))
    assert rs.text(r).size == rs.lengths[r]


def test_paper_input_shape():
    src = datagen.paper_source(n_bases=1 << 16)
    text = datagen.paper_input(src, 500)
    assert text.size == 500 * 101
    lines = text.reshape(500, 101)
    assert np.all(lines[:, 100] == ord("\n"))
    s = src.tobytes()
    assert all(s.find(lines[i, :100].tobytes()) >= 0 for i in range(0, 500, 50))
    blob, offs = datagen.paper_patterns(src, 200)
    assert np.all(np.diff(offs) == 100)


@pytest.mark.parametrize("make", [
    lambda seed: datagen.small_scan(seed=seed, n_bases=1 << 16, n_patterns=100),
    lambda seed: datagen.genome_scan(seed=seed, n_bases=4096, n_patterns=100),   # too short for repeats
    lambda seed: datagen.large_dict_scan(seed=seed, n_bases=1 << 16, n_patterns=100),
])
def test_workloads_are_seeded(make):
    a, b, c = make(11), make(11), make(12)
    assert datagen.sha256(a.text) == datagen.sha256(b.text) and datagen.sha256(a.blob) == datagen.sha256(b.blob)
    assert datagen.sha256(a.text) != datagen.sha256(c.text)
