"""Table construction on the GPU (pfac_build_device): for the same patterns, every table
equals the host builder's element for element (rows with terminal flags, ids, depth
levels, skip entries, prefix filter, dense entries, sampled screen, and the counts that
pfac_info_ex reports), and scans with the GPU-built table equal the oracle."""
import numpy as np
import pytest

import oracle
from gpu_util import first_diff, gpu_match_packed, host_threads, require_cuda, to_dev
from paper_1811_10498_gb300 import _binding as b
from paper_1811_10498_gb300 import datagen

pytestmark = pytest.mark.gpu

FIG1 = [b"AC", b"ACG", b"CTGT", b"TG"]
INFO_KEYS = ["n_states", "n_patterns", "max_len", "min_len", "filter_b", "n_duplicates", "table_bytes", "rows_bytes",
             "skip_bytes", "filter_set", "has_skip", "rank_wide", "sample_q", "sample_s"]


def device_inputs(pats):
    blob = np.frombuffer(b"".join(pats), dtype=np.uint8)
    offs = np.zeros(len(pats) + 1, dtype=np.int64)
    np.cumsum([len(p) for p in pats], out=offs[1:])
    return to_dev(blob if blob.size else np.zeros(1, dtype=np.uint8)), to_dev(offs)


def compare_builds(pats, **kw):
    require_cuda()
    host = b.Table(pats, **kw)
    d_blob, d_offs = device_inputs(pats)
    dev = b.Table.from_device(d_blob, d_offs, **kw)
    hi, di = host.info, dev.info
    assert {k: hi[k] for k in INFO_KEYS} == {k: di[k] for k in INFO_KEYS}
    for x, y in zip(b.pfac_export(host.h), b.pfac_export(dev.h)):
        assert np.array_equal(x, y)
    for x, y in zip(b.pfac_export_shortcuts(host.h), b.pfac_export_shortcuts(dev.h)):
        assert np.array_equal(x, y)
    qh, sh, gh = b.pfac_export_sample(host.h)
    qd, sd, gd = b.pfac_export_sample(dev.h)
    assert (qh, sh) == (qd, sd) and np.array_equal(gh, gd)
    host.close()
    return dev


@pytest.mark.parametrize("filter_b", [0, -1, 1, 3, 6])
def test_fig1_set(filter_b):
    dev = compare_builds(FIG1, filter_b=filter_b)
    text = np.frombuffer(b"ACGTGACTGTTGACG" * 5, dtype=np.uint8)
    got = gpu_match_packed(dev, text)
    assert np.array_equal(got, oracle.Trie(FIG1).scan(text))
    dev.close()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_sets_with_prefixes_and_duplicates(seed):
    rng = datagen.rng_for(seed)
    text = datagen.iid_text(5000, rng)
    blob, offs = datagen.pattern_set(text, rng, 300, (1, 40), 0.6)
    pats = datagen.pattern_list(blob, offs)
    pats += pats[:20] + [p[:3] for p in pats[20:40] if len(p) > 3]    # duplicates and prefixes
    for fb in (0, 4, 8):
        dev = compare_builds(pats, filter_b=fb)
        got = gpu_match_packed(dev, text)
        want = oracle.Trie(pats).scan(text)
        assert np.array_equal(got, want), first_diff(got, want)
        dev.close()


@pytest.mark.parametrize("sample", [0, 1])
def test_genome_scale_set(sample):
    """20,000 patterns of 20-100 bases (the genome-scale dictionary), order-10 filter,
    with and without the 10-gram screen."""
    w = datagen.genome_scan(n_bases=1 << 22, n_patterns=20_000)
    pats = datagen.pattern_list(w.blob, w.offsets)
    dev = compare_builds(pats, sample=sample)
    got = gpu_match_packed(dev, w.text)
    want = oracle.Trie(pats).scan_threads(w.text, host_threads())
    assert np.array_equal(got, want), first_diff(got, want)
    dev.close()


@pytest.mark.parametrize("filter_b,sample", [(14, 0), (12, 0), (11, -1)])
def test_large_set_with_deep_filters(filter_b, sample):
    """100,000 patterns of 16-64 bases: order 11-14 filters, first-level filter and the
    sampled screen built on the GPU as on the host."""
    rng = datagen.rng_for(51)
    text = datagen.iid_text((1 << 21) + 77, rng, datagen.GC41)
    blob, offs = datagen.pattern_set(text, rng, 100_000, (16, 64), 0.5, datagen.GC41)
    pats = datagen.pattern_list(blob, offs)
    dev = compare_builds(pats, filter_b=filter_b, sample=sample)
    assert dev.info["filter_b"] == filter_b
    got = gpu_match_packed(dev, text)
    want = oracle.Trie(pats).scan_threads(text, host_threads())
    assert np.array_equal(got, want), first_diff(got, want)
    dev.close()


def test_long_single_chains():
    """Patterns far longer than the 16-base skip cap, with ends at and around its
    multiples (skip entries cut at 16 bases, at terminals and at a branch)."""
    rng = datagen.rng_for(61)
    long = datagen.iid_text(200, rng).tobytes()
    other = b"A" if long[20:21] != b"A" else b"C"
    pats = [long] + [long[:k] for k in (15, 16, 17, 31, 32, 33, 48, 100)] + [long[:20] + other + long[21:80]]
    dev = compare_builds(pats, filter_b=5)
    dev.close()


@pytest.mark.parametrize("bad,code", [([b"ACGT", b""], "PFAC_ERR_EMPTY_PATTERN"),
                                      ([b"ACGT", b"ACNT"], "PFAC_ERR_BAD_SYMBOL"),
                                      ([b"ACGT", b"acgt"], "PFAC_ERR_BAD_SYMBOL")])
def test_errors(bad, code):
    require_cuda()
    d_blob, d_offs = device_inputs(bad)
    with pytest.raises(b.PfacError) as e:
        b.pfac_build_device(d_blob, d_offs)
    assert e.value.code == b.CODE[code]


def test_offsets_going_backwards_and_host_pointers():
    import torch
    require_cuda()
    d_blob = to_dev(np.frombuffer(b"ACGTACGT", dtype=np.uint8))
    with pytest.raises(b.PfacError) as e:
        b.pfac_build_device(d_blob, to_dev(np.array([0, 5, 3], dtype=np.int64)))
    assert e.value.code == b.CODE["PFAC_ERR_INVALID_ARG"]
    h_offs = torch.tensor([0, 4, 8], dtype=torch.int64)
    L = b.lib()
    assert L.pfac_build_device(d_blob.data_ptr(), h_offs.data_ptr(), 2, None, None) is None
    assert L.pfac_last_error() == b.CODE["PFAC_ERR_INVALID_ARG"]
