"""CUDA scan vs the CPU oracle, element by element (bit-exact: the output is integer)."""
import numpy as np
import pytest

import oracle
from gpu_util import first_diff, gpu_match, gpu_match_packed, host_threads, require_cuda, to_dev
from paper_1811_10498_gb300 import _binding as b
from paper_1811_10498_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()


def ref(text, patterns):
    return oracle.Trie(patterns).scan_threads(text, host_threads())


# ---- the small workload (1 M uniform bases, 1,000 patterns of 8-32) ----------

@pytest.fixture(scope="module")
def small():
    w = datagen.small_scan()
    return w, ref(w.text, (w.blob, w.offsets))


@pytest.mark.parametrize("kernel", [1, 2])
def test_small_ascii(small, kernel):
    w, want = small
    t = b.Table((w.blob, w.offsets))
    got = gpu_match(t, w.text, kernel=kernel)
    assert np.array_equal(got, want), first_diff(got, want)
    assert (want != 0).sum() > 400


@pytest.mark.parametrize("kernel", [1, 2])
def test_small_packed(small, kernel):
    w, want = small
    t = b.Table((w.blob, w.offsets))
    got = gpu_match_packed(t, w.text, kernel=kernel)
    assert np.array_equal(got, want), first_diff(got, want)


# ---- genome-like text, several tiles and a ragged tail ------------------------

@pytest.fixture(scope="module")
def genome_small():
    w = datagen.genome_scan(n_bases=(3 << 20) + 12345, n_patterns=20_000)
    return w, ref(w.text, (w.blob, w.offsets))


@pytest.mark.parametrize("packed", [True, False])
@pytest.mark.parametrize("cfg", [
    dict(kernel=1),
    dict(kernel=2),
    dict(kernel=2, threads=64),
    dict(kernel=2, threads=96, stages=2),
    dict(kernel=2, threads=512, stages=8),
    dict(kernel=2, threads=1024, stages=3),
    dict(kernel=2, rank_in_smem=-1),
    dict(kernel=2, l2_persist=1),
    dict(kernel=2, ctas_per_sm=2, threads=512),
    dict(kernel=2, walk_loads=1),
    dict(kernel=2, walk_loads=64),
    dict(kernel=2, lane_offsets=32),
    dict(kernel=2, lane_offsets=32, threads=64),
    dict(kernel=2, lane_offsets=16),
    dict(kernel=2, lane_offsets=16, stages=4),
    dict(kernel=2, lane_offsets=32, stages=3, threads=1024),
    dict(kernel=2, zero_writer=1),
    dict(kernel=2, zero_writer=2),
    dict(kernel=2, zero_writer=3),
    dict(kernel=2, zero_writer=2, threads=96, stages=2),
    dict(kernel=2, zero_writer=3, threads=96, stages=2),
    dict(kernel=2, zero_writer=3, rank_in_smem=-1),
    dict(kernel=2, zero_writer=3, walk_loads=1),
    dict(kernel=2, zero_writer=4),
    dict(kernel=2, zero_writer=4, threads=96, stages=2),
    dict(kernel=2, zero_writer=4, walk_loads=1, rank_in_smem=-1),
    dict(kernel=2, screen=1),
], ids=lambda c: ",".join(f"{k}={v}" for k, v in c.items()))
def test_genome_configs(genome_small, cfg, packed):
    w, want = genome_small
    t = b.Table((w.blob, w.offsets))
    got = (gpu_match_packed if packed else gpu_match)(t, w.text, **cfg)
    assert np.array_equal(got, want), first_diff(got, want)
    assert (want != 0).sum() > 1000


def test_deferred_list_overflow(genome_small, monkeypatch):
    """A deferred-walk list of 7 items: the walks that find it full finish inline."""
    import torch
    w, want = genome_small
    monkeypatch.setenv("PFAC_DEFER_CAP", "7")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        t = b.Table((w.blob, w.offsets))
        got = gpu_match_packed(t, w.text, kernel=2, walk_loads=1)
    assert np.array_equal(got, want), first_diff(got, want)


@pytest.mark.parametrize("cfg", [dict(screen=2), dict(screen=2, rank_in_smem=-1), dict(screen=2, walk_loads=1),
                                 dict(screen=2, zero_writer=2), dict(screen=0)],
                         ids=lambda c: ",".join(f"{k}={v}" for k, v in c.items()))
def test_shared_memory_10gram_screen(genome_small, cfg):
    """A table built with the 10-gram screen (sample = 1): scans with it in shared memory
    in the order-10 filter's place, and without it."""
    w, want = genome_small
    t = b.Table((w.blob, w.offsets), sample=1)
    assert (t.info["sample_q"], t.info["filter_b"]) == (10, 10)
    got = gpu_match_packed(t, w.text, kernel=2, **cfg)
    assert np.array_equal(got, want), first_diff(got, want)
    t.close()


@pytest.mark.parametrize("filter_b", [-1, 1, 3, 5, 8, 9, 10, 11, 12])
def test_filter_orders(genome_small, filter_b):
    """Prefix-filter orders, including filters too large for shared memory and a
    table without a filter (kernel 1)."""
    w, want = genome_small
    t = b.Table((w.blob, w.offsets), filter_b=filter_b)
    assert t.info["filter_b"] == max(filter_b, 0)
    got = gpu_match_packed(t, w.text)
    assert np.array_equal(got, want), first_diff(got, want)
    got = gpu_match(t, w.text)
    assert np.array_equal(got, want), first_diff(got, want)


# ---- adversarial small cases ---------------------------------------------------

FIG1 = [b"AC", b"ACG", b"CTGT", b"TG"]

CASES = [
    ("fig1", b"ACGCTGTGACNTGANCTGT", FIG1),
    ("len1", b"A", [b"A", b"C"]),
    ("len1_nomatch", b"G", [b"A", b"CA"]),
    ("shorter_than_all", b"ACG", [b"ACGT", b"TTTTT"]),
    ("whole_text", b"GATTACAGATTACA", [b"GATTACAGATTACA"]),
    ("nested", b"ACGTACGTACG", [b"A", b"AC", b"ACG", b"ACGT", b"ACGTACGTACGT"]),
    ("duplicates", b"CATGGCATGG", [b"CAT", b"GG", b"CAT", b"GG", b"CATGG"]),
    ("non_acgt", b"ACGTNACGT\nACgTacgtACGT-ACGT", [b"ACGT", b"AC", b"GTA"]),
    ("lmax1", b"ACGTTGCA" * 100, [b"G", b"T"]),
    ("single_pattern", b"TTAGGG" * 500 + b"TTAGG", [b"TTAGGGTTAGGG"]),
    ("end_of_text", b"CCCCCCACGTA", [b"ACGTA", b"CGTA", b"GTA", b"TA", b"A"]),
    ("all_N", b"N" * 1000, [b"A"]),
]


@pytest.mark.parametrize("name,text,pats", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("kernel", [1, 2])
def test_adversarial(name, text, pats, kernel):
    t = b.Table(pats)
    a = np.frombuffer(text, dtype=np.uint8)
    want = ref(a, pats)
    got = gpu_match(t, a, kernel=kernel, threads=64)
    assert np.array_equal(got, want), (name, first_diff(got, want))
    if all(c in b"ACGT" for c in text):
        got = gpu_match_packed(t, a, kernel=kernel, threads=64)
        assert np.array_equal(got, want), (name, first_diff(got, want))


def test_empty_text():
    t = b.Table(FIG1)
    assert gpu_match(t, np.zeros(0, dtype=np.uint8)).size == 0


@pytest.mark.parametrize("threads,lw,zw", [(64, 16, 0), (128, 32, 0), (1024, 16, 0), (1024, 32, 0), (96, 32, 2),
                                           (96, 32, 3), (1024, 32, 3), (64, 32, 4), (1024, 32, 4)])
def test_matches_across_tile_edges(threads, lw, zw):
    """Long patterns planted so they start just before, at and after tile edges (a tile
    is 32 x lw bases per consumer warp; a zero-writer warp takes one warp from the
    consumers) and end exactly at a tile edge, at a 32-base lane batch edge, at a 64-base
    window edge, and at the text end."""
    tile = 32 * lw * (threads // 32 - 1 - (zw in (2, 3)))
    rng = datagen.rng_for(99)
    n = tile * 6 + 37
    text = datagen.iid_text(n, rng)
    pats = []
    for edge in range(tile, n, tile):
        for start in (edge - 40, edge - 33, edge - 17, edge - 1, edge, edge + 1, edge + 31, edge + 33):
            L = 40 if start + 40 <= n else n - start
            if 0 <= start and L > 0:
                pats.append(text[start:start + L].tobytes())
        pats.append(text[edge - 25:edge].tobytes())          # ends exactly at the edge
        pats.append(text[edge + 2:edge + 64].tobytes())      # ends at the 64-base window edge
    pats.append(text[n - 30:].tobytes())                     # ends at the text end
    want = ref(text, pats)
    t = b.Table(pats)
    for kernel in (1, 2):
        got = gpu_match(t, text, kernel=kernel, threads=threads, lane_offsets=lw, zero_writer=zw)
        assert np.array_equal(got, want), (kernel, first_diff(got, want))
        got = gpu_match_packed(t, text, kernel=kernel, threads=threads, lane_offsets=lw, zero_writer=zw)
        assert np.array_equal(got, want), (kernel, first_diff(got, want))
    assert (want != 0).sum() >= len(pats) // 2


def test_random_small_sets_both_kernels():
    """Many tiny random cases (alphabet with N and newline, short patterns so that
    terminals fall inside the filter prefix)."""
    import random

    import pins
    rng = random.Random(5)
    for _ in range(60):
        text, pats = pins.random_case(rng, max_len=300, max_pats=12, max_plen=9)
        if not text:
            continue
        a = np.frombuffer(text, dtype=np.uint8)
        want = ref(a, pats)
        for fb in (0, 2, 9):
            t = b.Table(pats, filter_b=fb)
            for kernel in (1, 2):
                got = gpu_match(t, a, kernel=kernel, threads=64)
                assert np.array_equal(got, want), (text, pats, fb, kernel, first_diff(got, want))


def test_unaligned_buffers_fall_back():
    """A text that does not start on a 16-byte boundary still gives exact results."""
    import torch
    w = datagen.small_scan(n_bases=50_000, n_patterns=300)
    want = ref(w.text[3:], (w.blob, w.offsets))
    t = b.Table((w.blob, w.offsets))
    d = to_dev(w.text)
    out = torch.empty(w.text.size + 1, dtype=torch.int32, device="cuda")
    b.pfac_match(t.h, d[3:], out[1:])
    torch.cuda.synchronize()
    got = out[1:w.text.size - 2].cpu().numpy()
    assert np.array_equal(got, want), first_diff(got, want)


# ---- packing ---------------------------------------------------------------

@pytest.mark.parametrize("n", [0, 1, 15, 16, 17, 4096 + 5, 1_000_003])
def test_pack_matches_definition(n):
    import torch
    rng = datagen.rng_for(n + 1)
    text = datagen.iid_text(n, rng)
    words, bad = oracle.pack(text)
    d = to_dev(text) if n else torch.empty(0, dtype=torch.uint8, device="cuda")
    packed, status, first_bad = b.pack(d)
    torch.cuda.synchronize()
    got = packed.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, words)
    assert int(status.item()) == 0 and int(first_bad.item()) == -1


def test_pack_every_byte_value():
    """Every byte value at every position of a packed word: bases pack to their codes,
    other bytes pack as A and the first of them is reported."""
    import torch
    rng = np.random.default_rng(3)
    vals = np.arange(256, dtype=np.uint8)
    text = np.concatenate([np.roll(vals, k) for k in range(16)] + [rng.integers(0, 256, 4099, dtype=np.uint8)])
    words, first = oracle.pack(text)
    packed, status, first_bad = b.pack(to_dev(text))
    torch.cuda.synchronize()
    assert np.array_equal(packed.cpu().numpy().view(np.uint32), words)
    assert int(status.item()) == b.CODE["PFAC_ERR_BAD_SYMBOL"] and int(first_bad.item()) == first


def test_ascii_scan_with_every_byte_value():
    """ASCII texts mixing bases with every other byte value (lowercase, N, newline, high
    bytes): a walk stops at any non-base byte."""
    rng = np.random.default_rng(4)
    base = datagen.iid_text(200_000, datagen.rng_for(12))
    noise = rng.integers(0, 256, base.size, dtype=np.uint8)
    text = np.where(rng.random(base.size) < 0.03, noise, base).astype(np.uint8)
    pats = [base[i:i + L].tobytes() for i, L in zip(rng.integers(0, base.size - 40, 300), rng.integers(3, 30, 300))]
    want = ref(text, pats)
    t = b.Table(pats)
    for kernel in (1, 2):
        got = gpu_match(t, text, kernel=kernel)
        assert np.array_equal(got, want), (kernel, first_diff(got, want))
    assert (want != 0).sum() > 500


def test_pack_reports_first_bad_symbol():
    import torch
    text = np.frombuffer(b"ACGT" * 100 + b"ACGN" + b"ACGT" * 10 + b"x", dtype=np.uint8)
    packed, status, first_bad = b.pack(to_dev(text))
    torch.cuda.synchronize()
    assert int(status.item()) == b.CODE["PFAC_ERR_BAD_SYMBOL"]
    assert int(first_bad.item()) == 403
    words, _ = oracle.pack(text)
    assert np.array_equal(packed.cpu().numpy().view(np.uint32), words)


# ---- compaction ------------------------------------------------------------------

@pytest.mark.parametrize("kernel", [1, 2])
def test_compact_list(genome_small, kernel):
    import torch
    w, want = genome_small
    t = b.Table((w.blob, w.offsets))
    b.pfac_set_config(t.h, {"kernel": kernel})
    packed, _, _ = b.pack(to_dev(w.text))
    offs_want, ids_want = oracle.compact(want)
    cap = offs_want.size + 10
    d_off = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    d_ids = torch.zeros(cap, dtype=torch.int32, device="cuda")
    d_cnt = torch.full((1,), 123, dtype=torch.int64, device="cuda")
    b.pfac_match_compact(t.h, packed, w.text.size, d_off, d_ids, d_cnt)
    torch.cuda.synchronize()
    cnt = int(d_cnt.item())
    assert cnt == offs_want.size
    o = d_off[:cnt].cpu().numpy()
    i = d_ids[:cnt].cpu().numpy()
    order = np.argsort(o, kind="stable")
    assert np.array_equal(o[order], offs_want) and np.array_equal(i[order], ids_want)
    assert b.pfac_device_status(t.h) == b.CODE["PFAC_OK"]    # the list had room


@pytest.mark.parametrize("kernel", [1, 2])
def test_compact_overflow(genome_small, kernel):
    """A list with room for a third of the matches: the true count, every slot written
    once with a real match, and PFAC_ERR_OVERFLOW in the handle's device status."""
    import torch
    w, want = genome_small
    t = b.Table((w.blob, w.offsets))
    b.pfac_set_config(t.h, {"kernel": kernel})
    packed, _, _ = b.pack(to_dev(w.text))
    assert b.pfac_device_status(t.h) == b.CODE["PFAC_OK"]
    total = int((want != 0).sum())
    cap = total // 3
    d_off = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    d_ids = torch.zeros(cap, dtype=torch.int32, device="cuda")
    d_cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    b.pfac_match_compact(t.h, packed, w.text.size, d_off, d_ids, d_cnt)
    torch.cuda.synchronize()
    assert int(d_cnt.item()) == total            # the true count, beyond capacity
    o = d_off.cpu().numpy()
    i = d_ids.cpu().numpy()
    assert np.unique(o).size == cap               # every slot written once
    assert np.array_equal(want[o], i)             # each written pair is a real match
    assert b.pfac_device_status(t.h) == b.CODE["PFAC_ERR_OVERFLOW"]
    assert b.pfac_device_status(t.h) == b.CODE["PFAC_OK"]    # reading cleared it


# ---- failure handling ----------------------------------------------------------

def test_bounded_wait_times_out_and_context_survives():
    import time

    import torch
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    t0 = time.time()
    b.pfac_debug_timeout_probe(st, 20_000_000)        # 20 ms
    torch.cuda.synchronize()
    assert int(st.item()) == b.CODE["PFAC_ERR_TIMEOUT"]
    assert time.time() - t0 < 10
    # the context is still usable: a scan afterwards is exact
    w = datagen.small_scan(n_bases=20_000, n_patterns=100)
    t = b.Table((w.blob, w.offsets))
    assert np.array_equal(gpu_match(t, w.text), ref(w.text, (w.blob, w.offsets)))
    assert b.pfac_device_status(t.h) == 0


def test_host_pointers_rejected():
    import torch
    t = b.Table(FIG1)
    cpu = torch.zeros(16, dtype=torch.uint8)
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    rc = b.lib().pfac_match(t.h, cpu.data_ptr(), 16, out.data_ptr(), None)
    assert rc == b.CODE["PFAC_ERR_INVALID_ARG"]
    rc = b.lib().pfac_match(t.h, out.data_ptr(), 16, cpu.data_ptr(), None)
    assert rc == b.CODE["PFAC_ERR_INVALID_ARG"]


@pytest.mark.parametrize("cfg", [dict(kernel=2, lane_offsets=32, walk_loads=8), dict(kernel=2, walk_loads=64),
                                 dict(kernel=2, zero_writer=2, walk_loads=8), dict(kernel=2, zero_writer=3, walk_loads=8),
                                 dict(kernel=2, zero_writer=4, walk_loads=8)],
                         ids=["lw32_loads8", "lw16_loads64", "writer16B_loads8", "writerbulk_loads8", "warpbulk_loads8"])
def test_repeated_scans_with_long_walks_in_kernel(genome_small, cfg):
    """Matches found inside the scan kernel are stored by the lane that walks them,
    after the zero stores of the lane that owns the offset; repeated runs must agree
    with the oracle every time (this once showed lost and spurious matches when the
    two stores were not ordered)."""
    w, want = genome_small
    t = b.Table((w.blob, w.offsets))
    for _ in range(6):
        got = gpu_match_packed(t, w.text, **cfg)
        assert np.array_equal(got, want), first_diff(got, want)
