"""Batched scan (many reads, many resident tables) vs the CPU oracle, read by read."""
import numpy as np
import pytest

import oracle
from gpu_util import first_diff, require_cuda, to_dev
from paper_1811_10498_gb300 import _binding as b
from paper_1811_10498_gb300 import datagen
from paper_1811_10498_gb300.batched import BatchedScanner, scan_per_read

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()


@pytest.fixture(scope="module")
def batch():
    w = datagen.read_batch(seed=4, n_reads=300, n_sets=8, source_bases=1 << 22, median=1500.0,
                           set_range=(100, 5000), pat_len=(12, 64))
    want = oracle.pfac_scan_reads(w.reads, w.read_offsets, w.read_set, w.sets)
    tables = [b.Table(s) for s in w.sets]
    return w, want, tables


def run_batched(tables, reads, offs, read_set):
    import torch
    d_text = to_dev(reads) if len(reads) else torch.zeros(1, dtype=torch.uint8, device="cuda")
    out = torch.full((max(1, len(reads)),), -9, dtype=torch.int32, device="cuda")
    b.pfac_match_batched([t.h for t in tables], d_text[:len(reads)], to_dev(np.asarray(offs, dtype=np.int64)),
                         to_dev(np.asarray(read_set, dtype=np.int32)), out)
    torch.cuda.synchronize()
    return out[:len(reads)].cpu().numpy()


def test_batched_matches_oracle(batch):
    w, want, tables = batch
    got = run_batched(tables, w.reads, w.read_offsets, w.read_set)
    assert np.array_equal(got, want), first_diff(got, want)
    assert (want != 0).sum() > 50


def test_batched_with_deferred_walks(batch):
    """One dependent load per walk in the scan kernel: most walks that go on are
    finished by the batched tail kernel, with the table recorded in each item."""
    w, want, tables = batch
    b.pfac_set_config(tables[0].h, {"walk_loads": 1})
    try:
        got = run_batched(tables, w.reads, w.read_offsets, w.read_set)
    finally:
        b.pfac_set_config(tables[0].h, None)
    assert np.array_equal(got, want), first_diff(got, want)


def test_per_read_launches_match(batch):
    import torch
    w, want, tables = batch
    d = to_dev(w.reads)
    out = torch.full((w.reads.size,), -9, dtype=torch.int32, device="cuda")
    scan_per_read(tables, d, w.read_offsets, w.read_set, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.array_equal(got, want), first_diff(got, want)


def test_graph_replay_with_new_batches(batch):
    """One captured CUDA graph, replayed on different batches copied into its buffers."""
    w, want, tables = batch
    sc = BatchedScanner(tables, max_bases=w.reads.size, max_reads=len(w.read_set), graph=True)
    got = sc.scan(w.reads, w.read_offsets, w.read_set)
    assert np.array_equal(got, want), first_diff(got, want)
    # a second, different batch: the first 120 reads with their sets rotated
    k = 120
    offs = w.read_offsets[:k + 1]
    rs = (w.read_set[:k] + 3) % len(tables)
    reads = w.reads[:offs[-1]]
    want2 = oracle.pfac_scan_reads(reads, offs, rs, w.sets)
    got2 = sc.scan(reads, offs, rs)
    assert np.array_equal(got2, want2), first_diff(got2, want2)
    # and the first batch again
    got3 = sc.scan(w.reads, w.read_offsets, w.read_set)
    assert np.array_equal(got3, want), first_diff(got3, want)


def test_per_read_graph_baseline_equals_the_oracle(batch):
    """The baseline of the batched pass (one pfac_match per read, captured once in a CUDA
    graph and replayed twice) gives the oracle's ids."""
    import torch
    from paper_1811_10498_gb300.batched import PerReadGraph
    w, want, tables = batch
    d_text = to_dev(w.reads)
    out = torch.full((w.reads.size,), -3, dtype=torch.int32, device="cuda")
    pg = PerReadGraph(tables, d_text, w.read_offsets, w.read_set, out)
    out.fill_(-3)
    torch.cuda.synchronize()
    for _ in range(2):
        pg.run()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.array_equal(got, want), first_diff(got, want)
    assert pg.launches == 2 * int((np.diff(w.read_offsets) > 0).sum())


def test_reads_do_not_cross_into_each_other():
    sets = [[b"ACGT", b"GTAC", b"TT"], [b"CCCCAAAA", b"AT"]]
    tables = [b.Table(s) for s in sets]
    reads_list = [b"ACG", b"TACGT", b"", b"T", b"CCCC", b"AAAAT", b"ACGTN\nGTACTT", b"ACGT" * 300 + b"AC"]
    read_set = [0, 0, 1, 0, 1, 1, 0, 0]
    offs = np.zeros(len(reads_list) + 1, dtype=np.int64)
    np.cumsum([len(r) for r in reads_list], out=offs[1:])
    reads = np.frombuffer(b"".join(reads_list), dtype=np.uint8)
    want = oracle.pfac_scan_reads(reads, offs, np.array(read_set, dtype=np.int32), sets)
    got = run_batched(tables, reads, offs, read_set)
    assert np.array_equal(got, want), first_diff(got, want)
    # read 0 = "ACG" must not see the T that starts read 1
    assert got[0] == 0


def test_many_uneven_reads_and_item_edges():
    """Reads whose lengths straddle the 512-offset work items, with planted matches
    across item edges and at read ends."""
    rng = datagen.rng_for(21)
    lens = [511, 512, 513, 1, 1023, 1024, 1025, 7, 2048, 3, 600, 0, 5000]
    reads_list = [datagen.iid_text(L, rng) for L in lens]
    pats = []
    for r in reads_list:
        for start in (500, 507, 1020, len(r) - 20):
            if 0 <= start and start + 20 <= len(r):
                pats.append(r[start:start + 20].tobytes())
    pats.append(b"ACGTACGTACGT")
    sets = [pats, pats[::2] + [b"GATTACA"]]
    tables = [b.Table(s) for s in sets]
    offs = np.zeros(len(lens) + 1, dtype=np.int64)
    np.cumsum(lens, out=offs[1:])
    reads = np.concatenate(reads_list)
    read_set = np.array([i % 2 for i in range(len(lens))], dtype=np.int32)
    want = oracle.pfac_scan_reads(reads, offs, read_set, sets)
    got = run_batched(tables, reads, offs, read_set)
    assert np.array_equal(got, want), first_diff(got, want)
    assert (want != 0).sum() >= 10


def test_bad_table_index_is_reported():
    import torch
    tables = [b.Table([b"ACGT"])]
    reads = np.frombuffer(b"ACGTACGT", dtype=np.uint8)
    out = torch.full((8,), -9, dtype=torch.int32, device="cuda")
    b.pfac_match_batched([tables[0].h], to_dev(reads), to_dev(np.array([0, 4, 8], dtype=np.int64)),
                         to_dev(np.array([0, 5], dtype=np.int32)), out)
    torch.cuda.synchronize()
    assert out[:4].cpu().numpy().tolist() == [1, 0, 0, 0]
    assert b.pfac_device_status(tables[0].h) == b.CODE["PFAC_ERR_INVALID_ARG"]


def test_many_tables_and_filters_of_every_size():
    """300 tables with filters of orders 1-12 next to one another in one batch."""
    rng = np.random.default_rng(31)
    src = datagen.markov2_text(1 << 20, datagen.rng_for(31))
    sets, tables = [], []
    for k in range(300):
        size = int(rng.integers(1, 400))
        blob, offs = datagen.pattern_set(src, datagen.rng_for(100 + k), size, (4, 40), 0.7)
        sets.append((blob, offs))
        fb = 12 if k % 50 == 0 else (int(rng.integers(1, 10)) if k % 7 == 0 else 0)
        tables.append(b.Table((blob, offs), filter_b=fb))
    lens = rng.integers(0, 3000, 900)
    offs = np.zeros(lens.size + 1, dtype=np.int64)
    np.cumsum(lens, out=offs[1:])
    starts = rng.integers(0, src.size - 3000, lens.size)
    reads = np.concatenate([src[s0:s0 + L] for s0, L in zip(starts, lens)]).astype(np.uint8)
    read_set = rng.integers(0, len(sets), lens.size).astype(np.int32)
    want = oracle.pfac_scan_reads(reads, offs, read_set, sets)
    got = run_batched(tables, reads, offs, read_set)
    assert np.array_equal(got, want), first_diff(got, want)
    assert (want != 0).sum() > 1000
    for t in tables:
        t.close()


@pytest.mark.parametrize("cfg", [{"lane_offsets": 32}, {"threads": 256}, {"threads": 512, "walk_loads": 1}])
def test_launch_shapes(batch, cfg):
    """The one-launch pass with 1,024-base work items, and with 8 or 16 warps per CTA
    (each CTA plans the whole batch itself)."""
    w, want, tables = batch
    b.pfac_set_config(tables[0].h, cfg)
    try:
        got = run_batched(tables, w.reads, w.read_offsets, w.read_set)
    finally:
        b.pfac_set_config(tables[0].h, None)
    assert np.array_equal(got, want), first_diff(got, want)


def test_unaligned_text_and_output_pointers(batch):
    """Reads whose bytes start one byte past a 16-byte boundary and ids 4 bytes past
    one: the 16-byte copies and stores give way to narrower ones, with the same ids."""
    import torch
    w, want, tables = batch
    d = torch.zeros(w.reads.size + 1, dtype=torch.uint8, device="cuda")
    d[1:] = to_dev(w.reads)
    out = torch.full((w.reads.size + 1,), -9, dtype=torch.int32, device="cuda")
    b.pfac_match_batched([t.h for t in tables], d[1:], to_dev(w.read_offsets), to_dev(w.read_set), out[1:])
    torch.cuda.synchronize()
    got = out[1:].cpu().numpy()
    assert np.array_equal(got, want), first_diff(got, want)


def test_more_reads_than_one_launch_plans():
    """9,000 reads (more than one CTA plans in shared memory): the pass falls back to its
    pack, plan, scan and tail launches, with the oracle's ids."""
    rng = datagen.rng_for(77)
    src = datagen.iid_text(1 << 18, rng)
    pats = [src[s0:s0 + 20].tobytes() for s0 in rng.integers(0, src.size - 20, 200)]
    sets = [pats[:120], pats[80:], [b"ACGTACGTAC"]]
    tables = [b.Table(s) for s in sets]
    lens = rng.integers(0, 120, 9000)
    offs = np.zeros(lens.size + 1, dtype=np.int64)
    np.cumsum(lens, out=offs[1:])
    starts = rng.integers(0, src.size - 120, lens.size)
    reads = np.concatenate([src[s0:s0 + L] for s0, L in zip(starts, lens)]).astype(np.uint8)
    read_set = rng.integers(0, len(sets), lens.size).astype(np.int32)
    want = oracle.pfac_scan_reads(reads, offs, read_set, sets)
    got = run_batched(tables, reads, offs, read_set)
    assert np.array_equal(got, want), first_diff(got, want)
    assert (want != 0).sum() > 100
    for t in tables:
        t.close()


@pytest.mark.parametrize("lane_offsets", [16, 32])
def test_most_reads_one_launch_plans(lane_offsets):
    """8,192 reads, the most one launch plans in shared memory (its largest shared-memory
    layout), with empty and one-base reads among them: the oracle's ids."""
    rng = datagen.rng_for(91)
    src = datagen.iid_text(1 << 18, rng)
    pats = [src[s0:s0 + 16].tobytes() for s0 in rng.integers(0, src.size - 16, 300)]
    sets = [pats[:200], pats[100:], [b"ACGTACGTAC", b"TTTT"]]
    tables = [b.Table(s) for s in sets]
    lens = rng.integers(0, 200, 8192)
    lens[::97] = 0
    lens[5::101] = 1
    offs = np.zeros(lens.size + 1, dtype=np.int64)
    np.cumsum(lens, out=offs[1:])
    starts = rng.integers(0, src.size - 200, lens.size)
    reads = np.concatenate([src[s0:s0 + L] for s0, L in zip(starts, lens)]).astype(np.uint8)
    read_set = rng.integers(0, len(sets), lens.size).astype(np.int32)
    want = oracle.pfac_scan_reads(reads, offs, read_set, sets)
    b.pfac_set_config(tables[0].h, {"lane_offsets": lane_offsets})
    try:
        got = run_batched(tables, reads, offs, read_set)
    finally:
        b.pfac_set_config(tables[0].h, None)
    assert np.array_equal(got, want), first_diff(got, want)
    assert (want != 0).sum() > 100
    for t in tables:
        t.close()
