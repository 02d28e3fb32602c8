"""Full-size workloads, in the launch configuration the benchmark times, against the CPU
oracle (complete comparisons where the oracle is fast enough on the host's cores,
otherwise every match plus a sample of offsets computed one by one)."""
import numpy as np
import pytest

import oracle
from gpu_util import first_diff, host_threads, require_cuda, to_dev
from paper_1811_10498_gb300 import _binding as b
from paper_1811_10498_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()


def scan_packed(table, text):
    import torch
    d = to_dev(text)
    packed, status, _ = b.pack(d)
    out = torch.empty(text.size, dtype=torch.int32, device="cuda")
    b.pfac_match_packed(table.h, packed, text.size, out)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    del d
    return packed, out


def test_small_workload_full():
    """1,000,000 uniform bases, 1,000 patterns of 8-32, ASCII input."""
    w = datagen.small_scan()
    want = oracle.Trie((w.blob, w.offsets)).scan(w.text)
    t = b.Table((w.blob, w.offsets))
    got = t.match(to_dev(w.text)).cpu().numpy()
    assert np.array_equal(got, want), first_diff(got, want)


def test_genome_scale_full():
    """256 Mi bases, 20,000 patterns: the benchmark's workload, compared at every offset."""
    w = datagen.genome_scan()
    t = b.Table((w.blob, w.offsets))
    _, out = scan_packed(t, w.text)
    got = out.cpu().numpy()
    want = oracle.Trie((w.blob, w.offsets)).scan_threads(w.text, host_threads())
    assert np.array_equal(got, want), first_diff(got, want)
    assert (want != 0).sum() > 10_000


@pytest.mark.slow
def test_large_dictionary_full():
    """1 Gi bases, 1,000,000 patterns of 16-64: dense ids at every offset and the
    compacted match list."""
    import torch
    w = datagen.large_dict_scan()
    t = b.Table((w.blob, w.offsets))
    packed, out = scan_packed(t, w.text)
    got = out.cpu().numpy()
    del out
    want = oracle.Trie((w.blob, w.offsets)).scan_threads(w.text, host_threads())
    assert np.array_equal(got, want), first_diff(got, want)
    offs_w, ids_w = oracle.compact(want)
    cap = offs_w.size + 1024
    d_off = torch.empty(cap, dtype=torch.int64, device="cuda")
    d_ids = torch.empty(cap, dtype=torch.int32, device="cuda")
    d_cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    b.pfac_match_compact(t.h, packed, w.text.size, d_off, d_ids, d_cnt)
    torch.cuda.synchronize()
    c = int(d_cnt.item())
    assert c == offs_w.size
    o = d_off[:c].cpu().numpy()
    i = d_ids[:c].cpu().numpy()
    order = np.argsort(o)
    assert np.array_equal(o[order], offs_w) and np.array_equal(i[order], ids_w)


def test_batched_workload_full():
    """4,096 reads against 64 resident tables, as one batched pass."""
    import torch
    w = datagen.read_batch()
    want = oracle.pfac_scan_reads(w.reads, w.read_offsets, w.read_set, w.sets)
    tables = [b.Table(s) for s in w.sets]
    out = torch.full((w.reads.size,), -9, dtype=torch.int32, device="cuda")
    b.pfac_match_batched([t.h for t in tables], to_dev(w.reads), to_dev(w.read_offsets),
                         to_dev(w.read_set), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.array_equal(got, want), first_diff(got, want)


def test_serving_workload_full():
    """The full request stream (Poisson arrivals at 2,000 requests/s for 1 s, texts of
    1 kb-10 Mb against 16 resident tables) through the server in real time; every
    request's ids are compared with the oracle's scan of that request alone."""
    from paper_1811_10498_gb300.serving import Server, requests_from_stream
    st = datagen.request_stream(seed=5, duration=1.0)
    reqs = requests_from_stream(st)
    tables = [b.Table(s) for s in st.sets]

    srv = Server(tables, slot_bases=1 << 24, n_slots=3, max_reads=4096, keep_results=True)
    _, results, stats = srv.run(reqs, realtime=True)
    assert stats["requests"] == len(reqs) > 1500
    assert len(results) == len(reqs)
    by_set = {}
    for r in reqs:
        by_set.setdefault(r.set_id, []).append(r)
    threads = host_threads()
    checked = 0
    for set_id, rs in sorted(by_set.items()):
        trie = oracle.Trie(st.sets[set_id])
        for r in rs:
            want = trie.scan_threads(r.text, threads if r.text.size > (1 << 20) else 1)
            got = results.pop(r.rid)
            assert np.array_equal(got, want), (r.rid, first_diff(got, want))
            checked += 1
        del trie
    assert checked == len(reqs)
    for t in tables:
        t.close()


def test_text_beyond_two_gigabases():
    """2^31 + 4,099 bases: offsets past 2^31 (64-bit indexing all the way), with
    patterns planted on both sides of 2^31 and at the very end of the text."""
    import torch
    n = (1 << 31) + 4099
    rng = datagen.rng_for(77)
    text = datagen.iid_text(n, rng, datagen.GC41)
    pats = []
    for pos in ((1 << 31) - 40, (1 << 31) - 7, 1 << 31, (1 << 31) + 1, n - 64, n - 30):
        pats.append(text[pos:pos + 30].tobytes())
    blob, offs = datagen.pattern_set(text[:1 << 24], rng, 2000, (16, 40), 0.5, datagen.GC41)
    pats += datagen.pattern_list(blob, offs)
    t = b.Table(pats)
    packed, out = scan_packed(t, text)
    got = out.cpu().numpy()
    del out, packed
    torch.cuda.empty_cache()
    want = oracle.Trie(pats).scan_threads(text, host_threads())
    assert np.array_equal(got, want), first_diff(got, want)
    assert (want[1 << 31:] != 0).sum() >= 3
