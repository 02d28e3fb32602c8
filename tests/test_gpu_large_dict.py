"""Large dictionaries: the order-14 prefix filter in global memory behind either screen
(the order-10 first-level filter in shared memory, or the sampled 13-gram screen probed
at every 4th offset), against the oracle at every offset: dense ids, the match list and
every occurrence, texts whose length is not a multiple of the lane width, and patterns
planted at the text's start and end."""
import numpy as np
import pytest

import oracle
from gpu_util import first_diff, gpu_match, gpu_match_packed, host_threads, require_cuda, to_dev
from paper_1811_10498_gb300 import _binding as b
from paper_1811_10498_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dictionary():
    require_cuda()
    rng = datagen.rng_for(31)
    n = (1 << 22) + 1234
    text = datagen.iid_text(n, rng, datagen.GC41)
    blob, offs = datagen.pattern_set(text, rng, 100_000, (16, 64), 0.5, datagen.GC41)
    pats = datagen.pattern_list(blob, offs)
    # matches at the very start and ending at the very end of the text
    pats += [text[:16].tobytes(), text[:40].tobytes(), text[n - 16:].tobytes(), text[n - 17:n - 1].tobytes(),
             text[n - 64:].tobytes()]
    want = oracle.Trie(pats).scan_threads(text, host_threads())
    assert want[0] != 0 and want[n - 16] != 0 and (want != 0).sum() > 1000
    return text, pats, want


@pytest.mark.parametrize("filter_b", [14, 12, 11])
@pytest.mark.parametrize("cfg", [dict(), dict(screen=1), dict(screen=2), dict(screen=2, zero_writer=2), dict(l2_persist=2),
                                 dict(screen=2, rank_in_smem=-1, walk_loads=1), dict(lane_offsets=16)],
                         ids=lambda c: ",".join(f"{k}={v}" for k, v in c.items()) or "auto")
def test_dense_ids(dictionary, filter_b, cfg):
    text, pats, want = dictionary
    t = b.Table(pats, filter_b=filter_b)
    info = t.info
    assert info["filter_b"] == filter_b and (info["sample_q"], info["sample_s"]) == (13, 4)
    got = gpu_match_packed(t, text, kernel=2, **cfg)
    assert np.array_equal(got, want), first_diff(got, want)
    assert b.pfac_device_status(t.h) == 0
    t.close()


def test_ascii_and_kernel_1(dictionary):
    """ASCII text (no sampled screen: the filter is read from global memory) and the
    one-thread-per-offset kernel over the same order-14 table."""
    text, pats, want = dictionary
    t = b.Table(pats, filter_b=14)
    got = gpu_match(t, text, kernel=2)
    assert np.array_equal(got, want), first_diff(got, want)
    got = gpu_match_packed(t, text, kernel=1)
    assert np.array_equal(got, want), first_diff(got, want)
    t.close()


def test_without_the_sampled_screen(dictionary):
    text, pats, want = dictionary
    t = b.Table(pats, filter_b=14, sample=-1)
    assert t.info["sample_q"] == 0
    got = gpu_match_packed(t, text, kernel=2, screen=2)     # falls back to the first-level filter
    assert np.array_equal(got, want), first_diff(got, want)
    t.close()


@pytest.mark.parametrize("screen", [1, 2])
def test_match_list_and_every_occurrence(dictionary, screen):
    import torch
    text, pats, want = dictionary
    t = b.Table(pats, filter_b=14)
    b.pfac_set_config(t.h, {"kernel": 2, "screen": screen})
    packed, _, _ = b.pack(to_dev(text))
    offs_w, ids_w = oracle.compact(want)
    cap = offs_w.size + 100
    d_off = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    d_ids = torch.zeros(cap, dtype=torch.int32, device="cuda")
    d_cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    b.pfac_match_compact(t.h, packed, text.size, d_off, d_ids, d_cnt)
    torch.cuda.synchronize()
    c = int(d_cnt.item())
    assert c == offs_w.size
    o, i = d_off[:c].cpu().numpy(), d_ids[:c].cpu().numpy()
    order = np.argsort(o)
    assert np.array_equal(o[order], offs_w) and np.array_equal(i[order], ids_w)
    # every occurrence (sub-patterns included)
    ws, wi = oracle.all_matches(pats, text[:1 << 20])
    cap = ws.size + 100
    d_off = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    d_ids = torch.zeros(cap, dtype=torch.int32, device="cuda")
    b.pfac_match_all(t.h, packed, 1 << 20, d_off, d_ids, d_cnt)
    torch.cuda.synchronize()
    c = int(d_cnt.item())
    assert c == ws.size
    got = sorted(zip(d_off[:c].cpu().numpy().tolist(), d_ids[:c].cpu().numpy().tolist()))
    assert got == sorted(zip(ws.tolist(), wi.tolist()))
    assert b.pfac_device_status(t.h) == 0
    t.close()


@pytest.mark.parametrize("n", [1, 15, 16, 17, 31, 33, 100, 1000, 4097])
def test_short_texts(dictionary, n):
    """Texts shorter than a lane's window or a tile: every probe past the end reads
    bases that are not the text's, and no offset may be lost or invented."""
    _, pats, _ = dictionary
    rng = datagen.rng_for(40 + n)
    base = datagen.iid_text(n, rng, datagen.GC41)
    extra = [base.tobytes()] if n >= 16 else []
    t = b.Table(pats + extra, filter_b=14)
    want = oracle.Trie(pats + extra).scan(base)
    got = gpu_match_packed(t, base, kernel=2, screen=2)
    assert np.array_equal(got, want), first_diff(got, want)
    t.close()
