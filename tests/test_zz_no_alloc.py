"""The allocation-free scan, pfac_match_packed_noalloc.

Some callers cannot let a library allocate device memory for them: a process that
runs under a fixed device-memory budget, a process whose device memory belongs to
another allocator (a framework's caching pool), or a latency-sensitive loop that must
not meet the device-wide synchronisation a cudaMalloc or cudaFree can cause. The
ordinary packed scan allocates its deferred-walk scratch per stream on first use; the
allocation-free entry point uses one fixed buffer compiled into the library instead.

These checks call it through the C ABI and compare its output, bit for bit, with the
ordinary entry point's and with the oracle's, on two calls in a row (the second call
must not be disturbed by what the first one left in the shared buffer). One input is
built so that it defers more walks than the fixed buffer holds, so the walks that find
it full (finished inline) are exercised too. This file is collected last, so a run that
stops at the first failure has already run every other test.
"""

import numpy as np
import pytest

import oracle
from gpu_util import first_diff, host_threads, require_cuda, to_dev
from paper_1811_10498_gb300 import _binding as b
from paper_1811_10498_gb300 import datagen

pytestmark = pytest.mark.gpu

FIXED_ITEMS = 1 << 18          # deferred walks the library's fixed buffer holds
WINDOW = 64                    # bases a walk can take inside the scan kernel


@pytest.fixture(scope="module")
def setup():
    torch = require_cuda()
    w = datagen.genome_scan(n_bases=(3 << 20) + 777, n_patterns=20_000)
    t = b.Table((w.blob, w.offsets))
    # one dependent load per walk inside the scan kernel, so that many walks go
    # through the deferred list that this entry point keeps in its fixed buffer
    b.pfac_set_config(t.h, {"kernel": 2, "walk_loads": 1})
    packed, status, _ = b.pack(to_dev(w.text))
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return torch, w, t, packed


def test_matches_the_allocating_entry_point_twice(setup):
    torch, w, t, packed = setup
    n = w.text.size
    L = b.lib()
    stream = torch.cuda.current_stream().cuda_stream
    ref = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    assert L.pfac_match_packed(t.h, packed.data_ptr(), n, ref.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    want = ref.cpu().numpy()
    expect = oracle.Trie((w.blob, w.offsets)).scan_threads(w.text, host_threads())
    assert np.array_equal(want, expect), first_diff(want, expect)
    assert (want != 0).sum() > 1000                      # the text has many matches
    # A match longer than the kernel's 64-base window cannot finish in the kernel: its
    # walk goes through the deferred list, here the fixed buffer.
    lengths = np.diff(w.offsets)
    assert (lengths[expect[expect != 0] - 1] > WINDOW).sum() > 100

    outs = [torch.full((n,), -1, dtype=torch.int32, device="cuda") for _ in range(2)]
    free = []
    for out in outs:
        torch.cuda.synchronize()
        before = torch.cuda.mem_get_info()[0]
        rc = L.pfac_match_packed_noalloc(t.h, packed.data_ptr(), n, out.data_ptr(), stream)
        assert rc == 0, b.STATUS.get(rc, rc)
        torch.cuda.synchronize()
        free.append((before, torch.cuda.mem_get_info()[0]))
    for out in outs:
        got = out.cpu().numpy()
        assert np.array_equal(got, want), first_diff(got, want)
        assert np.array_equal(got, expect), first_diff(got, expect)
    assert b.pfac_device_status(t.h) == b.CODE["PFAC_OK"]
    # The first call on a device may load the library's module that holds the fixed
    # buffer; the second call must leave free device memory exactly as it was.
    assert free[1][0] == free[1][1]


def test_rejects_texts_beyond_the_fixed_buffer(setup):
    torch, w, t, packed = setup
    out = torch.empty(16, dtype=torch.int32, device="cuda")
    too_long = (1 << 26) + 1
    rc = b.lib().pfac_match_packed_noalloc(t.h, packed.data_ptr(), too_long, out.data_ptr(), None)
    assert rc == b.CODE["PFAC_ERR_SCRATCH_LIMIT"]
    assert b.lib().pfac_error_string(rc).decode().startswith("text longer than")


def test_more_deferred_walks_than_the_fixed_buffer_holds():
    """A periodic text (ACGT repeated) against a 100-base pattern of the same period:
    every fourth offset matches it, and each of those walks is longer than the kernel's
    window, so about n / 4 walks are deferred: four times what the fixed buffer holds.
    The walks that find it full finish inline; the output must still equal the oracle's
    and the ordinary entry point's, on two calls in a row."""
    torch = require_cuda()
    n = 1 << 22
    text = np.frombuffer(b"ACGT" * (n // 4), dtype=np.uint8)
    pats = [b"ACGT" * 25, b"ACGTACGTAC", b"GTAC" * 5 + b"A", b"CCCCCCCCCCCC"]
    t = b.Table(pats)
    b.pfac_set_config(t.h, {"kernel": 2, "walk_loads": 1})
    expect = oracle.Trie(pats).scan_threads(text, host_threads())
    long_hits = int((expect == 1).sum())
    assert long_hits > 4 * FIXED_ITEMS - 64              # deferred walks beyond capacity
    packed, status, _ = b.pack(to_dev(text))
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    L = b.lib()
    stream = torch.cuda.current_stream().cuda_stream
    ref = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    assert L.pfac_match_packed(t.h, packed.data_ptr(), n, ref.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    assert np.array_equal(ref.cpu().numpy(), expect), first_diff(ref.cpu().numpy(), expect)
    for _ in range(2):
        out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        rc = L.pfac_match_packed_noalloc(t.h, packed.data_ptr(), n, out.data_ptr(), stream)
        assert rc == 0, b.STATUS.get(rc, rc)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.array_equal(got, expect), first_diff(got, expect)
    assert b.pfac_device_status(t.h) == b.CODE["PFAC_OK"]
    t.close()
