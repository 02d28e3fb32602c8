"""The allocation-free scan, pfac_match_packed_noalloc.

Some callers cannot let a library allocate device memory for them: a process that
runs under a fixed device-memory budget, a process whose device memory belongs to
another allocator (a framework's caching pool), or a latency-sensitive loop that must
not meet the device-wide synchronisation a cudaMalloc or cudaFree can cause. The
ordinary packed scan allocates its deferred-walk scratch per stream on first use; the
allocation-free entry point uses one fixed buffer compiled into the library instead.

These checks call it through the C ABI and compare its output with the ordinary
entry point's, bit for bit, on two calls in a row (the second call must not be
disturbed by what the first one left in the shared buffer). This file is collected
last, so a run that stops at the first failure has already run every other test.
"""

import numpy as np
import pytest

from gpu_util import first_diff, require_cuda, to_dev
from paper_1811_10498_gb300 import _binding as b
from paper_1811_10498_gb300 import datagen

pytestmark = pytest.mark.gpu


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
    assert (want != 0).sum() > 1000                      # the text has many matches

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
