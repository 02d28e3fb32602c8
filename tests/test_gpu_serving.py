"""Serving loop: every request's result is the same in the mix as alone (and equal to
the CPU oracle), with latency and throughput reported."""
import numpy as np
import pytest

import oracle
from gpu_util import require_cuda
from paper_1811_10498_gb300 import _binding as b
from paper_1811_10498_gb300 import datagen
from paper_1811_10498_gb300.serving import Request, Server, requests_from_stream, serve_per_request

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def workload():
    require_cuda()
    st = datagen.request_stream(seed=5, rate=2000.0, duration=0.06, n_sets=4, set_range=(200, 3000),
                                pat_len=(16, 64), text_range=(1000, 200_000), source_bases=1 << 22)
    reqs = requests_from_stream(st)
    tables = [b.Table(s) for s in st.sets]
    want = {r.rid: oracle.Trie(st.sets[r.set_id]).scan(r.text) for r in reqs}
    return st, reqs, tables, want


@pytest.mark.parametrize("realtime", [True, False])
def test_results_in_the_mix_equal_the_oracle(workload, realtime):
    st, reqs, tables, want = workload
    srv = Server(tables, slot_bases=1 << 21, n_slots=3, max_reads=64, keep_results=True)
    lat, results, stats = srv.run(reqs, realtime=realtime)
    assert stats["requests"] == len(reqs) > 50
    for r in reqs:
        assert np.array_equal(results[r.rid], want[r.rid]), r.rid
    assert stats["p50_ms"] is not None and stats["p99_ms"] >= stats["p50_ms"] > 0
    if not realtime:
        # everything arrives at once: requests share batches
        assert stats["batches"] < len(reqs)
    assert sum(int(np.count_nonzero(want[r.rid])) for r in reqs) > 20


def test_each_request_alone_equals_its_result_in_the_mix(workload):
    st, reqs, tables, want = workload
    srv = Server(tables, slot_bases=1 << 21, n_slots=2, max_reads=64, keep_results=True)
    _, mixed, _ = srv.run(reqs, realtime=False)
    for r in reqs[:12]:
        _, alone, stats = srv.run([Request(r.rid, r.set_id, r.text, 0.0)], realtime=False)
        assert stats["batches"] == 1
        assert np.array_equal(alone[r.rid], mixed[r.rid]), r.rid


def test_admission_waits_for_device_memory(workload):
    """With a device-memory budget below two requests, batches hold one request and
    the others wait for memory to free up; results are unchanged."""
    st, reqs, tables, want = workload
    srv = Server(tables, slot_bases=1 << 21, n_slots=3, max_reads=64, keep_results=True)
    big = max(r.text.shape[0] for r in reqs[:10])
    srv.budget = 5 * big + 1
    _, results, stats = srv.run(reqs[:10], realtime=False)
    assert stats["batches"] >= 5
    for r in reqs[:10]:
        assert np.array_equal(results[r.rid], want[r.rid])


@pytest.mark.parametrize("realtime", [True, False])
def test_per_request_baseline_equals_the_oracle(workload, realtime):
    """The baseline the server is compared with (one request at a time, one pfac_match
    launch each) gives the same ids, and reports one launch per request."""
    st, reqs, tables, want = workload
    lat, results, stats = serve_per_request(tables, reqs, realtime=realtime, max_bases=1 << 21,
                                            keep_results=True)
    assert stats["requests"] == stats["launches"] == len(reqs)
    for r in reqs:
        assert np.array_equal(results[r.rid], want[r.rid]), r.rid
    assert lat.size == len(reqs) and stats["p99_ms"] >= stats["p50_ms"] > 0
