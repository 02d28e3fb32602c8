"""The serving loop's batching and admission policy (host logic, no GPU)."""
from collections import deque

import numpy as np
import pytest

from paper_1811_10498_gb300.serving import BYTES_PER_BASE, Request, take_batch


def reqs(lengths, start=0):
    return deque(Request(start + i, 0, np.full(n, ord("A"), dtype=np.uint8), float(i))
                 for i, n in enumerate(lengths))


def ids(batch):
    return [r.rid for r in batch]


def test_takes_in_arrival_order_up_to_the_read_limit():
    w = reqs([10] * 7)
    assert ids(take_batch(w, 0, 10**9, 1000, 3)) == [0, 1, 2]
    assert ids(take_batch(w, 0, 10**9, 1000, 3)) == [3, 4, 5]
    assert ids(take_batch(w, 0, 10**9, 1000, 3)) == [6]
    assert not w and take_batch(w, 0, 10**9, 1000, 3) == []


def test_slot_capacity_ends_the_batch_without_skipping_ahead():
    w = reqs([40, 50, 5, 5])
    # 40 + 50 > 64: the batch stops at the second request, even though the short
    # requests behind it would fit (no reordering of arrivals)
    assert ids(take_batch(w, 0, 10**9, 64, 100)) == [0]
    assert ids(take_batch(w, 0, 10**9, 64, 100)) == [1, 2, 3]


def test_device_memory_budget():
    w = reqs([100, 100, 100])
    budget = BYTES_PER_BASE * 250
    assert ids(take_batch(w, 0, budget, 10**6, 100)) == [0, 1]
    # 200 bases in flight: the third request waits until they complete
    assert take_batch(w, BYTES_PER_BASE * 200, budget, 10**6, 100) == []
    assert ids(take_batch(w, 0, budget, 10**6, 100)) == [2]


def test_a_request_above_the_budget_runs_alone_when_nothing_is_in_flight():
    w = reqs([500, 10])
    budget = BYTES_PER_BASE * 100
    assert take_batch(w, 1, budget, 10**6, 100) == []
    assert ids(take_batch(w, 0, budget, 10**6, 100)) == [0]
    assert ids(take_batch(w, 0, budget, 10**6, 100)) == [1]


def test_a_request_longer_than_a_slot_is_an_error():
    w = reqs([10, 2000])
    assert ids(take_batch(w, 0, 10**9, 1000, 100)) == [0]
    with pytest.raises(ValueError, match="exceeds the slot capacity"):
        take_batch(w, 0, 10**9, 1000, 100)
    assert ids(w) == [1]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_simulated_slots_serve_everything_once_within_the_budget(seed):
    """Three slots whose batches complete at random times: every request is served
    once, batches hold consecutive arrivals, and the bytes in flight stay within the
    budget except for a lone request admitted with nothing else in flight."""
    rng = np.random.default_rng(seed)
    lengths = rng.integers(1, 400, size=500)
    lengths[rng.integers(0, 500, size=5)] = 900      # above the budget, below a slot
    w = reqs(lengths.tolist())
    budget, slot_bases, max_reads = BYTES_PER_BASE * 800, 1000, 16
    slots = [None, None, None]
    in_flight, served = 0, []
    while w or any(slots):
        for k in range(len(slots)):
            if slots[k] is not None and rng.random() < 0.4:
                in_flight -= BYTES_PER_BASE * sum(r.text.size for r in slots[k])
                slots[k] = None
        for k in range(len(slots)):
            if slots[k] is None and w:
                before = in_flight
                batch = take_batch(w, in_flight, budget, slot_bases, max_reads)
                if not batch:
                    continue
                n = sum(r.text.size for r in batch)
                assert len(batch) <= max_reads and n <= slot_bases
                in_flight += BYTES_PER_BASE * n
                assert in_flight <= budget or (before == 0 and len(batch) == 1)
                slots[k] = batch
                served.extend(ids(batch))
    assert in_flight == 0
    assert served == list(range(500))
