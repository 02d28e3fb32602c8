"""The CPU oracle against what the paper and the mathematics fix (no GPU)."""
import numpy as np
import pytest

import oracle
import pins
from paper_1811_10498_gb300 import datagen


@pytest.mark.parametrize("check", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(check, oracle_lib):
    check(oracle_lib)


def test_build_errors(oracle_lib):
    with pytest.raises(oracle.OracleError) as e:
        oracle.Trie([b"ACG", b""], oracle_lib)
    assert e.value.code == 2
    with pytest.raises(oracle.OracleError) as e:
        oracle.Trie([b"ACG", b"ACN"], oracle_lib)
    assert e.value.code == 3
    with pytest.raises(oracle.OracleError) as e:
        oracle.Trie([], oracle_lib)
    assert e.value.code == 1


def test_classic_ac_equals_pfac_on_small_workload(oracle_lib):
    """Full 1 M-base small workload: the failure-link machine and the failure-less
    scan agree at every offset."""
    w = datagen.small_scan()
    pf = oracle.Trie((w.blob, w.offsets), oracle_lib).scan(w.text)
    ac = oracle.AhoCorasick((w.blob, w.offsets), oracle_lib).longest(w.text)
    assert np.array_equal(pf, ac)
    # half the patterns are text substrings, so every one of them must be found
    # at its source or be shadowed there by a longer pattern.
    assert (pf != 0).sum() >= 400


def test_classic_ac_equals_pfac_on_markov_text(oracle_lib):
    w = datagen.genome_scan(n_bases=1 << 21, n_patterns=2000)
    pf = oracle.Trie((w.blob, w.offsets), oracle_lib).scan(w.text)
    ac = oracle.AhoCorasick((w.blob, w.offsets), oracle_lib).longest(w.text)
    assert np.array_equal(pf, ac)
    assert (pf != 0).sum() > 100


def test_threaded_scan_equals_single(oracle_lib):
    w = datagen.small_scan(n_bases=200_000, n_patterns=300)
    t = oracle.Trie((w.blob, w.offsets), oracle_lib)
    assert np.array_equal(t.scan(w.text), t.scan_threads(w.text, 7))
