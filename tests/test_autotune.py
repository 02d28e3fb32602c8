"""The launch autotuner: search and cache logic on the CPU, tuning on the GPU."""
import math

import numpy as np
import pytest

from paper_1811_10498_gb300 import autotune


def test_coordinate_search_finds_separable_optimum():
    knobs = [("a", (1, 2, 3)), ("b", (10, 20)), ("c", (0, 5, 7))]
    best_of = {"a": 3, "b": 20, "c": 5}
    calls = []

    def measure(cfg):
        calls.append(dict(cfg))
        return 1.0 + sum(0.1 * (cfg[k] != v) for k, v in best_of.items())

    best, t, hist = autotune.coordinate_search(measure, {"a": 1, "b": 10, "c": 0}, knobs)
    assert best == best_of
    assert t == pytest.approx(1.0)
    assert len(hist) == len(calls)
    assert hist[0][0] == {"a": 1, "b": 10, "c": 0}


def test_coordinate_search_skips_configs_that_cannot_run_and_keeps_ties():
    knobs = [("x", (1, 2, 3))]

    def measure(cfg):
        return {1: 2.0, 2: math.inf, 3: 1.995}[cfg["x"]]

    best, t, _ = autotune.coordinate_search(measure, {"x": 1}, knobs, rel_gain=0.01)
    assert best == {"x": 1} and t == 2.0          # 0.25 % faster is within the noise margin
    best, t, _ = autotune.coordinate_search(measure, {"x": 1}, knobs, rel_gain=0.0)
    assert best == {"x": 3}


def test_keys_bucket_sizes():
    dev = autotune.device_key({"name": "NVIDIA GB300", "multi_processor_count": 152, "L2_cache_size": 132644864})
    k1 = autotune.scan_key(dev, {"n_states": 1_072_991, "filter_b": 10}, 256 << 20, True)
    k2 = autotune.scan_key(dev, {"n_states": 1_100_000, "filter_b": 10}, (256 << 20) + 5, True)
    k3 = autotune.scan_key(dev, {"n_states": 1_072_991, "filter_b": 10}, 256 << 20, False)
    assert k1 == k2 and k1 != k3
    assert "sm152" in k1 and "n=2^28" in k1
    assert autotune.batch_key(dev, 64, 10_137_526, 4096) == autotune.batch_key(dev, 64, 10_000_000, 4096)


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "sub" / "tune.json")
    assert autotune.load_cache(p) == {}
    autotune.save_cache({"k1": {"config": {"threads": 512}}}, p)
    autotune.save_cache({"k2": {"config": {"stages": 3}}}, p)
    d = autotune.load_cache(p)
    assert d["k1"]["config"] == {"threads": 512} and d["k2"]["config"] == {"stages": 3}
    (tmp_path / "bad.json").write_text("not json")
    assert autotune.load_cache(str(tmp_path / "bad.json")) == {}


@pytest.mark.gpu
def test_tune_scan_is_exact_and_cached(tmp_path):
    from gpu_util import require_cuda, to_dev
    import oracle
    from paper_1811_10498_gb300 import _binding as b
    from paper_1811_10498_gb300 import datagen
    torch = require_cuda()
    w = datagen.genome_scan(n_bases=(4 << 20) + 333, n_patterns=5000)
    t = b.Table((w.blob, w.offsets))
    packed, status, _ = b.pack(to_dev(w.text))
    torch.cuda.synchronize()
    cache = str(tmp_path / "tune.json")
    logs = []
    cfg = autotune.tune_scan(t, packed, w.text.size, packed=True, reps=3, cache=cache, log=logs.append)
    assert not cfg["cached"] and cfg["candidates"] >= 8 and logs
    got = t.match_packed(packed, w.text.size)
    want = oracle.Trie((w.blob, w.offsets)).scan(w.text)
    assert np.array_equal(got.cpu().numpy(), want)
    # the second call reads the cache and measures nothing
    logs.clear()
    again = autotune.tune_scan(t, packed, w.text.size, packed=True, cache=cache, log=logs.append)
    assert again["cached"] and not logs
    assert {k: again[k] for k, _ in autotune.SCAN_KNOBS} == {k: cfg[k] for k, _ in autotune.SCAN_KNOBS}
    t.close()


@pytest.mark.gpu
def test_tune_batched_is_exact(tmp_path):
    from gpu_util import require_cuda
    import oracle
    from paper_1811_10498_gb300 import _binding as b
    from paper_1811_10498_gb300 import datagen
    torch = require_cuda()
    w = datagen.read_batch(seed=9, n_reads=300, n_sets=6, source_bases=1 << 20, median=800,
                           set_range=(50, 3000))
    tables = [b.Table(s) for s in w.sets]
    d_texts = torch.from_numpy(w.reads).cuda()
    d_offs = torch.from_numpy(w.read_offsets).cuda()
    d_set = torch.from_numpy(w.read_set).cuda()
    d_out = torch.empty(w.reads.size, dtype=torch.int32, device="cuda")
    cfg = autotune.tune_batched(tables, d_texts, d_offs, d_set, d_out, reps=3, cache=str(tmp_path / "t.json"))
    assert not cfg["cached"]
    d_out.fill_(-1)
    b.pfac_match_batched([t.h for t in tables], d_texts, d_offs, d_set, d_out)
    want = oracle.pfac_scan_reads(w.reads, w.read_offsets, w.read_set, w.sets)
    assert np.array_equal(d_out.cpu().numpy(), want)
    for t in tables:
        t.close()


@pytest.mark.gpu
def test_tune_scan_ascii_is_exact(tmp_path):
    """ASCII text with newline-separated lines (the paper's input shape)."""
    from gpu_util import require_cuda, to_dev
    import oracle
    from paper_1811_10498_gb300 import _binding as b
    from paper_1811_10498_gb300 import datagen
    torch = require_cuda()
    src = datagen.paper_source(n_bases=1 << 18)
    text = datagen.paper_input(src, 30_000)
    blob, offs = datagen.paper_patterns(src, 2000, length=30)
    t = b.Table((blob, offs))
    d = to_dev(text)
    cfg = autotune.tune_scan(t, d, text.size, packed=False, reps=3, cache=str(tmp_path / "a.json"))
    assert not cfg["cached"]
    got = t.match(d).cpu().numpy()
    assert np.array_equal(got, oracle.Trie((blob, offs)).scan(text))
    t.close()


def test_search_starts_from_the_default_of_the_launch_kind(cuda_lib_path):
    """The first candidate timed is the configuration the library uses when none is set:
    3 stages and 32 offsets per lane for packed text, 2 and 16 for ASCII text and for
    batched passes (a host-only handle is enough to read it)."""
    from paper_1811_10498_gb300 import _binding as b
    h = b.pfac_build([b"ACGT", b"GATTACA"], host_only=True)
    try:
        b.pfac_set_config(h, None)
        packed = autotune._start(h, 1 << 20, autotune.SCAN_KNOBS, packed=True)
        ascii_ = autotune._start(h, 1 << 20, autotune.SCAN_KNOBS, packed=False)
        batch = autotune._start(h, 0, autotune.BATCH_KNOBS, packed=False)
    finally:
        b.pfac_destroy(h)
    assert (packed["stages"], packed["lane_offsets"]) == (3, 32)
    assert (ascii_["stages"], ascii_["lane_offsets"]) == (2, 16)
    assert batch["lane_offsets"] == 16 and batch["threads"] == 1024 and batch["ctas_per_sm"] == 1
    assert packed["walk_loads"] == ascii_["walk_loads"] == batch["walk_loads"] == 2
