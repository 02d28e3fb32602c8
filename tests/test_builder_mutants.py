"""Plant plausible mistakes in copies of the library's table builder
(csrc/trie_build.cpp) and check that the host-build tests catch every one of them
(CPU only). Each copy is compiled with the host compiler, with no CUDA, into a small
library around the builder alone (tests/native/builder_shim.cpp); the checks of
tests/test_host_build.py then run against it in place of the CUDA library's binding.
The unchanged builder, compiled the same way, must pass every check."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import test_host_build as thb
from paper_1811_10498_gb300 import _binding

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1811_10498_gb300", "csrc")
SRC = os.path.join(CSRC, "trie_build.cpp")

MUTANTS = {
    # Duplicates: the lowest id is kept (patterns of three bases or more).
    "last_duplicate_wins": (
        "        if (term[(size_t)s] == 0) term[(size_t)s] = j + 1;\n        else B.dups++;",
        "        term[(size_t)s] = j + 1;"),
    # The same for patterns shorter than the sub-trie prefix.
    "last_short_duplicate_wins": (
        "            else if (top_term[(size_t)lengths[j]][code] == 0) top_term[(size_t)lengths[j]][code] = j + 1;\n"
        "            else dups++;",
        "            else top_term[(size_t)lengths[j]][code] = j + 1;"),
    # Sub-tries take their id ranges in prefix order, not in the order they were built.
    "subtries_in_work_order": (
        "            for (int t = 0; t < kSubTries; t++) {\n                SubTrie &B = sub[(size_t)t];",
        "            for (int t : used) {\n                SubTrie &B = sub[(size_t)t];"),
    # Breadth-first order visits children in A, C, G, T order.
    "children_in_reverse_order": (
        "        for (int c = 0; c < 4; c++) {\n            const int32_t ch = g[c];",
        "        for (int c = 3; c >= 0; c--) {\n            const int32_t ch = g[c];"),
    # The edge into a sub-trie's first state carries its terminal flag.
    "subtrie_root_edge_not_terminal": (
        "e = (uint32_t)sub[cc].base[0] | (sub[cc].out[0] ? 0x80000000u : 0u);",
        "e = (uint32_t)sub[cc].base[0];"),
    # A skip chain holds at most 16 bases.
    "skip_cap_off_by_one": (
        "if (child_len < (uint32_t)kSkipMaxLen) {",
        "if (child_len <= (uint32_t)kSkipMaxLen) {"),
    # A chain cut at 16 bases stops at the parent of the child's target.
    "capped_chain_keeps_child_target": (
        "target = (uint32_t)parent[(size_t)ce[2]];",
        "target = ce[2];"),
    # A prefix whose walk stops at symbol d fixes every b-mer congruent to it mod 4^(d+1).
    # (A shorter stride would be an equivalent mutant: the extra b-mers it fills pass
    # through a state below which a pattern has already ended, so they are special anyway.)
    "filter_fill_stride_too_long": (
        "const size_t stride = (size_t)1 << (2 * (d + 1));",
        "const size_t stride = (size_t)1 << (2 * (d + 2));"),
    # "A pattern ends on the path" is inherited from the parent.
    "filter_pattern_end_not_inherited": (
        "seen[child] = (uint8_t)(seen[(size_t)s] | (e >> 31));",
        "seen[child] = (uint8_t)(e >> 31);"),
    # Without short patterns: dense entries follow the b-mer codes, not the state ids.
    "deep_filter_dense_in_state_order": (
        "            std::sort(at_b.begin(), at_b.end());\n",
        ""),
    # Without short patterns: a state's code holds its first base in the low bits.
    "deep_filter_code_reversed": (
        "code[(size_t)st] | ((uint64_t)c << (32 + 2 * d));",
        "code[(size_t)st] | ((uint64_t)c << (32 + 2 * (b - 1 - d)));"),
    # The sampled screen holds the q-grams at every position 0 .. s-1.
    "sample_misses_last_position": (
        "for (int d = 0; d < kSampleS; d++) {",
        "for (int d = 0; d < kSampleS - 1; d++) {"),
    # ... with the first base of a q-gram in its low bits.
    "sample_qgram_reversed": (
        "g |= (uint32_t)base_code(p[d + k]) << (2 * k);",
        "g |= (uint32_t)base_code(p[d + k]) << (2 * (q - 1 - k));"),
}


class BuilderOnly:
    """The calls of the CUDA library's binding that the host-build checks use, served by
    a host-compiled builder."""

    def __init__(self, so: str):
        L = C.CDLL(so)
        P, I32 = C.c_void_p, C.c_int32
        L.shim_build.restype = P
        L.shim_build.argtypes = [P, P, I32, I32, I32, P]
        L.shim_destroy.argtypes = [P]
        L.shim_info.argtypes = [P, P]
        L.shim_export.argtypes = [P, P, P, P]
        L.shim_export_shortcuts.argtypes = [P, P, P, P]
        L.shim_export_sample.argtypes = [P, P, P]
        self.L = L

    def pfac_build(self, patterns, host_only=True, filter_b=0, sample=0):
        blob, ptrs, lengths, n = _binding._patterns(patterns)
        st = C.c_int32(0)
        h = self.L.shim_build(ptrs.ctypes.data, lengths.ctypes.data, n, filter_b, sample, C.byref(st))
        if not h:
            raise _binding.PfacError(st.value, "build")
        self._keep = blob
        return h

    def pfac_destroy(self, h):
        self.L.shim_destroy(h)

    def pfac_info_ex(self, h):
        v = np.zeros(8, dtype=np.int64)
        self.L.shim_info(h, v.ctypes.data)
        keys = ["n_states", "n_patterns", "max_len", "min_len", "n_duplicates", "filter_b", "filter_set", "has_skip"]
        return {k: int(x) for k, x in zip(keys, v)}

    def pfac_export(self, h):
        i = self.pfac_info_ex(h)
        rows = np.zeros((i["n_states"], 4), dtype=np.int32)
        out_id = np.zeros(i["n_states"], dtype=np.int32)
        level = np.zeros(i["max_len"] + 2, dtype=np.int64)
        self.L.shim_export(h, rows.ctypes.data, out_id.ctypes.data, level.ctypes.data)
        return rows, out_id, level

    def pfac_export_sample(self, h):
        qs = np.zeros(2, dtype=np.int32)
        self.L.shim_export_sample(h, qs.ctypes.data, None)
        q, smp = int(qs[0]), int(qs[1])
        g = np.zeros(((1 << (2 * q)) // 32) if q else 1, dtype=np.uint32)
        self.L.shim_export_sample(h, qs.ctypes.data, g.ctypes.data)
        return q, smp, (g if q else g[:0])

    def pfac_export_shortcuts(self, h):
        i = self.pfac_info_ex(h)
        S, b, F = i["n_states"], i["filter_b"], i["filter_set"]
        skip = np.zeros((S if i["has_skip"] else 0, 4), dtype=np.uint32)
        filt = np.zeros(max(1, (1 << (2 * b)) // 32) if b else 0, dtype=np.uint32)
        dense = np.zeros((F, 4), dtype=np.uint32)
        self.L.shim_export_shortcuts(h, skip.ctypes.data, filt.ctypes.data, dense.ctypes.data)
        return skip, filt, dense


# The host-build checks, fastest first; a mutant needs to fail only one of them.
CHECKS = [
    ("fig1", lambda: thb.test_fig1_example_breadth_first()),
    ("duplicates", lambda: thb.test_duplicates_and_prefixes()),
    *[(f"random_{s}", (lambda s=s: thb.test_random_sets(s))) for s in (1, 2, 3)],
    *[(f"shortcuts_{s}_{b}", (lambda s=s, b=b: thb.test_skip_filter_dense_definition(s, b)))
      for s, b in [(1, 4), (2, 3), (3, 5), (4, 6), (5, 1), (6, 2)]],
    *[(f"chain_cap_{i}", (lambda c=c: thb.test_skip_entries_at_the_chain_cap(c)))
      for i, c in enumerate([(15, 16, 17, 33), (16, 32, 48), (1, 17, 34, 40), (31, 32, 47), ()])],
    ("threaded_numbering", lambda: thb.test_threaded_build_numbers_prefixes_by_length_then_lexicographically()),
    *[(f"long_patterns_{s}_{b}", (lambda s=s, b=b: thb.test_filter_when_no_pattern_ends_inside_a_bmer(s, b)))
      for s, b in [(7, 4), (8, 6), (9, 7)]],
    ("sampled_screen", lambda: thb.test_sampled_screen_definition(11)),
    ("order14", lambda: thb.test_order_14_filter_of_long_patterns()),
]


def build_shim(src_text: str, tmp_path, name: str) -> str:
    if not shutil.which("g++"):
        pytest.skip("no host C++ compiler")
    from paper_1811_10498_gb300 import build_ext
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(build_ext.nvcc()))), "include")
    src = tmp_path / f"{name}.cpp"
    src.write_text(src_text)
    so = str(tmp_path / f"lib_{name}.so")
    subprocess.run(["g++", "-std=c++17", "-O1", "-shared", "-fPIC", "-pthread", f"-I{CSRC}", f"-I{cuda_inc}",
                    "-I" + os.path.join(ROOT, "include"), str(src), os.path.join(HERE, "native", "builder_shim.cpp"),
                    "-o", so], check=True)
    return so


def run_checks(monkeypatch, so: str, stop_at_first: bool):
    fake = BuilderOnly(so)
    monkeypatch.setattr(thb, "b", fake)
    monkeypatch.setattr(thb, "b_", fake)
    failed = []
    for name, check in CHECKS:
        try:
            check()
        except (AssertionError, _binding.PfacError):
            failed.append(name)
            if stop_at_first:
                break
    return failed


def test_unchanged_builder_passes_every_check(tmp_path, monkeypatch):
    so = build_shim(open(SRC).read(), tmp_path, "unchanged")
    assert run_checks(monkeypatch, so, stop_at_first=False) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_checks_catch_builder_mutant(name, tmp_path, monkeypatch):
    src = open(SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    so = build_shim(src.replace(old, new), tmp_path, name)
    assert run_checks(monkeypatch, so, stop_at_first=True), f"no check detects the builder mutant {name}"
