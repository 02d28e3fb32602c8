"""Plant plausible mistakes in copies of the CPU oracle and check that the pins
catch every one of them (CPU only; the mutants are built with the host compiler
into a temporary folder and never touch the real oracle)."""
import os
import subprocess

import pytest

import oracle
import pins

MUTANTS = {
    # Section IV: report the longest pattern, not the first one met on the walk.
    "first_match_instead_of_longest": (
        "if (t->term[s] != 0) best = t->term[s];",
        "if (t->term[s] != 0) { best = t->term[s]; break; }"),
    # Duplicates: the lowest id must be kept.
    "last_duplicate_wins": (
        "if (t->term[s] == 0) t->term[s] = j + 1;",
        "t->term[s] = j + 1;"),
    # The walk must be allowed to use the last text byte.
    "stops_one_before_text_end": (
        "for (int64_t k = i; k < len; k++) {",
        "for (int64_t k = i; k + 1 < len; k++) {"),
    # Transposed table operands.
    "transposed_goto_index": (
        "int64_t nxt = t->go[4 * s + c];",
        "int64_t nxt = t->go[4 * c + s];"),
    # A byte outside ACGT ends the walk; it must not be skipped.
    "non_acgt_skipped": (
        "if (c < 0) break;\n            int64_t nxt",
        "if (c < 0) continue;\n            int64_t nxt"),
    # Failure-less: a missing edge ends the walk instead of restarting at the root.
    "restart_at_root_on_miss": (
        "if (nxt == 0) break;",
        "if (nxt == 0) { s = 0; continue; }"),
    # Classic AC: failure links must follow the textbook definition.
    "failure_always_root": (
        "m->fail[r] = g->go[4 * t + c];",
        "m->fail[r] = 0;"),
    # Classic AC: output(s) must include output(f(s)).
    "output_link_dropped": (
        "m->onext[r] = (m->id_start[f + 1] > m->id_start[f]) ? f : m->onext[f];",
        "m->onext[r] = 0;"),
    # Insertion order: a new state is the next free number.
    "states_numbered_from_two": (
        "t->n = 1;\n    for (int32_t j = 0; j < n; j++) {",
        "t->n = 2;\n    for (int32_t j = 0; j < n; j++) {"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    src = open(oracle.SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    so = str(tmp_path / f"lib_{name}.so")
    subprocess.run(["gcc", "-O1", "-shared", "-fPIC", str(path), "-o", so], check=True)
    lib = oracle.load(so)
    failed = []
    for check in pins.ALL_PINS:
        try:
            if check is pins.check_random_tiny:
                check(lib, cases=150)
            else:
                check(lib)
        except (AssertionError, oracle.OracleError):
            failed.append(check.__name__)
    assert failed, f"no pin detects the mutant {name}"
