"""Plant plausible mistakes in copies of the CPU oracle and check that the pins
catch every one of them (CPU only). Mutants of the C part are built with the host
compiler into a temporary folder; mutants of the Python part are executed as a
separate module whose function stands in for the oracle's during the test. Neither
touches the real oracle."""
import subprocess
import types

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


# Mutants of the Python part of the oracle: (function replaced, old text, new text).
PY_MUTANTS = {
    # A start is end - length + 1.
    "all_matches_start_off_by_one": ("all_matches",
        "starts = ends - lens + 1",
        "starts = ends - lens"),
    # Equal pattern strings at one start: the lowest id is reported.
    "all_matches_keeps_highest_duplicate_id": ("all_matches",
        "order = np.lexsort((ids, lens, starts))",
        "order = np.lexsort((-ids, lens, starts))"),
    # Equal pattern strings at one start are reported once.
    "all_matches_without_dedupe": ("all_matches",
        "keep[1:] = (starts[1:] != starts[:-1]) | (lens[1:] != lens[:-1])",
        "keep[1:] = True"),
    # Within a start the list is ordered by length, not by id.
    "all_matches_sorted_by_id": ("all_matches",
        "order = np.lexsort((ids, lens, starts))",
        "order = np.lexsort((lens, ids, starts))"),
    # Base p goes to the low bits of its word first.
    "pack_high_bits_first": ("pack",
        "shifts = (2 * np.arange(16, dtype=np.uint32))",
        "shifts = (30 - 2 * np.arange(16, dtype=np.uint32))"),
    # The first bad byte is reported at its own offset.
    "pack_first_bad_off_by_one": ("pack",
        "first_bad = int(bad[0]) if bad.size else -1",
        "first_bad = int(bad[0]) + 1 if bad.size else -1"),
    # A walk ends at its read's end, not at the end of the concatenated reads.
    "reads_walk_into_the_next_read": ("pfac_scan_reads",
        "out[lo:hi] = tries[k].scan(reads[lo:hi])",
        "out[lo:hi] = tries[k].scan(reads, lo, hi)[lo:hi]"),
    # Each read uses the table its entry names.
    "reads_all_with_the_first_set": ("pfac_scan_reads",
        "k = int(read_set[r])",
        "k = 0"),
    # Offsets with id 0 are not matches.
    "compact_keeps_zeros": ("compact",
        "offs = np.flatnonzero(out_ids).astype(np.int64)",
        "offs = np.arange(out_ids.size, dtype=np.int64)"),
}


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_pins_catch_python_mutant(name, monkeypatch):
    func, old, new = PY_MUTANTS[name]
    path = oracle.__file__
    src = open(path).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mod = types.ModuleType("oracle_mutant")
    mod.__file__ = path
    exec(compile(src.replace(old, new), path, "exec"), mod.__dict__)
    monkeypatch.setattr(oracle, func, getattr(mod, func))
    lib = oracle.load()
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


def test_python_mutant_harness_passes_the_unchanged_oracle(monkeypatch):
    """Control: the oracle's own source, executed the same way, passes every pin."""
    path = oracle.__file__
    mod = types.ModuleType("oracle_copy")
    mod.__file__ = path
    exec(compile(open(path).read(), path, "exec"), mod.__dict__)
    for func in {f for f, _, _ in PY_MUTANTS.values()}:
        monkeypatch.setattr(oracle, func, getattr(mod, func))
    lib = oracle.load()
    for check in pins.ALL_PINS:
        check(lib)
