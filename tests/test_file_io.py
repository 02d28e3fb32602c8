"""The file front end (pattern and text files, as the paper's host program reads them,
Section V-B, Figs. 4 and 5): host-only handles, so no GPU is needed."""
import numpy as np
import pytest

from paper_1811_10498_gb300 import _binding as b


@pytest.fixture(scope="module", autouse=True)
def _lib(cuda_lib_path):
    return cuda_lib_path


def export(h):
    rows, out_id, _ = b.pfac_export(h)
    return rows, out_id


def same_table(h_file, pats):
    want = b.pfac_build(pats, host_only=True)
    try:
        r1, o1 = export(h_file)
        r2, o2 = export(want)
        assert np.array_equal(r1, r2) and np.array_equal(o1, o2)
    finally:
        b.pfac_destroy(want)


def test_pattern_file_one_per_line(tmp_path):
    p = tmp_path / "pats.txt"
    p.write_bytes(b"ACGT\r\n\nGATTACA\nACG\n\n\nTT")       # CRLF, blank lines, no final newline
    h = b.pfac_build_file(str(p), host_only=True)
    try:
        same_table(h, [b"ACGT", b"GATTACA", b"ACG", b"TT"])
        assert b.pfac_info_ex(h)["n_patterns"] == 4
    finally:
        b.pfac_destroy(h)


def test_pattern_file_fasta(tmp_path):
    p = tmp_path / "pats.fa"
    p.write_bytes(b"\n>p1 first\nACGT\nAC\n>p2\r\nGGG\r\n>p3\nT\n")
    h = b.pfac_build_file(str(p), host_only=True)
    try:
        same_table(h, [b"ACGTAC", b"GGG", b"T"])
    finally:
        b.pfac_destroy(h)


def test_pattern_file_errors(tmp_path):
    with pytest.raises(b.PfacError) as e:
        b.pfac_build_file(str(tmp_path / "missing.txt"), host_only=True)
    assert e.value.code == b.CODE["PFAC_ERR_IO"]
    bad = tmp_path / "bad.txt"
    bad.write_bytes(b"ACGT\nacgt\n")                          # no case folding
    with pytest.raises(b.PfacError) as e:
        b.pfac_build_file(str(bad), host_only=True)
    assert e.value.code == b.CODE["PFAC_ERR_BAD_SYMBOL"]
    empty = tmp_path / "empty.txt"
    empty.write_bytes(b"\n\n")
    with pytest.raises(b.PfacError) as e:
        b.pfac_build_file(str(empty), host_only=True)
    assert e.value.code == b.CODE["PFAC_ERR_INVALID_ARG"]


def test_text_file_as_is_and_fasta(tmp_path):
    raw = b"ACGTNACGT\nGATTACA\r\n\nTTT"
    p = tmp_path / "text.txt"
    p.write_bytes(raw)
    assert b.read_text_file(str(p)).tobytes() == raw          # bytes as they are
    fa = tmp_path / "reads.fa"
    fa.write_bytes(b">r1\nACGT\nACGT\n>r2 x\r\nGG\r\nCC\r\n>r3\nA\n")
    assert b.read_text_file(str(fa), fasta=True).tobytes() == b"ACGTACGT\nGGCC\nA"
    with pytest.raises(b.PfacError) as e:
        b.read_text_file(str(tmp_path / "missing.txt"))
    assert e.value.code == b.CODE["PFAC_ERR_IO"]
    e0 = tmp_path / "zero.txt"
    e0.write_bytes(b"")
    assert b.read_text_file(str(e0)).size == 0


def fasta_reference(raw: bytes):
    """Records of a FASTA file by the front end's rules, written out plainly: lines split
    at '\\n' with a trailing '\\r' dropped, empty lines skipped, a line starting with '>'
    opens a record, a sequence line before any header opens one too, and a record's
    sequence lines are joined."""
    recs = []
    for line in raw.split(b"\n"):
        if line.endswith(b"\r"):
            line = line[:-1]
        if not line:
            continue
        if line.startswith(b">"):
            recs.append(b"")
            continue
        if not recs:
            recs.append(b"")
        recs[-1] += line
    return recs


@pytest.mark.parametrize("seed", range(12))
def test_fasta_files_against_the_plain_rules(tmp_path, seed):
    """Random line mixes (seeds 0-5, headers without sequence included) and well-formed
    files where every header has one to three sequence lines (seeds 6-11)."""
    rng = np.random.default_rng(seed)

    def seq():
        return rng.choice(np.frombuffer(b"ACGT", dtype=np.uint8), size=int(rng.integers(1, 30))).tobytes()

    parts = []
    for _ in range(int(rng.integers(1, 40))):
        kind = rng.integers(0, 10)
        if kind < 3:
            parts.append(b">rec " + str(int(rng.integers(1000))).encode())
            if seed >= 6:
                parts += [seq() for _ in range(int(rng.integers(1, 4)))]
        elif kind < 4:
            parts.append(b"")
        else:
            parts.append(seq())
    ends = [b"\r\n" if rng.random() < 0.3 else b"\n" for _ in parts]
    raw = b"".join(p + e for p, e in zip(parts, ends))
    if rng.random() < 0.5:
        raw = raw.rstrip(b"\r\n")                        # no final newline
    if seed % 2 == 0 and not raw.lstrip(b"\r\n").startswith(b">"):
        raw = b">first\n" + raw                          # a FASTA file for the pattern front end
    f = tmp_path / "x.fa"
    f.write_bytes(raw)
    recs = fasta_reference(raw)
    assert b.read_text_file(str(f), fasta=True).tobytes() == b"\n".join(recs)
    if not raw.lstrip(b"\r\n\t ").startswith(b">"):
        return                                           # read as one pattern per line instead
    if not recs or any(len(r) == 0 for r in recs):
        with pytest.raises(b.PfacError) as e:
            b.pfac_build_file(str(f), host_only=True)
        assert e.value.code in (b.CODE["PFAC_ERR_EMPTY_PATTERN"], b.CODE["PFAC_ERR_INVALID_ARG"])
        return
    h = b.pfac_build_file(str(f), host_only=True)
    try:
        same_table(h, recs)
        assert b.pfac_info_ex(h)["n_patterns"] == len(recs)
    finally:
        b.pfac_destroy(h)


def test_fasta_header_without_sequence_is_an_empty_pattern(tmp_path):
    f = tmp_path / "e.fa"
    f.write_bytes(b">a\nACGT\n>b\n>c\nGG\n")
    with pytest.raises(b.PfacError) as e:
        b.pfac_build_file(str(f), host_only=True)
    assert e.value.code == b.CODE["PFAC_ERR_EMPTY_PATTERN"]
    assert b.read_text_file(str(f), fasta=True).tobytes() == b"ACGT\n\nGG"
