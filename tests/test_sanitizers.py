"""The host code under AddressSanitizer and UndefinedBehaviorSanitizer (no GPU): the
table builder (csrc/trie_build.cpp) and the file front end (csrc/pfac_io.cpp) of the CUDA
library and, separately, the CPU oracle, each driven by a fuzz program in tests/sanitize/
with random inputs; and the builder's threads under ThreadSanitizer."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SAN = ["-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer"]


def _cuda_include():
    from paper_1811_10498_gb300 import build_ext
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(build_ext.nvcc()))), "include")


def _run(cmd, exe, tmp_path, *args):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip(f"sanitizer build unavailable: {r.stderr[-300:]}")
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1", UBSAN_OPTIONS="print_stacktrace=1",
               TSAN_OPTIONS="halt_on_error=1")
    r = subprocess.run([str(exe), *args], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    return r.stdout


def test_table_builder_under_sanitizers(tmp_path):
    if not shutil.which("g++"):
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "builder_fuzz"
    cmd = ["g++", "-std=c++17", "-pthread", *SAN, f"-I{_cuda_include()}", "-I" + os.path.join(ROOT, "include"),
           os.path.join(HERE, "sanitize", "builder_fuzz.cpp"),
           os.path.join(ROOT, "paper_1811_10498_gb300", "csrc", "trie_build.cpp"), "-o", str(exe)]
    assert "builder_fuzz: ok" in _run(cmd, exe, tmp_path)


def test_table_builder_threads_under_thread_sanitizer(tmp_path):
    """The sub-tries are built and written out on several threads: no data race."""
    if not shutil.which("g++"):
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "builder_fuzz_tsan"
    cmd = ["g++", "-std=c++17", "-pthread", "-O1", "-g", "-fsanitize=thread", f"-I{_cuda_include()}",
           "-I" + os.path.join(ROOT, "include"), os.path.join(HERE, "sanitize", "builder_fuzz.cpp"),
           os.path.join(ROOT, "paper_1811_10498_gb300", "csrc", "trie_build.cpp"), "-o", str(exe)]
    assert "builder_fuzz: ok" in _run(cmd, exe, tmp_path, "threaded")


def test_file_front_end_under_sanitizers(tmp_path):
    """Files read as texts and as pattern files: FASTA records are joined in place, and
    every pattern pointer handed to the table build stays inside the file's bytes."""
    if not shutil.which("g++"):
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "io_fuzz"
    cmd = ["g++", "-std=c++17", *SAN, f"-I{_cuda_include()}", "-I" + os.path.join(ROOT, "include"),
           os.path.join(HERE, "sanitize", "io_fuzz.cpp"),
           os.path.join(ROOT, "paper_1811_10498_gb300", "csrc", "pfac_io.cpp"), "-o", str(exe)]
    assert "io_fuzz: ok" in _run(cmd, exe, tmp_path, str(tmp_path / "f.txt"))


def test_oracle_under_sanitizers(tmp_path):
    if not shutil.which("gcc"):
        pytest.skip("no host C compiler")
    exe = tmp_path / "oracle_fuzz"
    cmd = ["gcc", "-std=c11", *SAN, os.path.join(HERE, "sanitize", "oracle_fuzz.c"),
           os.path.join(ROOT, "oracle", "pfac_oracle.c"), "-o", str(exe)]
    assert "oracle_fuzz: ok" in _run(cmd, exe, tmp_path)
