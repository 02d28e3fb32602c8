"""The C-ABI library loads and exports every entry point include/pfac.h declares
(no GPU needed; no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pfac.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(pfac_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["pfac_build", "pfac_destroy", "pfac_info", "pfac_pack", "pfac_match",
                     "pfac_match_packed", "pfac_match_compact", "pfac_match_batched",
                     "pfac_last_error", "pfac_error_string"]:
        assert required in names


def test_library_exports_every_declared_symbol(cuda_lib_path):
    lib = ctypes.CDLL(cuda_lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(cuda_lib_path):
    from paper_1811_10498_gb300 import _binding
    assert sorted(_binding._SIGS) == declared_functions()


def test_error_strings(cuda_lib_path):
    from paper_1811_10498_gb300 import _binding as b
    L = b.lib()
    for code, name in b.STATUS.items():
        s = L.pfac_error_string(code).decode()
        assert s and s != "unknown status", (code, name)
    assert L.pfac_error_string(999).decode() == "unknown status"


def test_build_errors_without_gpu(cuda_lib_path):
    from paper_1811_10498_gb300 import _binding as b
    cases = [([b"ACG", b""], "PFAC_ERR_EMPTY_PATTERN"), ([b"ACG", b"ACN"], "PFAC_ERR_BAD_SYMBOL"),
             ([b"acg"], "PFAC_ERR_BAD_SYMBOL"), ([], "PFAC_ERR_INVALID_ARG")]
    for pats, code in cases:
        with pytest.raises(b.PfacError) as e:
            b.pfac_build(pats, host_only=True)
        assert e.value.code == b.CODE[code]


def test_host_only_handle_rejects_scans(cuda_lib_path):
    from paper_1811_10498_gb300 import _binding as b
    L = b.lib()
    h = b.pfac_build([b"ACGT"], host_only=True)
    try:
        assert L.pfac_match(h, None, 10, None, None) == b.CODE["PFAC_ERR_HOST_ONLY"]
        assert L.pfac_match_packed(h, None, 10, None, None) == b.CODE["PFAC_ERR_HOST_ONLY"]
        assert b.pfac_info_ex(h)["device"] == -1
    finally:
        b.pfac_destroy(h)


def test_launch_configuration_checks(cuda_lib_path):
    """pfac_set_config rejects values outside the documented ranges, refuses kernel 2 for
    a table without a prefix filter, and pfac_get_config reports what was set (host-only
    handles: no device call)."""
    from paper_1811_10498_gb300 import _binding as b
    h = b.pfac_build([b"ACGT", b"GATTACA", b"TTAGG"], host_only=True, filter_b=4)
    h_plain = b.pfac_build([b"ACGT"], host_only=True, filter_b=-1)
    try:
        good = {"kernel": 2, "threads": 512, "ctas_per_sm": 1, "stages": 4, "walk_loads": 3, "lane_offsets": 32,
                "table_layout": 2, "row_loads": 2, "text_smem": 1, "zero_writer": 3}
        b.pfac_set_config(h, good)
        got = b.pfac_get_config(h)
        assert {k: got[k] for k in good} == good
        for field, bad in [("kernel", 3), ("kernel", -1), ("threads", 100), ("threads", 32), ("threads", 2048),
                           ("ctas_per_sm", 33), ("stages", 1), ("stages", 9), ("walk_loads", -1),
                           ("lane_offsets", 8), ("lane_offsets", 64), ("table_layout", 3), ("table_layout", -1),
                           ("row_loads", 3), ("text_smem", 2), ("zero_writer", 5), ("zero_writer", -1), ("l2_persist", 3), ("l2_persist", -2)]:
            with pytest.raises(b.PfacError) as e:
                b.pfac_set_config(h, dict(good, **{field: bad}))
            assert e.value.code == b.CODE["PFAC_ERR_INVALID_ARG"], (field, bad)
        # a rejected configuration leaves the previous one in place
        assert {k: b.pfac_get_config(h)[k] for k in good} == good
        with pytest.raises(b.PfacError) as e:
            b.pfac_set_config(h_plain, {"kernel": 2})
        assert e.value.code == b.CODE["PFAC_ERR_UNSUPPORTED"]
        b.pfac_set_config(h_plain, {"kernel": 1})
        # zero fields mean the library's default; a reset restores every default
        b.pfac_set_config(h, {"kernel": 0})
        d = b.pfac_get_config(h)
        assert d["stages"] == 3 and d["lane_offsets"] == 32 and d["threads"] == 1024
        b.pfac_set_config(h, None)
        assert b.pfac_get_config(h) == d
    finally:
        b.pfac_destroy(h)
        b.pfac_destroy(h_plain)


_OOM_CHILD = r"""
import resource, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
from paper_1811_10498_gb300 import _binding as b
b.lib()
rng = np.random.default_rng(0)
n, L = 200_000, 200                     # about 40M trie states: gigabytes of tables
blob = np.frombuffer(b"ACGT", dtype=np.uint8)[rng.integers(0, 4, n * L)]
offs = np.arange(0, n * L + 1, L, dtype=np.int64)
vm = next(int(l.split()[1]) * 1024 for l in open("/proc/self/status") if l.startswith("VmSize"))
limit = vm + (400 << 20)
resource.setrlimit(resource.RLIMIT_AS, (limit, limit))
try:
    b.pfac_build((blob, offs), host_only=True)
    print("built")
except b.PfacError as e:
    print("code", e.code)
h = b.pfac_build([b"ACGT", b"GATTACA"], host_only=True)      # the library still works
print("small ok", b.pfac_info_ex(h)["n_states"])
b.pfac_destroy(h)
"""


def test_build_out_of_host_memory_reports_oom(cuda_lib_path, tmp_path):
    """A build whose tables do not fit in the memory the process may take fails with
    PFAC_ERR_OOM and a NULL handle (the failure is made on the host: the child process
    caps its own address space), and the library keeps working afterwards."""
    import subprocess
    import sys
    if not os.path.exists("/proc/self/status"):
        pytest.skip("needs /proc")
    script = tmp_path / "oom_child.py"
    script.write_text(_OOM_CHILD)
    r = subprocess.run([sys.executable, str(script), ROOT], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = r.stdout.split("\n")
    from paper_1811_10498_gb300 import _binding as b
    assert f"code {b.CODE['PFAC_ERR_OOM']}" in lines, r.stdout
    assert "small ok 12" in lines, r.stdout


def test_table_lifecycle(cuda_lib_path, tmp_path):
    """Table owns its handle: a context manager closes it, close() twice is harmless, and
    a closed table raises instead of passing a stale handle to the library."""
    from paper_1811_10498_gb300 import _binding as b
    with b.Table([b"ACGT", b"GATTACA"], host_only=True) as t:
        assert t.info["n_patterns"] == 2
    assert t.h is None
    t.close()
    with pytest.raises(b.PfacError) as e:
        t.info
    assert e.value.code == b.CODE["PFAC_ERR_INVALID_ARG"]
    f = tmp_path / "p.txt"
    f.write_bytes(b"ACGT\nGATTACA\n")
    with b.Table.from_file(str(f), host_only=True) as t2:
        assert t2.info["n_states"] == 12


def test_plain_c_client(cuda_lib_path, tmp_path):
    """The header compiles as strict C99, and a C program linked against the library
    builds, exports and destroys host-only tables and reads its error codes, with no
    Python in between (tests/native/c_client.c)."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no host C compiler")
    exe = tmp_path / "c_client"
    libdir = os.path.dirname(cuda_lib_path)
    lib = os.path.basename(cuda_lib_path)
    assert lib.startswith("lib") and lib.endswith(".so")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I" + os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "native", "c_client.c"), f"-L{libdir}", f"-l{lib[3:-3]}",
                    f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("c_client: ok")
