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
