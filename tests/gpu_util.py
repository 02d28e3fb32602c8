"""Shared helpers for the GPU tests: device buffers in, numpy out, oracle beside."""
from __future__ import annotations

import os

import numpy as np
import pytest


def require_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1811_10498_gb300 import build_ext, _binding
    build_ext.build()
    _binding.lib()
    return torch


def host_threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def to_dev(a: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_match(table, text: np.ndarray, kernel: int | None = None, **cfg) -> np.ndarray:
    """Scan ASCII text through pfac_match."""
    import torch
    from paper_1811_10498_gb300 import _binding as b
    if kernel is not None or cfg:
        b.pfac_set_config(table.h, {"kernel": kernel or 0, **cfg})
    d_text = to_dev(text.astype(np.uint8)) if text.size else torch.empty(0, dtype=torch.uint8, device="cuda")
    d_out = torch.full((max(1, text.size),), -7, dtype=torch.int32, device="cuda")
    b.pfac_match(table.h, d_text, d_out)
    torch.cuda.synchronize()
    return d_out[: text.size].cpu().numpy()


def gpu_match_packed(table, text: np.ndarray, kernel: int | None = None, **cfg) -> np.ndarray:
    """Pack on the GPU, then scan through pfac_match_packed."""
    import torch
    from paper_1811_10498_gb300 import _binding as b
    if kernel is not None or cfg:
        b.pfac_set_config(table.h, {"kernel": kernel or 0, **cfg})
    d_text = to_dev(text.astype(np.uint8))
    packed, status, bad = b.pack(d_text)
    d_out = torch.full((max(1, text.size),), -7, dtype=torch.int32, device="cuda")
    b.pfac_match_packed(table.h, packed, text.size, d_out)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return d_out[: text.size].cpu().numpy()


def first_diff(a: np.ndarray, b: np.ndarray) -> str:
    d = np.flatnonzero(a != b)
    if d.size == 0:
        return "equal"
    i = int(d[0])
    return f"{d.size} differences, first at {i}: got {a[i]} want {b[i]}"
