"""Helpers shared by the GPU tests (not collected)."""
from __future__ import annotations

import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def lib():
    need_gpu()
    import paper_2603_02207_gb300 as L
    return L


def rel_err(got, want) -> float:
    """max |got - want| / max |want| (block max-norm relative error)."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    den = np.max(np.abs(want))
    return float(np.max(np.abs(got - want)) / (den if den > 0 else 1.0))


# tolerances of the parity bar: FP64-class paths 1e-10, FP32-mixed 2e-5 (relative)
TOL = {"f64": 1e-10, "df64": 1e-10, "f32": 2e-5}
