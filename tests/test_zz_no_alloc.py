"""The allocation-free entry point hodlr_apply_static (for callers that cannot allocate device
memory) gives the same product as the context-based hodlr_apply, on two calls in a row.

Kept in a file of its own that pytest collects last, so a run that stops at the first
failure has run every other test before it; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_static_scratch_entry_point_matches_context_entry_point():
    from paper_2303_10102_gb300 import Hodlr, lib as plib
    lib = plib.load()
    G = 1024
    h = Hodlr(1, G, 1, 1.5, "fp64", 64, 24, 0, 0.0, 1, device=DEV)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(11)
    for theta in [(1.0, 0.1, 5.0, 1e-4), (0.7, 0.23, 3.0, 2e-2)]:           # two calls in a row
        X = torch.as_tensor(rng.standard_normal((7, G)), device=DEV)       # 7 columns, column-major G x 7
        ref = h.apply(theta, "K", X.t()).t().contiguous()
        Y = torch.full_like(X, float("nan"))
        th = np.ascontiguousarray(theta, dtype=np.float64)
        rc = lib.hodlr_apply_static(G, 1.5, th.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()), 7, stream)
        torch.cuda.synchronize()
        assert rc == 0
        err = (Y - ref).abs().max().item() / ref.abs().max().item()
        assert err < 1e-13, err


def test_static_entry_point_rejects_oversized_grids():
    from paper_2303_10102_gb300 import lib as plib
    lib = plib.load()
    th = np.array([1.0, 0.1, 5.0, 1e-4])
    X = torch.zeros(4096, device=DEV, dtype=torch.float64)
    Y = torch.zeros_like(X)
    rc = lib.hodlr_apply_static(4096, 1.5, th.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()), 1, None)
    assert rc == -1
