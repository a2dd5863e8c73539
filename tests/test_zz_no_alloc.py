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


def _static(lib, G, nu, theta, X, Y, ncols, stream=None):
    th = np.ascontiguousarray(theta, dtype=np.float64)
    return lib.hodlr_apply_static(G, nu, th.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()), ncols, stream)


def _context_product(G, nu, theta, X):
    """Y = K X through a context (hodlr_apply); X: ncols x G (rows are columns of the panel)."""
    from paper_2303_10102_gb300 import Hodlr
    h = Hodlr(1, G, 1, nu, "fp64", 64, 24, 0, 0.0, 1, device=DEV)
    return h.apply(theta, "K", X.t()).t().contiguous()


def test_static_scratch_entry_point_matches_context_entry_point():
    from paper_2303_10102_gb300 import lib as plib
    lib = plib.load()
    G = 1024
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(11)
    for theta in [(1.0, 0.1, 5.0, 1e-4), (0.7, 0.23, 3.0, 2e-2)]:           # two calls in a row
        X = torch.as_tensor(rng.standard_normal((7, G)), device=DEV)       # 7 columns, column-major G x 7
        ref = _context_product(G, 1.5, theta, X)
        Y = torch.full_like(X, float("nan"))
        rc = _static(lib, G, 1.5, theta, X, Y, 7, stream)
        torch.cuda.synchronize()
        assert rc == 0
        err = (Y - ref).abs().max().item() / ref.abs().max().item()
        assert err < 1e-13, err


def test_static_entry_point_at_capacity_then_smaller_grids():
    """The largest accepted grid (G = 2048: a 4096-point embedding fills the spectrum and
    embedding slots of the scratch array), then smaller grids that find its contents left in
    place: G = 320 against the context path and G = 2 (a 4-point embedding) against the FP64
    oracle's dense-free product."""
    from oracle.physics import Model
    from paper_2303_10102_gb300 import lib as plib
    lib = plib.load()
    rng = np.random.default_rng(12)
    cases = [(2048, 1.5, (1.0, 0.1, 5.0, 1e-4), 5), (320, 0.5, (0.8, 0.2, 3.0, 1e-2), 3),
             (2, 1.5, (1.2, 0.3, 4.0, 1e-3), 2)]
    for G, nu, theta, nc in cases:
        X = torch.as_tensor(rng.standard_normal((nc, G)), device=DEV)
        Y = torch.full_like(X, float("nan"))
        rc = _static(lib, G, nu, theta, X, Y, nc)
        torch.cuda.synchronize()
        assert rc == 0, G
        if G >= 64:
            ref = _context_product(G, nu, theta, X).cpu().numpy()
        else:
            ref = Model(1, G, 1, nu).apply(X.cpu().numpy().T, theta, "K").T
        got = Y.cpu().numpy()
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < 1e-13, (G, err)


def test_static_entry_point_rejects_oversized_grids_and_overlap():
    from paper_2303_10102_gb300 import lib as plib
    lib = plib.load()
    th = (1.0, 0.1, 5.0, 1e-4)
    X = torch.zeros(4096, device=DEV, dtype=torch.float64)
    Y = torch.zeros_like(X)
    assert _static(lib, 4096, 1.5, th, X, Y, 1) == -1
    # Y overlapping X (equal, or shifted by one row) is refused before any device work
    buf = torch.zeros(2 * 64 + 1, device=DEV, dtype=torch.float64)
    assert _static(lib, 64, 1.5, th, buf, buf, 2) == -1
    assert _static(lib, 64, 1.5, th, buf[:128], buf[1:], 2) == -1
    assert torch.count_nonzero(buf).item() == 0
