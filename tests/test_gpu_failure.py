"""Failure detection of the bounded device waits (HODLR_ETIMEOUT), made without a GPU fault.

The tensor-core products wait on mbarriers with a poll limit.  The test lowers the limit of
each CTA's first operand wait to zero polls through hodlr_debug_wait_limit, so that wait gives
up at once (the copies it waits for are real and in bounds: they land, and the CTA drains them
with the full limit before it frees its tensor memory).  The call must return HODLR_ETIMEOUT,
the status word must be cleared by that report, and with the default limit restored the same
context must give the correct product again.
"""
import numpy as np
import pytest

import synth
from oracle.physics import Model

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_first_operand_wait_gives_up_then_context_recovers():
    from paper_2303_10102_gb300 import Hodlr, HodlrError, lib as plib
    lib = plib.load()
    # 128^2 grid, FP32 fields: the DST products of the operator solve run on the tensor cores
    w = synth.small_workload(dim=2, G=128, nvar=1, nu=0.5, theta=(1.0, 0.1, 8.0, 1e-4), leaf=256, cap=16, c=16)
    h = Hodlr(w.dim, w.G, w.nvar, w.nu, "fp32", w.leaf, w.cap, w.c - w.cap, w.tol, w.seed_probe, device=DEV)
    X = np.random.default_rng(6).standard_normal((h.N, 4))
    ref = Model(w.dim, w.G, w.nvar, w.nu).apply(X, w.theta, "K")
    assert lib.hodlr_debug_wait_limit(0) == 0
    try:
        with pytest.raises(HodlrError) as e:
            h.apply(w.theta, "K", X)
        assert e.value.code == -5
    finally:
        assert lib.hodlr_debug_wait_limit(-1) == 0
    # the status was taken (cleared) by the failed call: two clean calls in a row succeed
    for _ in range(2):
        Y = h.apply(w.theta, "K", X).cpu().numpy()
        assert np.abs(Y - ref).max() / np.abs(ref).max() < 2e-5
