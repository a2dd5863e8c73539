"""The tile autotuner (hodlr_autotune) on the mixed BF16 path.

A 1-D model at N = 16384 whose peeling updates (block rows x rank x probe columns) and
projections (rank x probe columns over a block) are both shapes with fused and sliced-plane
candidates.  With tuning on, the first evaluation times every candidate of each new product
shape and remembers the fastest; the evaluation agrees with the untuned one to the rounding of
the products (different kernels, the same digit arithmetic), a second tuned evaluation repeats
the first bit for bit, and every remembered fused plan is one the shape allows.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_autotuned_evaluation_matches_and_repeats():
    from paper_2303_10102_gb300 import Hodlr
    from paper_2303_10102_gb300 import lib as plib
    lib = plib.load()
    assert lib.hodlr_autotune_clear() == 0
    w = synth.small_workload(dim=1, G=16384, nvar=1, nu=1.5, theta=(1.0, 0.1, 5.0, 1e-4), leaf=64, cap=24, c=32)
    y = torch.as_tensor(synth.simulate_y(w), device=DEV)
    h = Hodlr(1, w.G, 1, 1.5, "bf16", w.leaf, w.cap, w.c - w.cap, 0.0, w.seed_probe, device=DEV, guard=1e-7)
    theta = (0.9, 0.12, 4.5, 2e-4)
    f0, g0, F0 = h.eval(theta, y)
    h.autotune(True)
    f1, g1, F1 = h.eval(theta, y)
    table = plib.autotune_table()
    f2, g2, F2 = h.eval(theta, y)
    h.autotune(False)
    try:
        assert len(table) > 0
        kinds = set()
        for r in table:
            if r["path"] == 1:
                Kp = -(-r["K"] // 32) * 32
                long_k = r["tA"] == 1 and r["tB"] == 0 and r["M"] <= 128 and Kp >= 1024
                short_k = r["tA"] == 0 and Kp <= 64 and r["M"] >= 128 and r["M"] * r["batch"] >= 4096
                assert long_k or short_k, r
                kinds.add("long" if long_k else "short")
                assert r["tile"] in (0, 1) and r["cprx"] in (1, 4)
        print(f"{len(table)} shapes tuned; fused plans chosen for {sorted(kinds)}")
        assert f1 == f2 and np.array_equal(np.asarray(g1), np.asarray(g2)) and np.array_equal(np.asarray(F1), np.asarray(F2))
        assert abs(f1 - f0) <= 1e-9 * abs(f0)
        assert np.all(np.abs(np.asarray(g1) - np.asarray(g0)) <= 1e-5 * np.abs(np.asarray(g0)) + 1e-9)
        assert np.all(np.abs(np.asarray(F1) - np.asarray(F0)) <= 1e-5 * np.abs(np.asarray(F0)))
    finally:
        lib.hodlr_autotune_clear()
