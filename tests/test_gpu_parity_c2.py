"""Parity of the mixed-precision path (HODLR_MIXED_BF16: FP64-class products on the BF16 tensor
cores) at the benched configuration's settings.

Workload P2: C2's model and HODLR settings (2-D univariate, Matern nu = 1/2, kappa = 8, leaf 256,
rank cap 128, c = 136 probe columns, tol = guard = 1e-6, FP32/TF32 bulk) on a 128^2 grid
(N = 16384, tau = 6).  At this size the level-1 blocks are 8192 rows high, so the tensor-core
products run with many 128-row M tiles, split K and batched row offsets, as at C2.

Expected values come from tests/golden/p2_oracle.txt, written by tests/golden/make_p2_golden.py
from the FP64 oracle (densified K~ and K~_j; dense NLL, gradient and Fisher) at two parameter
points: theta0, the configuration's own (where the score is a zero-mean random vector), and a
starting point of an optimisation away from it, where every score component is large.

Two comparisons per point:
  * frozen pivots: the GPU builds with the oracle's pivot sets, so both sides evaluate the same
    approximation; every result is compared with its own relative error against the stated
    targets (NLL 1e-6, each gradient component and each Fisher entry 1e-4), and the paper's
    scale-free errors eta_g and eta_I (Sec. 5.2.2, eq. score-error and eq. fisher-error) are
    checked against 1e-4 as well;
  * own pivots: the GPU takes its own rank decisions on FP32 data; the kept ranks must stay
    within the ambiguity of the rank rule (a few columns per block near the threshold
    max(tol, guard) |R_11|), and the likelihood must stay within its target.
"""
import os

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GOLD = os.path.join(os.path.dirname(__file__), "golden", "p2_oracle.txt")


def load_golden():
    pts = []
    with open(GOLD) as f:
        for ln in f:
            if not ln.strip() or ln.startswith("#"):
                continue
            k, *v = ln.split()
            if k == "theta":
                pts.append({"theta": tuple(float(x) for x in v), "piv": {}})
            elif k in ("nll", "grad", "fisher"):
                pts[-1][k] = np.array([float(x) for x in v])
            elif k == "piv":
                l, p, r = int(v[0]), int(v[1]), int(v[2])
                pts[-1]["piv"][(l, p)] = [int(x) for x in v[3:3 + r]]
    for d in pts:
        d["nll"] = float(d["nll"][0])
        d["fisher"] = d["fisher"].reshape(4, 4)
        tau = max(l for l, _ in d["piv"])
        d["sets"] = [[d["piv"][(l, p)] for p in range(1 << (l - 1))] for l in range(1, tau + 1)]
    return pts


def eta_g(S, S0, F0):
    """||S - S~|| in the I^{-1} norm (eq. score-error)."""
    d = np.asarray(S) - np.asarray(S0)
    return float(np.sqrt(d @ np.linalg.solve(F0, d)))


def eta_I(F, F0):
    """tr((I - I~)(I^{-1} - I~^{-1}))^{1/2} (eq. fisher-error)."""
    return float(np.sqrt(abs(np.trace((F0 - F) @ (np.linalg.inv(F0) - np.linalg.inv(F))))))


def errors(f, g, F, d):
    return {"nll": abs(f - d["nll"]) / abs(d["nll"]),
            "grad": np.abs(g - d["grad"]) / np.abs(d["grad"]),
            "fisher": np.abs(F - d["fisher"]) / np.abs(d["fisher"]),
            "eta_g": eta_g(g, d["grad"], d["fisher"]), "eta_I": eta_I(F, d["fisher"])}


@pytest.fixture(scope="module")
def p2():
    from paper_2303_10102_gb300 import Hodlr
    w = synth.workload("P2")
    h = Hodlr(w.dim, w.G, w.nvar, w.nu, "bf16", w.leaf, w.cap, w.c - w.cap, w.tol, w.seed_probe, device=DEV,
              guard=w.guard)
    y = torch.as_tensor(synth.simulate_y(w), device=DEV)
    yield w, h, y
    del h
    torch.cuda.empty_cache()


@pytest.mark.parametrize("point", [0, 1])
def test_p2_mixed_frozen_pivots_per_result(p2, point):
    w, h, y = p2
    d = load_golden()[point]
    h.set_pivots(h.pivots_from_sets(d["sets"]))
    try:
        f, g, F = h.eval(d["theta"], y)
    finally:
        h.set_pivots(None)
    e = errors(f, g, np.asarray(F), d)
    print(f"P2 point {point} frozen pivots: nll {e['nll']:.2e} grad {np.array2string(e['grad'], formatter={'float_kind': lambda v: f'{v:.2e}'})} "
          f"fisher max {e['fisher'].max():.2e} eta_g {e['eta_g']:.2e} eta_I {e['eta_I']:.2e}")
    assert e["nll"] <= 1e-6, e
    assert np.all(e["grad"] <= 1e-4), e
    assert np.all(e["fisher"] <= 1e-4), e
    assert e["eta_g"] <= 1e-4 and e["eta_I"] <= 1e-4, e


@pytest.mark.parametrize("point", [0, 1])
def test_p2_mixed_own_rank_decisions(p2, point):
    w, h, y = p2
    d = load_golden()[point]
    h.set_pivots(None)
    f, g, F = h.eval(d["theta"], y)
    ranks = h.ranks()
    diffs = [abs(a - len(J)) for rl, Jl in zip(ranks, d["sets"]) for a, J in zip(rl, Jl)]
    e = errors(f, g, np.asarray(F), d)
    print(f"P2 point {point} own pivots: max rank difference {max(diffs)}, mean {np.mean(diffs):.2f}; "
          f"nll {e['nll']:.2e} grad {np.array2string(e['grad'], formatter={'float_kind': lambda v: f'{v:.2e}'})} fisher max {e['fisher'].max():.2e} "
          f"eta_g {e['eta_g']:.2e} eta_I {e['eta_I']:.2e}")
    assert max(diffs) <= 4, diffs
    assert e["nll"] <= 1e-6, e
