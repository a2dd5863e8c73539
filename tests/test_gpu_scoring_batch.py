"""Fisher scoring (host loop over the CUDA evaluation) and the batched entry point, against the
FP64 oracle."""
import numpy as np
import pytest
import torch

import synth
from oracle import hodlr as oh, likelihood as ol, scoring as oscoring
from oracle.physics import Model
from oracle.tree import Tree

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_fisher_scoring_iterates_match_oracle():
    from paper_2303_10102_gb300 import Hodlr
    from paper_2303_10102_gb300.scoring import fisher_scoring
    w = synth.small_workload(dim=1, G=512, nvar=1, nu=1.5, theta=(1.0, 0.1, 3.0, 1e-2), leaf=32, cap=8, c=8)
    start = (0.8, 0.12, 3.5, 1.5e-2)
    m, t = Model(1, w.G, 1, 1.5), Tree(1, w.G, 1, 32)
    y = synth.simulate_y(w)
    h = Hodlr(1, w.G, 1, 1.5, "fp64", 32, 8, 0, 0.0, 1, device=DEV)
    h.build(start)
    h.set_pivots(h.get_pivots())          # probes and pivots fixed across theta (Sec. 3.3)
    H0 = oh.build(m, t, start, c=8, cap=8, guard=1e-5, seed=1, params=())
    J = H0.pivots()
    yt = t.to_tree(y)

    def ev(th):
        return ol.evaluate(oh.build(m, t, tuple(th), c=8, cap=8, guard=1e-5, seed=1, frozen=J), yt)

    hist_g, hist_o = [], []
    fisher_scoring(h, torch.as_tensor(y, device=DEV), start, max_iter=3, history=hist_g)
    oscoring.fisher_scoring(ev, start, max_iter=3, history=hist_o)
    assert len(hist_g) == len(hist_o) == 3
    for a, b in zip(hist_g, hist_o):
        assert np.allclose(a["theta"], b["theta"], rtol=1e-6, atol=0), (a, b)
        assert abs(a["nll"] - b["nll"]) <= 1e-9 * abs(b["nll"])


def test_batched_entry_point_matches_single_calls():
    import ctypes
    from paper_2303_10102_gb300 import Hodlr, lib as plib
    lib = plib.load()
    ws = [synth.small_workload(dim=1, G=G, nvar=1, nu=1.5, theta=th, leaf=64, cap=8, c=8)
          for G, th in [(1024, (1.0, 0.1, 5.0, 1e-3)), (2048, (1.2, 0.05, 9.0, 1e-3)), (512, (0.7, 0.2, 2.5, 1e-2))]]
    hs = [Hodlr(1, w.G, 1, 1.5, "fp64", 64, 8, 0, 0.0, 1, device=DEV) for w in ws]
    ys = [torch.as_tensor(synth.simulate_y(w), device=DEV) for w in ws]
    thetas = np.ascontiguousarray(np.array([w.theta for w in ws]), dtype=np.float64)
    nll = np.zeros(3)
    grad = np.zeros(12)
    HP = ctypes.c_void_p * 3
    rc = lib.hodlr_batch_nll_grad(HP(*[h.h for h in hs]), 3, thetas.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  HP(*[ctypes.c_void_p(y.data_ptr()) for y in ys]),
                                  nll.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  grad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert rc == 0
    for i, (w, h, y) in enumerate(zip(ws, hs, ys)):
        # a single call after the batched one rebuilds (the graph leaves no host-side state)
        f, g, _ = h.eval(w.theta, y)
        # the graph evaluation uses the rank cap as every level's width (zero columns past a
        # pair's rank), so its products differ from the single call's in rounding only
        assert abs(f - nll[i]) <= 1e-12 * abs(f)
        assert np.abs(g - grad[4 * i:4 * i + 4]).max() <= 1e-10 * np.abs(g).max()
        m, t = Model(1, w.G, 1, 1.5), Tree(1, w.G, 1, 64)
        f0, g0, _ = ol.evaluate(oh.build(m, t, w.theta, c=8, cap=8, guard=1e-5, seed=1), t.to_tree(y.cpu().numpy()))
        assert abs(f - f0) <= 1e-10 * abs(f0)


def test_batched_uneven_datasets_in_one_graph():
    """The batched 1-D workload's structure (uneven dataset sizes, per-dataset theta, leaf 64 and
    24 probe columns, every NLL and gradient in one CUDA-graph launch) on four small datasets of
    uneven cluster trees, each against the FP64 oracle; a second launch with the same inputs
    replays the cached graph and gives the same numbers."""
    import ctypes
    from paper_2303_10102_gb300 import Hodlr, lib as plib
    lib = plib.load()
    sizes = [4100, 5000, 6001, 4096]
    thetas = [(1.0, 0.08, 4.0, 1e-4), (1.0, 0.21, 12.0, 1e-4), (1.0, 0.03, 2.5, 1e-4), (1.0, 0.12, 17.0, 1e-4)]
    ws = [synth.small_workload(dim=1, G=G, nvar=1, nu=1.5, theta=th, leaf=64, cap=24, c=24)
          for G, th in zip(sizes, thetas)]
    hs = [Hodlr(1, w.G, 1, 1.5, "bf16", 64, 24, 0, 0.0, 1, device=DEV) for w in ws]
    ys = [torch.as_tensor(synth.simulate_y(w), device=DEV) for w in ws]
    th = np.ascontiguousarray(np.array(thetas), dtype=np.float64)
    HP = ctypes.c_void_p * len(ws)
    outs = []
    for _ in range(2):
        nll = np.zeros(len(ws))
        grad = np.zeros(4 * len(ws))
        rc = lib.hodlr_batch_nll_grad(HP(*[h.h for h in hs]), len(ws), th.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      HP(*[ctypes.c_void_p(y.data_ptr()) for y in ys]),
                                      nll.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      grad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        assert rc == 0
        outs.append((nll, grad))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    nll, grad = outs[0]
    for i, (w, y) in enumerate(zip(ws, ys)):
        m, t = Model(1, w.G, 1, 1.5), Tree(1, w.G, 1, 64)
        assert t.tau >= 6
        H = oh.build(m, t, w.theta, c=24, cap=24, guard=1e-5, seed=1)
        f0, g0, _ = ol.evaluate(H, t.to_tree(y.cpu().numpy()))
        assert abs(nll[i] - f0) <= 1e-9 * abs(f0), (i, nll[i], f0)
        g = grad[4 * i:4 * i + 4]
        assert np.all(np.abs(g - g0) <= 1e-6 * np.abs(g0) + 1e-9 * np.abs(g0).max()), (i, g, g0)
