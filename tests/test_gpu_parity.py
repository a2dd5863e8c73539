"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Every case uses the same seeded inputs on both sides.  Tolerances:
  * integer / index work (tree order, ranks, pivots, apply counts): bit-exact;
  * FP64 path: physics products 1e-11, densified K~ 1e-10, NLL 1e-10, gradient and Fisher
    1e-9 (relative to the largest entry), log-det 1e-11;
  * FP32 (mixed) path, univariate: NLL 1e-6, gradient 1e-3, Fisher 1e-4 -- Alg. 2 amplifies
    the FP32 rounding of the sketch by cond(R) <= 1/guard = 1e5 (measured gradient errors
    2.5e-5 to 1.4e-4); bivariate: NLL 1e-5, while score and Fisher are refused (ENOTIMPL);
  * FP32 physics products (tensor-core DST on 128^2 grids): 2e-5.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import hodlr as oh, likelihood as ol
from oracle.philox import level_probe
from oracle.physics import Model
from oracle.tree import Tree

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
PARAMS = ("sigma2", "ell", "kappa", "tau2")


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def ctx(w, prec=None):
    from paper_2303_10102_gb300 import Hodlr
    p = prec or w.precision
    return Hodlr(w.dim, w.G, w.nvar, w.nu, p, w.leaf, w.cap, w.c - w.cap, w.tol, w.seed_probe, device=DEV)


def oracle_build(w, prec, theta=None, frozen=None, params=("ell", "kappa")):
    m, t = Model(w.dim, w.G, w.nvar, w.nu), Tree(w.dim, w.G, w.nvar, w.leaf)
    H = oh.build(m, t, theta or w.theta, c=w.c, cap=w.cap, tol=w.tol, guard=synth.GUARD[prec], seed=w.seed_probe,
                 frozen=frozen, params=params)
    return m, t, H


NLL_TOL = {}
GRAD_TOL = {}

SMALL = {
    "1d-uni": synth.small_workload(dim=1, G=512, nvar=1, nu=1.5, theta=(1.0, 0.1, 5.0, 1e-3), leaf=32, cap=10, c=12),
    "1d-biv": synth.small_workload(dim=1, G=256, nvar=2, nu=0.5, theta=(1.3, 0.07, 8.0, 2e-3), leaf=32, cap=10, c=14),
    "2d-uni": synth.small_workload(dim=2, G=16, nvar=1, nu=0.5, theta=(1.0, 0.1, 8.0, 1e-3), leaf=16, cap=24, c=32,
                                   tol=1e-6),
    "2d-biv": synth.small_workload(dim=2, G=16, nvar=2, nu=1.5, theta=(1.0, 0.05, 10.0, 1e-3), leaf=32, cap=48,
                                   c=56),
    "1d-nonpow2": synth.small_workload(dim=1, G=320, nvar=1, nu=1.5, theta=(0.8, 0.2, 3.0, 1e-2), leaf=40,
                                                 cap=6, c=9),
    # leaves of 128: the blocked leaf Cholesky and the two-level block inversion of the factors
    "1d-leaf128": synth.small_workload(dim=1, G=2048, nvar=1, nu=1.5, theta=(1.0, 0.1, 5.0, 1e-3), leaf=128,
                                       cap=10, c=12),
    # uneven cluster trees (median splits of sizes that are not leaf x 2^tau): leaves of 62/63
    # points, bivariate leaves of 31/32 points per variable, and a 23^2 grid (leaves of 33/34)
    "1d-uneven": synth.small_workload(dim=1, G=1000, nvar=1, nu=1.5, theta=(1.0, 0.1, 5.0, 1e-3), leaf=64,
                                      cap=12, c=16),
    "1d-biv-uneven": synth.small_workload(dim=1, G=1001, nvar=2, nu=0.5, theta=(1.3, 0.07, 8.0, 2e-3), leaf=64,
                                          cap=10, c=14),
    "2d-uneven": synth.small_workload(dim=2, G=23, nvar=1, nu=0.5, theta=(1.0, 0.1, 8.0, 1e-3), leaf=64, cap=24,
                                      c=32, tol=1e-6),
}


@pytest.mark.parametrize("name", list(SMALL))
def test_tree_probe_and_physics(name):
    w = SMALL[name]
    h = ctx(w, "fp64")
    m, t = Model(w.dim, w.G, w.nvar, w.nu), Tree(w.dim, w.G, w.nvar, w.leaf)
    assert np.array_equal(h.perm(), t.perm)
    assert h.tau == t.tau and h.N == t.N
    for l in range(1, t.tau + 1):
        P = h.probe(l, w.c).cpu().numpy()
        Po = level_probe(t, l, w.c, w.seed_probe)
        assert np.array_equal(P != 0, Po != 0)
        assert rel(P, Po) < 1e-14
    X = np.random.default_rng(3).standard_normal((t.N, 5))
    for which in PARAMS + ("K",):
        Y = h.apply(w.theta, which, X).cpu().numpy()
        assert rel(Y, m.apply(X, w.theta, which)) < 1e-11, which


@pytest.mark.parametrize("name", ["1d-uni", "2d-uni", "2d-biv", "1d-uneven", "1d-long"])
def test_bf16_path_physics_products(name):
    """Physics products of the mixed BF16 path (FP64 fields; FFT butterflies in double-float,
    DST products as BF16 digit slices) against the FP64 oracle.  "1d-long" has a 16384-point
    embedding, which takes the four-step FFT passes."""
    w = SMALL[name] if name in SMALL else synth.small_workload(dim=1, G=8192, nvar=1, nu=1.5,
                                                               theta=(1.0, 0.1, 5.0, 1e-3), leaf=64, cap=12, c=12)
    h = ctx(w, "bf16")
    m = Model(w.dim, w.G, w.nvar, w.nu)
    X = np.random.default_rng(7).standard_normal((h.N, 5))
    for which in PARAMS + ("K",):
        Y = h.apply(w.theta, which, X).cpu().numpy()
        assert rel(Y, m.apply(X, w.theta, which)) < 1e-11, which


@pytest.mark.parametrize("nvar", [1, 2])
def test_fp32_physics_products_2d(nvar):
    """FP32 physics products on a 128 x 128 grid, where the DST products of the operator solve
    run on the tensor cores (3xTF32), against the FP64 oracle."""
    w = synth.small_workload(dim=2, G=128, nvar=nvar, nu=0.5, theta=(1.0, 0.1, 8.0, 1e-4), leaf=256, cap=16, c=16)
    h = ctx(w, "fp32")
    m = Model(w.dim, w.G, w.nvar, w.nu)
    X = np.random.default_rng(5).standard_normal((h.N, 24))
    for which in PARAMS + ("K",):
        Y = h.apply(w.theta, which, X).cpu().numpy()
        assert rel(Y, m.apply(X, w.theta, which)) < 2e-5, which


@pytest.mark.parametrize("name", list(SMALL))
def test_fp64_construction_matches_oracle(name):
    w = SMALL[name]
    m, t, H = oracle_build(w, "fp64")
    h = ctx(w, "fp64")
    h.build(w.theta)
    assert h.ranks() == H.ranks()
    piv = h.get_pivots().reshape(-1, w.c)
    k = 0
    for L in H.levels:
        for J in L.J:
            assert np.array_equal(piv[k, :J.size], J) and np.all(piv[k, J.size:] == -1)
            k += 1
    assert h.napply() == H.napply == oh.napply_formula(H, w.c)
    for which in ("K", "sigma2", "tau2"):
        assert rel(h.densify(which).cpu().numpy(), H.densify(which)) < 1e-10, which
    for which in ("ell", "kappa"):
        assert rel(h.densify(which).cpu().numpy(), H.densify(which)) < 1e-7, which
    # the HODLR product of the API (natural order) against the oracle's densified K~, K~_j
    X = np.random.default_rng(7).standard_normal((t.N, 5))
    for which in ("K", "sigma2", "tau2", "ell", "kappa"):
        ref = np.empty_like(X)
        ref[t.perm] = H.densify(which) @ X[t.perm]
        Y = h.matvec(X, which).cpu().numpy()
        assert rel(Y, ref) < (1e-7 if which in ("ell", "kappa") else 1e-10), which


@pytest.mark.parametrize("name", list(SMALL))
def test_fp64_likelihood_gradient_fisher(name):
    w = SMALL[name]
    m, t, H = oracle_build(w, "fp64")
    y = synth.simulate_y(w)
    h = ctx(w, "fp64")
    f, g, F = h.eval(w.theta, torch.as_tensor(y, device=DEV))
    f0, g0, F0 = ol.evaluate(H, t.to_tree(y))
    assert abs(f - f0) <= NLL_TOL.get(name, 1e-10) * abs(f0), (f, f0)
    assert rel(g, g0) < GRAD_TOL.get(name, 1e-9), (g, g0)
    assert rel(F, F0) < 1e-9
    assert np.allclose(F, F.T, rtol=0, atol=1e-12 * np.abs(F).max())
    # log-det, solve and the exact traces separately (App. B, App. C)
    K = H.densify()
    assert abs(h.logdet() - ol.logdet(K)) <= 1e-11 * abs(ol.logdet(K))
    x = h.solve(torch.as_tensor(y, device=DEV)).cpu().numpy()
    assert rel(x, t.to_natural(ol.solve(K, t.to_tree(y)))) < 1e-10
    tt, ff = h.traces()
    to, fo = ol.traces(K, [np.eye(t.N), H.densify("ell"), H.densify("kappa")])
    assert rel(tt, to) < 1e-10 and rel(ff, fo) < 1e-9


def test_c0_full_size_fp64():
    w = synth.workload("C0")
    m, t, H = oracle_build(w, "fp64")
    y = synth.simulate_y(w)
    h = ctx(w, "fp64")
    f, g, F = h.eval(w.theta, torch.as_tensor(y, device=DEV))
    assert h.ranks() == H.ranks()
    f0, g0, F0 = ol.evaluate(H, t.to_tree(y))
    assert abs(f - f0) <= 1e-10 * abs(f0)
    assert rel(g, g0) < 1e-9
    assert rel(F, F0) < 1e-9


@pytest.mark.parametrize("name", ["1d-uni", "2d-uni"])
def test_mixed_fp32_against_fp64_oracle(name):
    w = SMALL[name]
    m, t, H = oracle_build(w, "fp32")
    y = synth.simulate_y(w)
    h = ctx(w, "fp32")
    h.build(w.theta)
    # rank decisions are taken on FP32 data: freeze the oracle's pivots so that both sides
    # evaluate the same approximation, then compare values.
    h.set_pivots(h.pivots_from_sets(H.pivots()))
    f, g, F = h.eval(w.theta, torch.as_tensor(y, device=DEV))
    f0, g0, F0 = ol.evaluate(H, t.to_tree(y))
    # FP32 sketch rounding (6e-8) amplified by cond(R) <= 1/guard in Alg. 2's dY R^{-1}
    assert abs(f - f0) <= 1e-6 * abs(f0), (f, f0)
    assert rel(g, g0) < 1e-3, (g, g0)
    assert rel(F, F0) < 1e-4


def test_mixed_fp32_bivariate_likelihood_only():
    from paper_2303_10102_gb300 import HodlrError
    w = SMALL["2d-biv"]
    m, t, H = oracle_build(w, "fp32")
    y = torch.as_tensor(synth.simulate_y(w), device=DEV)
    h = ctx(w, "fp32")
    h.build(w.theta)
    h.set_pivots(h.pivots_from_sets(H.pivots()))
    f0, _, _ = ol.evaluate(H, t.to_tree(y.cpu().numpy()))
    assert abs(h.nll(w.theta, y) - f0) <= 1e-5 * abs(f0)
    for call in (lambda: h.grad(w.theta, y), lambda: h.fisher(w.theta), lambda: h.eval(w.theta, y)):
        with pytest.raises(HodlrError) as e:
            call()
        assert e.value.code == -6
    assert np.isfinite(h.nll(w.theta, y))      # the context stays usable


def test_mixed_fp32_own_rank_decisions_are_valid():
    w = SMALL["2d-uni"]
    m, t, H = oracle_build(w, "fp32")
    h = ctx(w, "fp32")
    h.build(w.theta)
    for rg, ro in zip(h.ranks(), H.ranks()):
        assert max(abs(a - b) for a, b in zip(rg, ro)) <= 2


def test_gradient_matches_central_differences_of_gpu_nll():
    w = SMALL["2d-uni"]
    y = torch.as_tensor(synth.simulate_y(w), device=DEV)
    h = ctx(w, "fp64")
    h.build(w.theta)
    h.set_pivots(h.get_pivots())
    _, g, _ = h.eval(w.theta, y)
    for j in range(4):
        step = 1e-5 * w.theta[j]
        tp, tm = list(w.theta), list(w.theta)
        tp[j] += step
        tm[j] -= step
        fd = (h.nll(tp, y) - h.nll(tm, y)) / (2 * step)
        assert abs(fd - g[j]) <= 1e-6 * np.abs(g).max(), (j, fd, g[j])


def test_error_paths():
    from paper_2303_10102_gb300 import HodlrError
    w = SMALL["1d-uni"]
    h = ctx(w, "fp64")
    with pytest.raises(HodlrError) as e:
        h.build((1.0, 0.1, 5.0, -1e-3))
    assert e.value.code == -1
    y = torch.as_tensor(synth.simulate_y(w), device=DEV)
    y[7] = float("nan")
    with pytest.raises(HodlrError) as e:
        h.nll(w.theta, y)
    assert e.value.code == -4
    # the context stays usable after a failure
    y[7] = 0.0
    assert np.isfinite(h.nll(w.theta, y))


@pytest.mark.parametrize("dim,G,nvar,leaf", [(2, 3, 1, 2), (2, 100, 1, 64), (2, 129, 2, 32), (2, 1000, 1, 256),
                                               (1, 40961, 1, 64), (1, 4097, 2, 128)])
def test_device_tree_order_uneven_grids(dim, G, nvar, leaf):
    """a1 on the device: the tree_order kernel's maps (read back by hodlr_perm) equal the oracle's
    sorted Morton order and halving tree bit for bit on grids whose side is not a power of two
    and trees whose leaves differ in size."""
    from paper_2303_10102_gb300 import Hodlr
    t = Tree(dim, G, nvar, leaf)
    h = Hodlr(dim, G, nvar, 1.5, "fp64", leaf, 2, 0, 0.0, 1, device=DEV)
    assert h.N == t.N and h.tau == t.tau
    assert np.array_equal(h.perm(), t.perm)


@pytest.mark.parametrize("name", ["C1", "C2", "C4"])
def test_full_size_tree_order_bit_exact(name):
    w = synth.workload(name)
    t = Tree(w.dim, w.G, w.nvar, w.leaf)
    from paper_2303_10102_gb300 import lib as plib
    import ctypes
    lib = plib.load()
    m = plib.Model(w.dim, (ctypes.c_int * 2)(w.G, w.G if w.dim == 2 else 1), w.nvar, w.nu, 1)
    o = plib.Opts(w.leaf, w.cap, w.c - w.cap, w.tol, 1, 0.0)
    # the context's tree order comes from the device kernel (closed-form Morton rank per point)
    nbytes = lib.hodlr_workspace_size(ctypes.byref(m), ctypes.byref(o))
    assert nbytes > 0
    h = ctx(w, "fp32")
    assert np.array_equal(h.perm(), t.perm)
    P = h.probe(1, 2).cpu().numpy()
    rows = np.random.default_rng(0).choice(t.N, 2000, replace=False)
    from oracle.philox import normal
    (_, _), (lo2, hi2) = t.pairs(1)[0]
    for j in range(2):
        ref = np.where((rows >= lo2) & (rows < hi2), normal(rows.astype(np.uint64), j, 1, 0, w.seed_probe), 0.0)
        assert rel(P[rows, j], ref) < 1e-6
    del h
    torch.cuda.empty_cache()


def test_full_size_physics_products_c2():
    """Physics products K X and dK/dtheta_j X (eq. cov model) at the bench's configuration (C2:
    512^2 grid, mixed path, FP32 fields with the tensor-core DST) on two seeded columns, against
    the FP64 oracle.  The FP32 rounding of the product (FFT embedding, DST products, Thomas
    recurrences, each about 1e-6) grows about sqrt(2) per grid doubling: measured 1.2e-5 at 128^2
    and 1.7e-5 at 256^2 for the kappa derivative (three solves), so about 2.5e-5 here; the bound
    keeps a factor 4."""
    w = synth.workload("C2")
    h = ctx(w, "fp32")
    m = Model(w.dim, w.G, w.nvar, w.nu)
    X = np.random.default_rng(11).standard_normal((h.N, 2))
    for which in PARAMS + ("K",):
        Y = h.apply(w.theta, which, X).cpu().numpy()
        assert rel(Y, m.apply(X, w.theta, which)) < 1e-4, which
    del h
    torch.cuda.empty_cache()

