"""Pins of the oracle's HODLR construction (Alg. 1, Sec. 3.2.2) and its derivative (Alg. 2, Sec. 3.3)."""
import numpy as np
import pytest

from oracle import hodlr
from oracle.physics import Model
from oracle.tree import Tree

THETA = (1.0, 0.1, 5.0, 1e-4)
PARAMS = ("sigma2", "ell", "kappa", "tau2")


def _setup(dim=1, G=256, nvar=1, nu=1.5, leaf=32):
    return Model(dim, G, nvar, nu), Tree(dim, G, nvar, leaf)


def _dense_tree(m, t, theta, which="K"):
    return m.dense_K(theta, which)[np.ix_(t.perm, t.perm)]


def test_full_range_sketch_reproduces_K():
    # Alg. 1 with a probe block as wide as every off-diagonal block: B^ = Q Q^T B = B,
    # so K~ = K (up to rounding and the guard, which drops only rounding-level columns).
    m, t = _setup(2, 8, 1, 0.5, leaf=16)              # N = 64, blocks of 32 and 16 rows
    H = hodlr.build(m, t, THETA, c=32, cap=32, guard=1e-13, seed=3)
    K = _dense_tree(m, t, THETA)
    assert np.abs(H.densify() - K).max() <= 1e-10 * np.abs(K).max()


def test_1d_semiseparable_rank4_exact():
    # In 1-D, A^{-1} has rank-1 and the Matern-3/2 matrix rank-2 off-diagonal blocks, so K's
    # off-diagonal blocks have rank <= 4 and 8 probe columns recover K to rounding level.
    m, t = _setup(1, 256, 1, 1.5, leaf=32)
    H = hodlr.build(m, t, THETA, c=8, cap=8, guard=1e-13, seed=1)
    assert max(max(r) for r in H.ranks()) <= 4
    K = _dense_tree(m, t, THETA)
    assert np.abs(H.densify() - K).max() <= 1e-11 * np.abs(K).max()
    for p in PARAMS:
        Kj = _dense_tree(m, t, THETA, p)
        assert np.abs(H.densify(p) - Kj).max() <= 1e-8 * np.abs(Kj).max(), p


def test_symmetric_and_spd():
    m, t = _setup(2, 8, 2, 1.5, leaf=16)
    H = hodlr.build(m, t, THETA, c=24, cap=24, seed=2)
    for which in PARAMS[:3]:
        D = H.densify(which)
        assert np.array_equal(D, D.T)
    K = H.densify()
    assert np.linalg.eigvalsh(K).min() > 0


def test_low_rank_error_near_optimal():
    # Alg. 1 error is close to sigma_{k+1}(B) (Sec. 3.2.1); level-1 block, rank 3.
    m, t = _setup(2, 8, 1, 0.5, leaf=16)
    H = hodlr.build(m, t, THETA, c=3, cap=3, seed=5)
    (a1, b1), (a2, b2) = t.pairs(1)[0]
    K = _dense_tree(m, t, THETA)
    B = K[a1:b1, a2:b2]
    Bh = H.levels[0].Q[0] @ H.levels[0].Bt[0].T
    s = np.linalg.svd(B, compute_uv=False)
    err = np.linalg.norm(B - Bh, 2)
    assert s[3] <= err <= 30.0 * s[3]


@pytest.mark.parametrize("case", [(1, 128, 1, 1.5, 16, 6), (2, 8, 1, 0.5, 8, 5), (2, 6, 2, 1.5, 18, 7)])
def test_derivatives_match_central_differences(case):
    # Sec. 3.3: with probes and pivots fixed the construction is differentiable and
    # K~_j is the exact derivative of the approximation.
    dim, G, nvar, nu, leaf, c = case
    m, t = _setup(dim, G, nvar, nu, leaf)
    H = hodlr.build(m, t, THETA, c=c, cap=c, seed=7)
    J = H.pivots()
    for j, p in enumerate(PARAMS):
        h = 1e-5 * THETA[j]
        tp = list(THETA); tm = list(THETA)
        tp[j] += h; tm[j] -= h
        Hp = hodlr.build(m, t, tp, c=c, cap=c, seed=7, frozen=J, params=())
        Hm = hodlr.build(m, t, tm, c=c, cap=c, seed=7, frozen=J, params=())
        fd = (Hp.densify() - Hm.densify()) / (2 * h)
        an = H.densify(p)
        assert np.abs(fd - an).max() <= 1e-6 * np.abs(an).max(), p


def test_sigma2_general_sweep_equals_identity():
    # dK~/dsigma2 = (K~ - tau2 I)/sigma2: the general sweep gives dQ = 0 and the identity.
    m, t = _setup(1, 128, 1, 1.5, 16)
    th = (1.7, 0.1, 5.0, 3e-3)
    H = hodlr.build(m, t, th, c=6, cap=6, seed=4, params=("sigma2",))
    gen = H.densify("sigma2")
    ident = (H.densify("K") - th[3] * np.eye(t.N)) / th[0]
    assert np.abs(gen - ident).max() <= 1e-12 * np.abs(ident).max()
    for dQs, _ in H.dlevels["sigma2"]:
        for dQ in dQs:
            assert np.abs(dQ).max() <= 1e-8


def test_apply_count():
    # O(k tau) K-vector products (Sec. 3.2.2 / Sec. 3.3): per level (1+2)c + (1+4)w, leaves 3 n_l.
    m, t = _setup(1, 256, 1, 1.5, 32)
    H = hodlr.build(m, t, THETA, c=8, cap=8, seed=1)
    assert H.napply == hodlr.napply_formula(H, 8)
    w = [L.width for L in H.levels]
    assert H.napply == sum(3 * 8 + 5 * x for x in w) + 3 * 32


def test_adaptive_tolerance_monotone():
    m, t = _setup(2, 8, 1, 0.5, 8)
    r_loose = sum(map(sum, hodlr.build(m, t, THETA, c=12, cap=12, tol=1e-2, params=()).ranks()))
    r_tight = sum(map(sum, hodlr.build(m, t, THETA, c=12, cap=12, tol=1e-6, params=()).ranks()))
    r_cap = max(map(max, hodlr.build(m, t, THETA, c=12, cap=3, tol=1e-6, params=()).ranks()))
    assert r_loose < r_tight and r_cap == 3
