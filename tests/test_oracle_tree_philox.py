"""Pins of the oracle's ordering / cluster tree (Sec. 5.2, Sec. 3.2.2) and probes (Alg. 1)."""
import os

import numpy as np
import pytest

from oracle import philox
from oracle.tree import Tree, n_levels, spatial_order

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_morton_4x4_hand_listed():
    rows = np.loadtxt(os.path.join(GOLD, "morton_4x4.txt"), dtype=np.int64)
    assert np.array_equal(spatial_order(2, 4), rows[:, 3])
    assert np.array_equal(rows[:, 3], rows[:, 2] * 4 + rows[:, 1])


def test_morton_is_kd_tree_alternating_y_then_x():
    G = 8
    order = spatial_order(2, G)
    iy, ix = np.divmod(order, G)
    # depth 1 splits y, depth 2 splits x, depth 3 splits y ... (median splits)
    assert np.all(iy[:32] < 4) and np.all(iy[32:] >= 4)
    for q in range(2):
        blk = slice(32 * q, 32 * q + 32)
        assert np.all(ix[blk][:16] < 4) and np.all(ix[blk][16:] >= 4)
    # every node at every depth is an axis-aligned rectangle of the grid
    for d in range(7):
        n = 64 >> d
        for b in range(1 << d):
            sx, sy = ix[b * n:(b + 1) * n], iy[b * n:(b + 1) * n]
            assert (sx.max() - sx.min() + 1) * (sy.max() - sy.min() + 1) == n


@pytest.mark.parametrize("Ns,leaf,tau", [(1024, 64, 4), (65536, 128, 9), (512 * 512, 256, 10),
                                         (1024 * 1024, 256, 12), (1000, 64, 4), (64, 64, 0)])
def test_levels(Ns, leaf, tau):
    assert n_levels(Ns, leaf) == tau


def test_tree_uneven_and_bivariate():
    t = Tree(1, 1000, 1, 64)
    assert t.tau == 4
    sizes = [hi - lo for lo, hi in t.leaves()]
    assert max(sizes) - min(sizes) <= 1 and sum(sizes) == 1000
    assert np.array_equal(np.sort(t.perm), np.arange(1000))
    tb = Tree(2, 8, 2, 16)                # 64 points, 8-point spatial leaves, 2 variables
    assert tb.N == 128 and tb.tau == 3
    assert np.array_equal(np.sort(tb.perm), np.arange(128))
    sp = spatial_order(2, 8)
    for b, (lo, hi) in enumerate(tb.leaves()):
        assert hi - lo == 16
        assert np.array_equal(tb.perm[lo:lo + 8], sp[8 * b:8 * b + 8])
        assert np.array_equal(tb.perm[lo + 8:hi], 64 + sp[8 * b:8 * b + 8])
    # pairs of level l are the two children of every depth-(l-1) node
    for l in range(1, tb.tau + 1):
        for (a1, b1), (a2, b2) in tb.pairs(l):
            assert b1 == a2 and (b1 - a1) == (b2 - a2)


def test_philox_known_answers():
    with open(os.path.join(GOLD, "philox4x32_10_kat.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox.philox4x32_10(v[0], v[1], v[2], v[3], v[4], v[5])
        assert [int(o) for o in out] == v[6:10]


def test_normal_deviates_at_known_answer_counters():
    """Deviates worked out by hand from the published Random123 output words: a wrong shift,
    offset or branch in the 53-bit uniforms or the Box-Muller step changes them."""
    with open(os.path.join(GOLD, "philox_normal_kat.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        c0, c1, c2, c3, k0, k1 = (int(x, 16) for x in r[:6])
        a, b, z = int(r[6]), int(r[7]), float(r[8])
        assert 0 < a <= 2 ** 53 and 0 <= b < 2 ** 53
        got = philox.normal(np.array([c0], dtype=np.uint64), c1, c2, c3, k0 + (k1 << 32))
        assert abs(float(got[0]) - z) <= 1e-14 * max(1.0, abs(z)), (r, got)


def test_normals_moments_and_counter_purity():
    rows = np.arange(200000, dtype=np.uint64)
    z = philox.normal(rows, 3, 2, 0, 12345)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.01
    assert abs(np.mean(z ** 4) - 3.0) < 0.05
    # a value depends only on its counter
    z2 = philox.normal(rows[::7], 3, 2, 0, 12345)
    assert np.array_equal(z[::7], z2)
    assert not np.array_equal(z[:100], philox.normal(rows[:100], 4, 2, 0, 12345))


def test_level_probe_pattern():
    t = Tree(1, 256, 1, 32)
    for l in range(1, t.tau + 1):
        R = philox.level_probe(t, l, 5, seed=1)
        for (a1, b1), (a2, b2) in t.pairs(l):
            assert np.all(R[a1:b1] == 0.0)
            assert np.all(R[a2:b2] != 0.0)
