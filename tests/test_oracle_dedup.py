"""Pins of the oracle's grouping of duplicated samples (oracle/dedup.py) against numpy's
row-unique routine, brute-force counting, and the ISGO invariance it exists for."""
import numpy as np

from oracle import dedup, gcn, isgo
from paper_2011_12453_gb300 import workloads as W


def test_matches_numpy_unique_in_first_occurrence_order():
    rng = np.random.default_rng(0)
    base = W.random_spins(10, 30, seed=1)
    s = base[rng.integers(0, 30, size=500)]
    lp = rng.normal(size=(500, 2))
    u, lu, c = dedup.group(s, lp)
    vals, first, cnt = np.unique(s, axis=0, return_index=True, return_counts=True)
    order = np.argsort(first)
    assert np.array_equal(u, vals[order])
    assert np.array_equal(c, cnt[order].astype(float))
    assert np.array_equal(lu, lp[np.sort(first)])


def test_brute_force_counts_and_coverage():
    s = np.array([[1, -1, 1, -1], [-1, 1, 1, -1], [1, -1, 1, -1], [1, -1, 1, -1], [-1, 1, 1, -1], [1, 1, -1, -1]],
                 dtype=np.int8)
    u, lu, c = dedup.group(s, np.arange(6.0))
    assert u.tolist() == [[1, -1, 1, -1], [-1, 1, 1, -1], [1, 1, -1, -1]]
    assert c.tolist() == [3.0, 2.0, 1.0]
    assert lu.tolist() == [0.0, 1.0, 5.0]
    assert c.sum() == len(s)


def test_empty_and_single():
    u, lu, c = dedup.group(np.zeros((0, 5), np.int8), np.zeros((0, 2)))
    assert u.shape == (0, 5) and c.shape == (0,)
    u, lu, c = dedup.group(np.ones((1, 3), np.int8), np.ones((1, 2)))
    assert c.tolist() == [1.0]


def test_isgo_gradient_is_unchanged_by_grouping():
    g = W.kagome(2)
    F, L = 4, 2
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    th0 = W.random_theta(F, L, seed=3, scale=0.5)
    th = th0 + W.random_theta(F, L, seed=4, scale=0.05)
    rng = np.random.default_rng(5)
    s = W.random_spins(g.n_sites, 12, seed=6)[rng.integers(0, 12, size=60)]
    lp0 = gcn.logpsi_complex(th0, F, L, Ah, s)
    u, lu, c = dedup.group(s, lp0)
    a = isgo.isgo_gradient(th, F, L, Ah, g.edges, g.J, u, lu, c)
    b = isgo.isgo_gradient(th, F, L, Ah, g.edges, g.J, s, lp0)
    np.testing.assert_allclose(a[0], b[0], rtol=1e-10, atol=1e-12)
    assert abs(a[1] - b[1]) < 1e-12
