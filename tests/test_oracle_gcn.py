"""Pins of the oracle's GCN log Psi against closed forms, invariants and an independent
loop formulation (Eq. gcn and the readout of the GNA section, arXiv:2011.12453)."""
import numpy as np
import pytest

from oracle import gcn
from paper_2011_12453_gb300 import workloads as W


@pytest.mark.parametrize("F,expected", [(16, 614), (32, 2246), (48, 4902), (64, 8582)])
def test_param_count_shared(F, expected):
    # embedding 2F+F, one shared layer 2F*F+F, readout (F+2)*2+2
    assert gcn.num_params(F, 4, True) == expected == W.num_params(F, 4, True)


def test_onehot_convention():
    oh = gcn.onehot(np.array([1, -1], dtype=np.int8))
    assert oh.tolist() == [[1.0, 0.0], [0.0, 1.0]]


@pytest.mark.parametrize("shared", [True, False])
@pytest.mark.parametrize("graph", ["kagome", "er", "star"])
def test_dense_matches_loops(graph, shared):
    if graph == "kagome":
        g = W.kagome(2)
    elif graph == "er":
        g = W.erdos_renyi(9, 0.35, seed=3)
    else:
        g = W.Graph(6, np.array([[0, k] for k in range(1, 5)], dtype=np.int32), np.ones(4))  # site 5 isolated
    F, L = 3, 3
    th = W.random_theta(F, L, seed=5, scale=0.7, shared=shared)
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    s = W.random_spins(g.n_sites, 5, seed=7)
    dense = gcn.logpsi(th, F, L, Ah, s, shared)
    loops = np.array([gcn.logpsi_loops(th, F, L, g.n_sites, g.edges, x, shared) for x in s])
    np.testing.assert_allclose(dense, loops, rtol=0, atol=1e-12)


def test_permutation_equivariance():
    g = W.erdos_renyi(10, 0.4, seed=11)
    F, L = 4, 3
    th = W.random_theta(F, L, seed=1, scale=0.8)
    s = W.random_spins(g.n_sites, 6, seed=2)
    perm = np.random.default_rng(0).permutation(g.n_sites)  # new label of old site v is perm[v]
    e2 = perm[g.edges]
    s2 = np.empty_like(s)
    s2[:, perm] = s
    A1 = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    A2 = gcn.norm_adjacency(gcn.adjacency(g.n_sites, e2))
    np.testing.assert_allclose(gcn.logpsi(th, F, L, A1, s), gcn.logpsi(th, F, L, A2, s2), atol=1e-12)


def test_L0_closed_form():
    # With no GCN layer: log Psi = sum_v tanh(W_e[c_v] + b_e) . w_r[:F] + (n_up, n_dn) . w_r[F:] + b_r
    g = W.kagome(2)
    F = 5
    th = W.random_theta(F, 0, seed=4, scale=0.9)
    p = gcn.unpack(th, F, 0)
    s = W.random_spins(g.n_sites, 3, seed=9, n_up=5)
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    got = gcn.logpsi(th, F, 0, Ah, s)
    for b in range(3):
        up = (s[b] > 0).sum()
        dn = g.n_sites - up
        h_up = np.tanh(p["W_e"][0] + p["b_e"])
        h_dn = np.tanh(p["W_e"][1] + p["b_e"])
        want = (up * h_up + dn * h_dn) @ p["w_r"][:F] + up * p["w_r"][F] + dn * p["w_r"][F + 1] + p["b_r"]
        np.testing.assert_allclose(got[b], want, atol=1e-13)


def test_single_site_closed_form():
    # A 1-site, 0-bond graph has D^-1/2 A D^-1/2 = 0: each layer is tanh(H W[F:2F] + b).
    F, L = 3, 2
    th = W.random_theta(F, L, seed=8, scale=0.9)
    p = gcn.unpack(th, F, L)
    Ah = np.zeros((1, 1))
    for spin, c in [(1, 0), (-1, 1)]:
        h = np.tanh(p["W_e"][c] + p["b_e"])
        for _ in range(L):
            h = np.tanh(h @ p["W"][0][F:] + p["b"][0])
        want = h @ p["w_r"][:F] + p["w_r"][F + c] + p["b_r"]
        got = gcn.logpsi(th, F, L, Ah, np.array([[spin]], dtype=np.int8))[0]
        np.testing.assert_allclose(got, want, atol=1e-14)


def test_two_site_scalar_by_hand():
    # F = 1, L = 1, two sites joined by one bond (degrees 1, so the normalised weight is 1).
    F, L = 1, 1
    we_up, we_dn, be, w_msg, w_self, b, wr0, wr_up, wr_dn, br = 0.3, -0.7, 0.1, 0.9, -0.4, 0.05, 1.3, 0.2, -0.6, 0.0
    # layout: W_e(2x1) b_e(1) W(2x1) b(1) w_r(3x2) b_r(2); only the Re column is exercised
    th = np.array([we_up, we_dn, be, w_msg, w_self, b, wr0, 0.0, wr_up, 0.0, wr_dn, 0.0, br, 0.0])
    Ah = gcn.norm_adjacency(gcn.adjacency(2, np.array([[0, 1]])))
    h_up, h_dn = np.tanh(we_up + be), np.tanh(we_dn + be)
    h1_0 = np.tanh(w_msg * h_dn + w_self * h_up + b)  # site 0 up, neighbour down
    h1_1 = np.tanh(w_msg * h_up + w_self * h_dn + b)
    want = (h1_0 + h1_1) * wr0 + wr_up + wr_dn + br
    got = gcn.logpsi(th, F, L, Ah, np.array([[1, -1]], dtype=np.int8))[0]
    assert abs(got[0] - want) < 1e-15 and got[1] == 0.0


def test_degree_normalisation_star_and_isolated():
    # star: centre 0 of degree 3, leaves of degree 1 -> weight 1/sqrt(3); site 4 isolated.
    A = gcn.adjacency(5, np.array([[0, 1], [0, 2], [0, 3]]))
    Ah = gcn.norm_adjacency(A)
    assert np.allclose(Ah[0, 1:4], 1 / np.sqrt(3)) and np.allclose(Ah[1:4, 0], 1 / np.sqrt(3))
    assert np.all(Ah[4] == 0) and np.all(Ah[:, 4] == 0)
    assert np.allclose(Ah, Ah.T)


def test_adjacency_rejects_bad_graphs():
    with pytest.raises(ValueError):
        gcn.adjacency(3, np.array([[0, 0]]))
    with pytest.raises(ValueError):
        gcn.adjacency(3, np.array([[0, 1], [1, 0]]))
