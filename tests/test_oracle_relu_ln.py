"""Pins of the oracle's ReLU + layer-norm nonlinearity (the paper's f in the GNA section) and
of its reverse mode: the per-site loop formulation, a two-feature closed form worked by
hand, the row invariants of a layer norm, invariance under a positive rescaling of every
dense layer (ReLU is positively homogeneous, the layer norm removes the scale), permutation
equivariance, central finite differences of the hand-written backward, and the ISGO
gradient against the exact gradient of the enumerated variational energy of the paper's
hard-core bosons."""
import numpy as np
import pytest

from oracle import gcn, heisenberg as hz, isgo
from paper_2011_12453_gb300 import workloads as W

ACT = "relu_ln"


def _ah(g):
    return gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))


@pytest.mark.parametrize("shared", [True, False])
def test_dense_matches_loops(shared):
    g = W.erdos_renyi(11, 0.35, seed=4)
    F, L = 5, 3
    th = W.random_theta(F, L, seed=1, scale=0.7, shared=shared)
    s = W.random_spins(g.n_sites, 3, seed=2)
    dense = gcn.logpsi(th, F, L, _ah(g), s, shared, ACT)
    for b in range(3):
        np.testing.assert_allclose(dense[b], gcn.logpsi_loops(th, F, L, g.n_sites, g.edges, s[b], shared, ACT),
                                   rtol=1e-12, atol=1e-12)


def test_two_feature_closed_form_by_hand():
    # F = 2, L = 0: a row (a, b) with a > 0 > b becomes (a, 0) after ReLU, centred
    # (a/2, -a/2), variance a^2/4, so H = (a/2, -a/2)/sqrt(a^2/4 + eps).  Up site:
    # (a, b) = (0.9, -0.4) -> H = (h, -h), h = 0.45/sqrt(0.2025 + 1e-6); down site:
    # (0.0, 0.5): ReLU keeps it, centred (-0.25, 0.25) -> H = (-k, k), k = 0.25/sqrt(0.0625 + 1e-6).
    F = 2
    th = np.zeros(gcn.num_params(F, 0))
    th[0:4] = [1.0, -0.1, 0.1, 0.8]   # W_e rows (up, down)
    th[4:6] = [-0.1, -0.3]            # b_e
    o = 6 + 2 * F * F + F
    w_r = np.array([[0.7, 0.2], [-0.3, 0.5], [0.11, 0.0], [-0.05, 0.0]])
    th[o:o + 8] = w_r.ravel()
    th[o + 8:o + 10] = [0.01, -0.02]
    h = 0.45 / np.sqrt(0.2025 + 1e-6)
    k = 0.25 / np.sqrt(0.0625 + 1e-6)
    s = np.array([[1, -1, -1]], dtype=np.int8)
    g_edges = np.array([[0, 1], [1, 2]], dtype=np.int32)
    Ah = gcn.norm_adjacency(gcn.adjacency(3, g_edges))
    z = np.array([h - 2 * k, -h + 2 * k, 1.0, 2.0])
    want = z @ w_r + np.array([0.01, -0.02])
    np.testing.assert_allclose(gcn.logpsi(th, F, 0, Ah, s, True, ACT)[0], want, rtol=1e-14, atol=1e-14)


def test_layer_rows_are_normalised():
    # every row of every layer: mean 0 and mean square var/(var + eps) of its ReLU output
    g = W.kagome(2)
    F, L = 16, 3
    th = W.random_theta(F, L, seed=3, scale=0.5)
    p = gcn.unpack(th, F, L)
    s = W.random_spins(g.n_sites, 4, seed=5)
    Hs = gcn.layers(th, F, L, _ah(g), s, True, ACT)
    Ah = _ah(g)
    for l, H in enumerate(Hs):
        np.testing.assert_allclose(H.mean(axis=-1), 0.0, atol=1e-12)
        if l == 0:
            Y = gcn.onehot(s) @ p["W_e"] + p["b_e"]
        else:
            Hp = Hs[l - 1]
            Y = np.concatenate([np.einsum("vu,buf->bvf", Ah, Hp), Hp], -1) @ p["W"][l - 1] + p["b"][l - 1]
        r = np.maximum(Y, 0)
        var = r.var(axis=-1)
        np.testing.assert_allclose((H * H).mean(axis=-1), var / (var + gcn.LN_EPS), rtol=1e-12)
        assert np.all(H[Y <= 0] == H.min(axis=-1, keepdims=True).repeat(F, -1)[Y <= 0])


def test_positive_rescaling_of_dense_layers_is_invariant():
    # relu(alpha y) = alpha relu(y) and the layer norm removes alpha (up to eps): scaling
    # (W_e, b_e) and every (W, b) by alpha > 0 leaves log Psi unchanged
    g = W.triangular(3, 4)
    F, L = 8, 3
    th = W.random_theta(F, L, seed=6, scale=0.6, shared=False)
    s = W.random_spins(g.n_sites, 5, seed=7)
    ref = gcn.logpsi(th, F, L, _ah(g), s, False, ACT)
    o_r = gcn.num_params(F, L, False) - (F + 2) * 2 - 2
    for alpha in (3.0, 0.5):
        t2 = th.copy()
        t2[:o_r] *= alpha
        # eps moves each row by at most eps/(2 var) relative (var of a row's ReLU output ~ 1e-2 here)
        np.testing.assert_allclose(gcn.logpsi(t2, F, L, _ah(g), s, False, ACT), ref, rtol=1e-4)
    # tanh has no such invariance (a check that the test can fail)
    t2 = th.copy()
    t2[:o_r] *= 3.0
    assert np.abs(gcn.logpsi(t2, F, L, _ah(g), s, False) - gcn.logpsi(th, F, L, _ah(g), s, False)).max() > 1e-2


def test_permutation_equivariance():
    g = W.erdos_renyi(10, 0.4, seed=8)
    F, L = 4, 3
    th = W.random_theta(F, L, seed=9, scale=0.8)
    s = W.random_spins(g.n_sites, 3, seed=1)
    perm = np.random.default_rng(2).permutation(g.n_sites)
    inv = np.argsort(perm)
    e2 = inv[g.edges]
    s2 = s[:, perm]
    a = gcn.logpsi(th, F, L, _ah(g), s, True, ACT)
    b = gcn.logpsi(th, F, L, gcn.norm_adjacency(gcn.adjacency(g.n_sites, e2)), s2, True, ACT)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("shared", [True, False])
def test_backward_matches_central_differences(shared):
    g = W.erdos_renyi(9, 0.4, seed=1)
    F, L = 4, 3
    th = W.random_theta(F, L, seed=2, scale=0.6, shared=shared)
    Ah = _ah(g)
    s = W.random_spins(g.n_sites, 4, seed=3)
    cot = np.random.default_rng(4).normal(size=(4, 2))
    grad = isgo.backward(th, F, L, Ah, s, cot, shared, ACT)

    def f(t):
        return (gcn.logpsi(t, F, L, Ah, s, shared, ACT) * cot).sum()

    h = 1e-6
    fd = np.array([(f(th + h * e) - f(th - h * e)) / (2 * h) for e in np.eye(th.size)])
    np.testing.assert_allclose(grad, fd, rtol=1e-5, atol=1e-7)


def test_isgo_gradient_equals_exact_gradient_bosons():
    # the paper's model on its Kagome 2x2x3 setup: hard-core bosons at t/V = 0.5, half filling
    F, L = 3, 2
    g = W.kagome(2)
    Ah = _ah(g)
    xxz = hz.hardcore_bosons(g.edges.shape[0], 0.5, 1.0)
    Hs, codes = hz.sector_hamiltonian(g.n_sites, g.edges, None, xxz=xxz)
    s = hz.codes_to_spins(codes, g.n_sites)
    th0 = W.random_theta(F, L, seed=10, scale=0.8)
    th = th0 + W.random_theta(F, L, seed=11, scale=0.05)
    lp0 = gcn.logpsi_complex(th0, F, L, Ah, s, True, ACT)
    counts = np.exp(2 * (lp0.real - lp0.real.max()))
    grad, Ebar, *_ = isgo.isgo_gradient(th, F, L, Ah, g.edges, None, s, lp0, counts, xxz=xxz, act=ACT)

    def Ev(t):
        return hz.variational_energy(gcn.logpsi_complex(t, F, L, Ah, s, True, ACT), Hs).real

    assert abs(Ebar - Ev(th)) < 1e-12
    h = 1e-6
    fd = np.array([(Ev(th + h * e) - Ev(th - h * e)) / (2 * h) for e in np.eye(th.size)])
    np.testing.assert_allclose(grad, fd, rtol=0, atol=1e-7 * max(np.abs(fd).max(), 1e-3))
