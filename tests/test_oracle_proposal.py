"""Pins of the oracle's learned exchange proposal (not part of the paper; a Metropolis-
Hastings proposal for its MCMC step): exact stationarity and detailed balance with the
mixture proposal density, the proposal density summing to one against the sampling
procedure, features by hand, the network's hand-written gradient against finite
differences, and the first Adam step in closed form."""
import numpy as np
import pytest

from oracle import gcn, heisenberg as hz, proposal as P
from paper_2011_12453_gb300 import workloads as W


def _model(g, scale=1.5, seed=2):
    F, L = 4, 2
    th = W.random_theta(F, L, seed=seed, scale=scale)
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    return lambda s: gcn.logpsi_complex(th, F, L, Ah, np.atleast_2d(s))


def test_param_count():
    assert P.N_PARAMS == W.proposal_num_params() == 4865


def test_features_by_hand():
    # path 0-1-2-3 plus 1-3 ; spins + - + -
    g = W.Graph(4, np.array([[0, 1], [1, 2], [2, 3], [1, 3]], dtype=np.int32), np.array([1.0, 0.7, 1.2, 0.9]))
    top = P.Topology(4, g.edges, g.J)
    s = np.array([1, -1, 1, -1])
    # pair (i=1, j=2): d_1 = 3 (0, 2, 3), d_2 = 2 (1, 3); n1(1) = s0+s2+s3 = 1, n1(2) = s1+s3 = -2
    # a_1 = (n1(1) - s_2)/(3-1) = 0, a_2 = (n1(2) - s_1)/(2-1) = -1
    # b_1 = mean over u in {0, 3} of n1(u)/d_u: n1(0) = -1 (d 1), n1(3) = s2+s1 = 0 (d 2) -> -0.5
    # b_2 = mean over u in {3}: n1(3)/d_3 = 0
    phi = P.features(top, s, 1, 2)
    np.testing.assert_allclose(phi, [-1, 1, 0.7, 1 / 3, 1 / 2, 0.0, -1.0, -0.5, 0.0], atol=1e-15)


def test_network_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    params = W.random_proposal_params(1, scale=0.5)
    phi = rng.normal(size=(13, P.D_IN))
    tgt = -np.abs(rng.normal(size=13))
    loss, grad = P.loss_and_grad(params, phi, tgt)
    h = 1e-6
    idx = rng.choice(params.size, 120, replace=False)
    idx = np.concatenate([idx, [params.size - 1, params.size - 2, 0]])
    for k in idx:
        e = np.zeros_like(params)
        e[k] = h
        fd = (P.loss_and_grad(params + e, phi, tgt)[0] - P.loss_and_grad(params - e, phi, tgt)[0]) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-7 + 1e-6 * abs(fd), (k, fd, grad[k])


def test_adam_first_step_is_signed_learning_rate():
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    p, m, v = P.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    np.testing.assert_allclose(p[:3], -0.01 * np.sign(g[:3]), rtol=1e-4)
    assert p[3] == 0.0


@pytest.mark.parametrize("graph", ["ring6", "k33", "er8"])
def test_proposal_density_sums_to_one(graph):
    g = {"ring6": W.ring(6), "k33": W.complete_bipartite(3, 3), "er8": W.erdos_renyi(8, 0.4, seed=4)}[graph]
    top = P.Topology(g.n_sites, g.edges, g.J)
    params = W.random_proposal_params(3, scale=1.0)
    eps = 0.1
    for s in W.random_spins(g.n_sites, 5, seed=1):
        total = 0.0
        for i, j in g.edges.tolist():
            if s[i] != s[j]:
                total += P.q_mix(top, params, s, i, j, eps)
        par = sum(1 for i, j in g.edges.tolist() if s[i] == s[j])
        lonely = sum(1 for i in range(g.n_sites) if not P.candidates(top, s, i))
        none = eps * par / g.n_edges + (1 - eps) * lonely / g.n_sites
        assert abs(total + none - 1.0) < 1e-13


@pytest.mark.parametrize("graph", ["ring6", "k33", "er8"])
def test_exact_stationarity_with_learned_proposal(graph):
    g = {"ring6": W.ring(6), "k33": W.complete_bipartite(3, 3), "er8": W.erdos_renyi(8, 0.4, seed=4)}[graph]
    top = P.Topology(g.n_sites, g.edges, g.J)
    params = W.random_proposal_params(5, scale=1.5)
    lp_fn = _model(g)
    codes = hz.sector_codes(g.n_sites, g.n_sites // 2)
    s = hz.codes_to_spins(codes, g.n_sites)
    lp = lp_fn(s)
    T = P.transition_matrix(lp, codes, top, params, eps=0.1)
    np.testing.assert_allclose(T.sum(axis=1), 1.0, atol=1e-13)
    assert T.min() >= -1e-15
    pi = np.exp(2 * (lp.real - lp.real.max()))
    pi /= pi.sum()
    np.testing.assert_allclose(pi @ T, pi, atol=1e-13)
    Fl = pi[:, None] * T
    np.testing.assert_allclose(Fl, Fl.T, atol=1e-14)


def test_learned_chain_matches_exact_transition_matrix():
    # independent chains started from known states: after k steps the state is
    # distributed as (initial distribution) T^k exactly, whatever the mixing time
    g = W.ring(6)
    top = P.Topology(g.n_sites, g.edges, g.J)
    params = W.random_proposal_params(7, scale=1.0)
    lp_fn = _model(g, scale=1.0, seed=4)
    codes = hz.sector_codes(6, 3)
    lp = lp_fn(hz.codes_to_spins(codes, 6))
    T = P.transition_matrix(lp, codes, top, params, eps=0.2)
    s0 = W.random_spins(6, 1500, seed=0)
    out, _, _ = P.run_chains(lp_fn, top, params, s0, seed=9, step0=0, n_sweeps=2, eps=0.2)
    T12 = np.linalg.matrix_power(T, 12)
    start = np.zeros(len(codes))
    for c in hz.spins_to_codes(s0):
        start[np.searchsorted(codes, c)] += 1
    want = start @ T12
    got = np.array([(hz.spins_to_codes(out) == c).sum() for c in codes])
    chi2 = ((got - want) ** 2 / want).sum()
    assert chi2 < 50.0, chi2  # 19 degrees of freedom: p < 1e-4 beyond this


def test_training_rows_cover_both_orientations():
    g = W.kagome(2)
    top = P.Topology(g.n_sites, g.edges, g.J)
    s = W.random_spins(g.n_sites, 3, seed=2)
    dl = np.random.default_rng(1).normal(size=(3, g.n_edges))
    phi, tgt = P.training_rows(top, s, dl)
    anti = (s[:, g.edges[:, 0]] != s[:, g.edges[:, 1]])
    assert phi.shape == (2 * anti.sum(), 9)
    want = np.repeat(np.minimum(0.0, 2 * dl[anti]), 2)
    np.testing.assert_allclose(tgt, want)
