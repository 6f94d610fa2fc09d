"""Pins of the oracle's Metropolis pair-exchange sampler (MCMC with P ~ |Psi|^2, scaling
section of arXiv:2011.12453): Philox4x64-10 against numpy's implementation, S_z
conservation, exact stationarity and detailed balance of the transition matrix, and a
chi-squared check of the actual chains against |Psi|^2."""
import numpy as np
import pytest

from oracle import gcn, heisenberg as hz, sampler
from paper_2011_12453_gb300 import workloads as W


@pytest.mark.parametrize("key,ctr", [((1, 2), 1), ((0, 0), 1), ((2**64 - 1, 12345), 77),
                                     ((987654321, 2**40 + 3), 2**63 + 5)])
def test_philox_matches_numpy(key, ctr):
    # numpy's Philox increments its counter before producing a block, so the block for
    # counter t is the first output of a generator started at counter t - 1.
    g = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array([ctr - 1, 0, 0, 0], dtype=np.uint64))
    want = [int(x) for x in g.random_raw(4)]
    assert list(sampler.philox4x64_10(key, (ctr, 0, 0, 0))) == want


def test_philox_full_counter_words():
    # all four counter words enter the block
    g = np.random.Philox(key=[5, 6], counter=[10, 20, 30, 40])
    want = [int(x) for x in g.random_raw(4)]
    assert list(sampler.philox4x64_10((5, 6), (11, 20, 30, 40))) == want


def test_bond_index_and_uniform_edges():
    assert sampler.bond_index(0, 24) == 0
    assert sampler.bond_index(2**64 - 1, 24) == 23
    assert sampler.bond_index(2**63, 24) == 12
    assert sampler.uniform(0) == 0.0
    assert sampler.uniform(2**64 - 1) == 1.0 - 2.0**-53
    assert sampler.uniform(2**64 - 1, "fp32") == np.float32(1.0 - 2.0**-24)
    assert sampler.accept(0.999, 0.0) and not sampler.accept(0.5, np.log(0.5) / 2 - 1e-9)


def _model(g, F=4, L=2, scale=1.0, seed=1):
    th = W.random_theta(F, L, seed=seed, scale=scale)
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    return lambda s: gcn.logpsi_complex(th, F, L, Ah, s)


def test_sz_conserved_and_records():
    g = W.kagome(2)
    lp_fn = _model(g)
    s0 = W.random_spins(g.n_sites, 6, seed=3)
    s, samples, slp, acc, trace = sampler.run_chains(lp_fn, g.edges, s0, seed=7, step0=0, n_sweeps=4)
    assert samples.shape == (4, 6, g.n_sites)
    assert np.all((samples > 0).sum(axis=2) == g.n_sites // 2)
    np.testing.assert_allclose(slp[-1], lp_fn(s), atol=1e-13)
    assert acc.sum() == trace[:, :, 1].sum()
    # parallel bonds never move the chain and carry NaN deltas
    par = np.isnan(trace[:, :, 2])
    assert np.all(trace[:, :, 1][par] == 0)


@pytest.mark.parametrize("graph", ["ring6", "er7", "kagome_like"])
def test_exact_stationarity_and_detailed_balance(graph):
    if graph == "ring6":
        g = W.ring(6)
    elif graph == "er7":
        g = W.erdos_renyi(8, 0.45, seed=5)
    else:
        g = W.complete_bipartite(3, 3)
    lp_fn = _model(g, scale=1.5, seed=2)
    codes = hz.sector_codes(g.n_sites, g.n_sites // 2)
    s = hz.codes_to_spins(codes, g.n_sites)
    lp = lp_fn(s)
    T = sampler.transition_matrix(lp, codes, g.edges)
    np.testing.assert_allclose(T.sum(axis=1), 1.0, atol=1e-14)
    pi = np.exp(2 * (lp.real - lp.real.max()))
    pi /= pi.sum()
    np.testing.assert_allclose(pi @ T, pi, atol=1e-13)
    F = pi[:, None] * T
    np.testing.assert_allclose(F, F.T, atol=1e-14)


def test_chain_histogram_matches_psi_squared():
    g = W.ring(4)
    lp_fn = _model(g, F=3, L=1, scale=2.0, seed=4)
    codes = hz.sector_codes(4, 2)
    s_all = hz.codes_to_spins(codes, 4)
    lp = lp_fn(s_all)
    pi = np.exp(2 * (lp.real - lp.real.max()))
    pi /= pi.sum()
    C = 64
    s0 = W.random_spins(4, C, seed=0)
    _, samples, _, _, _ = sampler.run_chains(lp_fn, g.edges, s0, seed=11, step0=0, n_sweeps=60)
    x = samples[10:].reshape(-1, 4)  # drop 10 sweeps of burn-in
    counts = np.array([(hz.spins_to_codes(x) == c).sum() for c in codes])
    n = counts.sum()
    chi2 = ((counts - n * pi) ** 2 / (n * pi)).sum()
    # correlated samples inflate the statistic; 6 states -> 5 dof; generous bound
    assert chi2 < 60.0, (chi2, counts, n * pi)
