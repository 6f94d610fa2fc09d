"""The tensor-core sampler (BF16 model, plain moves) at the benchmark's size and in the launch
configuration the benchmark times: Kagome 6x6x3, F = 32, L = 4, 16384 chains, one sweep,
parameters and spins from the benchmark's seeds (weight scale 0.1).

Checked on every chain: S_z is conserved and the acceptance counts equal the accepted steps
of the trace.  Checked on 256 chains drawn at random, replayed step by step with the
oracle's Philox4x64-10 words: every step's bond, the no-op on parallel bonds, the decision
u < exp(2 Re Delta) on the kernel's own Delta with the FP32 uniform (near-ties within 1e-6
skipped), and the final configuration.  Checked on 64 antiparallel proposals drawn from
those chains: Delta within 2e-3 of the FP64 oracle on the state it was made from (the BF16
tolerance of the small-size sampler test at the same weight scale)."""
import numpy as np
import pytest

from bounds import bf16_round
from oracle import gcn, heisenberg as hz, sampler
from paper_2011_12453_gb300 import build as B, gna, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t

    B.build()
    t.cuda.set_device(0)
    return t


def _replay_chain(g, s0, trc, seed, chain, step0):
    """States before each step of one chain, the final state and the near-tie count."""
    s = s0.copy()
    K = trc.shape[0]
    before = np.empty((K, g.n_sites), dtype=np.int8)
    near = 0
    for k in range(K):
        before[k] = s
        w = sampler.step_words(seed, chain, step0 + k)
        e = sampler.bond_index(w[0], g.n_edges)
        assert int(trc[k, 0]) == e, (chain, k)
        i, j = g.edges[e]
        if s[i] == s[j]:
            assert np.isnan(trc[k, 2]) and trc[k, 1] == 0, (chain, k)
            continue
        u = sampler.uniform(w[1], "fp32")
        if abs(float(u) - np.exp(2 * trc[k, 2])) < 1e-6:
            near += 1
        else:
            assert bool(trc[k, 1]) == sampler.accept(u, trc[k, 2], "fp32"), (chain, k)
        if trc[k, 1]:
            s[[i, j]] = s[[j, i]]
    return before, s, near


def test_bf16_sampler_at_benchmark_size(torch):
    g = W.kagome(6)
    F, L, C = 32, 4, 16384
    N = g.n_sites
    graph = gna.Graph.from_workload(g, L)
    model = gna.Model(F, L, gna.PREC_BF16)
    th = W.random_theta(F, L, 0)
    theta = torch.tensor(th, dtype=torch.float32, device="cuda")
    s0 = W.random_spins(N, C, 1)
    ch = torch.tensor(s0, device="cuda")
    seed, step0 = 7, 0
    gna.device_status(clear=True)  # the status word is sticky: start from a clean one
    _, _, acc, tr = gna.metropolis_sweep(graph, model, theta, ch, 1, 0, seed, step0, trace=True)
    assert gna.device_status(clear=True) == 0
    tr, final, acc = tr.cpu().numpy(), ch.cpu().numpy(), acc.cpu().numpy()
    assert tr.shape == (C, N, 4)
    assert np.all((final > 0).sum(axis=1) == N // 2)
    assert np.array_equal(acc, tr[:, :, 1].sum(axis=1).astype(acc.dtype))
    assert np.all(tr[:, :, 3] == 1.0)
    rng = np.random.default_rng(0)
    chains = rng.choice(C, size=256, replace=False)
    near, befores = 0, {}
    for c in chains:
        before, s_end, n_near = _replay_chain(g, s0[c], tr[c], seed, int(c), step0)
        near += n_near
        befores[int(c)] = before
        if n_near == 0:
            assert np.array_equal(s_end, final[c]), c
    assert near <= 4
    # Delta of sampled antiparallel proposals against the FP64 oracle
    cs, ks = [], []
    for c in chains:
        for k in np.nonzero(~np.isnan(tr[c, :, 2]))[0]:
            cs.append(int(c))
            ks.append(int(k))
    pick = rng.choice(len(cs), size=64, replace=False)
    states = np.stack([befores[cs[p]][ks[p]] for p in pick])
    Ah = gcn.norm_adjacency(gcn.adjacency(N, g.edges))
    # the model's parameters as the kernel holds them: float32, W a BF16 parameter
    th_or = theta.double().cpu().numpy()
    th_or[3 * F:3 * F + 2 * F * F] = bf16_round(th_or[3 * F:3 * F + 2 * F * F])
    d = hz.bond_log_ratios(lambda x: gcn.logpsi_complex(th_or, F, L, Ah, x), g.edges, states)
    bonds = np.array([int(tr[cs[p], ks[p], 0]) for p in pick])
    want = d.real[np.arange(len(pick)), bonds]
    got = np.array([tr[cs[p], ks[p], 2] for p in pick])
    assert np.abs(got - want).max() <= 2e-3, float(np.abs(got - want).max())
