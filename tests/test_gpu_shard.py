"""The device side of the sample-sharded ISGO step (gna_isgo_partials, gna_isgo_finish and
the backward per shard), with the collectives of paper_2011_12453_gb300.shard emulated in
one process over three unequal contiguous shards: the gradient and statistics equal those
of isgo_grad on the whole batch to 1e-12 (FP64), with and without counts."""
import numpy as np
import pytest

from paper_2011_12453_gb300 import build as B, gna, shard, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t

    B.build()
    t.cuda.set_device(0)
    return t


class _Gathered:
    """Emulated collectives: the shards' values are known in advance (max and sum over them)."""

    def __init__(self, values):
        self.values = values

    def max_(self, t):
        t.copy_(max(v for v in self.values).reshape(t.shape))
        return t

    def sum_(self, t):
        t.copy_(sum(self.values).reshape(t.shape))
        return t


@pytest.mark.parametrize("with_counts", [False, True])
def test_sharded_device_pieces_equal_isgo_grad(torch, with_counts):
    g = W.kagome(2)
    F, L, Bn, S = 16, 2, 61, 3
    graph = gna.Graph.from_workload(g, L)
    model = gna.Model(F, L, gna.PREC_FP64)
    theta = torch.tensor(W.random_theta(F, L, seed=1, scale=0.5), device="cuda")
    theta0 = theta - torch.tensor(W.random_theta(F, L, seed=2, scale=0.05), device="cuda")
    s = torch.tensor(W.random_spins(g.n_sites, Bn, seed=3), device="cuda")
    lp0 = gna.forward(graph, model, theta0, s)
    counts = torch.tensor(np.random.default_rng(4).integers(1, 5, size=Bn).astype(np.float64),
                          device="cuda") if with_counts else None
    want_g, want_st = gna.isgo_grad(graph, model, theta, s, lp0, counts=counts)
    K = shard.LibraryKernels(graph, model)
    blocks = [shard.shard_range(Bn, r, S) for r in range(S)]
    cnt = [counts[lo:hi].contiguous() if counts is not None else None for lo, hi in blocks]
    lp = [K.forward(theta, s[lo:hi].contiguous()) for lo, hi in blocks]
    E = [K.local_energy(theta, s[lo:hi].contiguous()) for lo, hi in blocks]
    p4 = [K.partials(lp[k], lp0[lo:hi].contiguous(), E[k], cnt[k]) for k, (lo, hi) in enumerate(blocks)]
    # collective 1 and 2: the shift and the rescaled sums
    m = max(float(p[0]) for p in p4)
    rescaled = [p[1:4] * torch.exp(p[0] - m) for p in p4]
    g4 = shard.combine_partials(p4[0], _Gathered2(m, rescaled, p4[0]))
    fin = [K.finish(lp[k], lp0[lo:hi].contiguous(), E[k], g4, cnt[k]) for k, (lo, hi) in enumerate(blocks)]
    stats, copies = shard.combine_stats(g4, fin[0][1], _Gathered([f[1] for f in fin]))
    grad = sum(K.backward(theta, s[lo:hi].contiguous(), fin[k][0]) for k, (lo, hi) in enumerate(blocks))
    want_g, want_st, grad, stats = (x.cpu().numpy() for x in (want_g, want_st, grad, stats))
    assert np.all(np.abs(grad - want_g) <= 1e-12 * np.abs(want_g).max())
    assert np.all(np.abs(stats - want_st) <= 1e-12 * np.maximum(np.abs(want_st), 1.0))
    assert float(copies) == (float(counts.sum()) if counts is not None else Bn)


class _Gathered2:
    """combine_partials' two collectives for shard 0: the global max, then the sum of every
    shard's rescaled sums (shard 0's own rescaled by the module itself)."""

    def __init__(self, m, rescaled, own):
        self.m, self.rescaled, self.own = m, rescaled, own

    def max_(self, t):
        t.fill_(self.m)
        return t

    def sum_(self, t):
        t.copy_(sum(self.rescaled))
        return t
