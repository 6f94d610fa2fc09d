"""Parity on the shapes of the two workloads that the other GPU tests do not cover at
size: the set of 32 Erdos-Renyi graphs (sizes 32-96, mean degree 4, J uniform in
[0.5, 1.5], L = 3, F = 32) and Kagome 12x12x3 (432 sites, L = 6, F = 64).  Checked against
the FP64 oracle where it finishes in seconds (log Psi, local energies of a few samples,
per-bond Delta of sampled bonds), else against properties: BF16 against FP32 local
energies, recorded log Psi against a fresh forward, conservation of the number of up spins.
Tolerances: FP32 1e-5 (log Psi) and 1e-4 (local energy, relative), BF16 2e-2 on log Psi,
1e-3 per-sample local energy and 2e-3 on Delta at weight scale 0.1 (oracle on BF16-rounded W)."""
import numpy as np
import pytest

from oracle import gcn, heisenberg as hz
from paper_2011_12453_gb300 import build as B, gna, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t

    B.build()
    t.cuda.set_device(0)
    return t


def _ah(g):
    return gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))


def _bf16_W(torch, th, F):
    out = th.copy()
    o = 3 * F
    out[o:o + 2 * F * F] = torch.tensor(out[o:o + 2 * F * F], dtype=torch.float32).to(torch.bfloat16).double().numpy()
    return out


def _rel(E, want):
    return (np.abs(E[:, 0] + 1j * E[:, 1] - want) / np.abs(want).clip(1.0)).max()


def test_random_graph_set(torch):
    F, L = 32, 3
    th = W.random_theta(F, L, seed=0, scale=0.1)
    theta = torch.tensor(th, dtype=torch.float32, device="cuda")
    th32 = theta.double().cpu().numpy()
    th16 = _bf16_W(torch, th32, F)
    m32, m16 = gna.Model(F, L, gna.PREC_FP32), gna.Model(F, L, gna.PREC_BF16)
    for gi, g in enumerate(W.random_graph_set()):
        graph = gna.Graph.from_workload(g, L)
        Ah = _ah(g)
        s = W.random_spins(g.n_sites, 3, seed=gi)
        st = torch.tensor(s, device="cuda")
        lp = gna.forward(graph, m32, theta, st).cpu().numpy()
        want = gcn.logpsi(th32, F, L, Ah, s)
        assert np.abs(lp - want).max() <= 1e-5 * max(1.0, np.abs(want).max()), gi
        want_e = hz.local_energy(lambda x: gcn.logpsi_complex(th32, F, L, Ah, x), g.edges, g.J, s)
        assert _rel(gna.local_energy(graph, m32, theta, st, gna.ELOC_INCREMENTAL).cpu().numpy(), want_e) <= 1e-4, gi
        want_16 = hz.local_energy(lambda x: gcn.logpsi_complex(th16, F, L, Ah, x), g.edges, g.J, s)
        assert _rel(gna.local_energy(graph, m16, theta, st, gna.ELOC_INCREMENTAL).cpu().numpy(), want_16) <= 1e-3, gi
        # chains: the number of up spins is conserved and the recorded log Psi is the forward's
        ch = torch.tensor(W.random_spins(g.n_sites, 256, seed=100 + gi), device="cuda")
        samples, lpo, acc, _ = gna.metropolis_sweep(graph, m32, theta, ch, 2, 1, 7 + gi, 0)
        x = samples.cpu().numpy()
        assert np.all((x > 0).sum(-1) == g.n_sites // 2), gi
        f = gna.forward(graph, m32, theta, samples[-1].contiguous()).cpu().numpy()
        assert np.abs(lpo[-1].cpu().numpy() - f).max() <= 1e-5 * max(1.0, np.abs(f).max()), gi


def test_kagome432(torch):
    g = W.kagome(12)
    F, L = 64, 6
    th = W.random_theta(F, L, seed=0, scale=0.1)
    graph = gna.Graph.from_workload(g, L)
    m32, m16 = gna.Model(F, L, gna.PREC_FP32), gna.Model(F, L, gna.PREC_BF16)
    theta = torch.tensor(th, dtype=torch.float32, device="cuda")
    th16 = _bf16_W(torch, theta.double().cpu().numpy(), F)
    Ah = _ah(g)
    s = W.random_spins(g.n_sites, 16, seed=1)
    st = torch.tensor(s, device="cuda")
    want = gcn.logpsi(th16, F, L, Ah, s[:2])
    got = gna.forward(graph, m16, theta, st).cpu().numpy()
    assert np.abs(got[:2] - want).max() <= 2e-2 * max(1.0, np.abs(want).max())
    E16, d16 = gna.local_energy(graph, m16, theta, st, gna.ELOC_INCREMENTAL, bonds=True)
    E32 = gna.local_energy(graph, m32, theta, st, gna.ELOC_INCREMENTAL).cpu().numpy()
    E16, d16 = E16.cpu().numpy(), d16.cpu().numpy()
    assert np.abs(E16 - E32).max() <= 1e-3 * np.abs(E32).max()
    assert abs(E16[:, 0].mean() - E32[:, 0].mean()) <= 1e-4 * abs(E32[:, 0].mean())
    anti = np.nonzero(s[0, g.edges[:, 0]] != s[0, g.edges[:, 1]])[0]
    for e in np.random.default_rng(2).choice(anti, size=6, replace=False):
        x = s[:1].copy()
        i, j = g.edges[e]
        x[0, [i, j]] = x[0, [j, i]]
        dw = gcn.logpsi(th16, F, L, Ah, x)[0, 0] - want[0, 0]
        assert abs(d16[0, e] - dw) <= 2e-3 * max(1.0, abs(dw)), (e, d16[0, e], dw)
    ch = torch.tensor(W.random_spins(g.n_sites, 64, seed=3), device="cuda")
    samples, lpo, acc, _ = gna.metropolis_sweep(graph, m16, theta, ch, 1, 1, 5, 0)
    x = samples.cpu().numpy()
    assert np.all((x > 0).sum(-1) == g.n_sites // 2)
    assert acc.cpu().numpy().sum() > 0
    f = gna.forward(graph, m16, theta, samples[-1].contiguous()).cpu().numpy()
    assert np.abs(lpo[-1].cpu().numpy() - f).max() <= 2e-2 * max(1.0, np.abs(f).max())
