"""GPU grouping of duplicated samples (gna_dedup) against the oracle (oracle/dedup.py):
unique states in first-occurrence order, their log Psi^0 and counts bit-exact; the ISGO
gradient with counts on the grouped states equals the gradient on the raw samples."""
import numpy as np
import pytest

from oracle import dedup as D, gcn
from paper_2011_12453_gb300 import build as B, gna, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t

    B.build()
    t.cuda.set_device(0)
    return t


def _with_duplicates(N, n_base, Bn, seed):
    rng = np.random.default_rng(seed)
    base = W.random_spins(N, n_base, seed=seed)
    s = base[rng.integers(0, n_base, size=Bn)]
    lp = rng.normal(size=(Bn, 2))
    return s, lp


@pytest.mark.parametrize("N,n_base,Bn", [(10, 40, 5000), (108, 3000, 20000), (300, 500, 3000), (64, 64, 64),
                                         (7, 1, 1000)])
def test_dedup_parity(torch, N, n_base, Bn):
    s, lp = _with_duplicates(N, n_base, Bn, seed=N)
    us, ul, uc = gna.dedup(torch.tensor(s, device="cuda"), torch.tensor(lp, device="cuda"))
    ws, wl, wc = D.group(s, lp)
    assert np.array_equal(us.cpu().numpy(), ws)
    assert np.array_equal(ul.cpu().numpy(), wl)
    assert np.array_equal(uc.cpu().numpy(), wc)


def test_dedup_empty_single_and_without_logpsi(torch):
    us, ul, uc = gna.dedup(torch.zeros((0, 5), dtype=torch.int8, device="cuda"))
    assert us.shape == (0, 5) and uc.numel() == 0
    one = torch.tensor(W.random_spins(9, 1, seed=1), device="cuda")
    us, ul, uc = gna.dedup(one, torch.zeros((1, 2), dtype=torch.float64, device="cuda"))
    assert torch.equal(us, one) and uc.tolist() == [1.0]
    s, _ = _with_duplicates(20, 10, 300, seed=3)
    us, ul, uc = gna.dedup(torch.tensor(s, device="cuda"))
    ws, _, wc = D.group(s, np.zeros((300, 2)))
    assert ul is None and np.array_equal(us.cpu().numpy(), ws) and np.array_equal(uc.cpu().numpy(), wc)


def test_isgo_grad_on_grouped_samples_equals_raw(torch):
    g = W.kagome(2)
    F, L = 16, 2
    graph = gna.Graph.from_workload(g, L)
    model = gna.Model(F, L, gna.PREC_FP64)
    th = W.random_theta(F, L, seed=2, scale=0.5)
    theta = torch.tensor(th, device="cuda")
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    s, _ = _with_duplicates(g.n_sites, 50, 2000, seed=4)
    lp0 = gcn.logpsi(th - W.random_theta(F, L, seed=5, scale=0.02), F, L, Ah, s)
    st, l0 = torch.tensor(s, device="cuda"), torch.tensor(lp0, device="cuda")
    g_raw, s_raw = gna.isgo_grad(graph, model, theta, st, l0)
    us, ul, uc = gna.dedup(st, l0)
    assert us.shape[0] <= 50
    g_grp, s_grp = gna.isgo_grad(graph, model, theta, us.contiguous(), ul.contiguous(), counts=uc.contiguous())
    a, b = g_grp.cpu().numpy(), g_raw.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-10 * max(1.0, np.abs(b).max())
    assert np.abs(s_grp.cpu().numpy()[:2] - s_raw.cpu().numpy()[:2]).max() <= 1e-10
