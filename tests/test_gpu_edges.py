"""Edge cases of the GPU path against the FP64 oracle: a graph without bonds, an isolated
site (a zero row of D^-1/2 A D^-1/2), an odd number of sites (N_up = floor(N/2)), the
largest model the library takes (L = 8, F = 64) on a graph that the deepest balls cover
completely, and the largest graph (4096 sites).  Tolerances: 1e-10 FP64, 1e-5 FP32, BF16
2e-2 on log Psi and 1e-3 per-sample local energy at weight scale 0.1."""
import numpy as np
import pytest

from oracle import gcn, heisenberg as hz, isgo
from paper_2011_12453_gb300 import build as B, gna, workloads as W

import scales as SC

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t

    B.build()
    t.cuda.set_device(0)
    return t


def _close(got, want, tol, scale=None):
    """Element by element: |got - want| <= tol * max(scale, 1), scale = |want| unless given (the
    magnitude of the terms the value is summed from, tests/scales.py)."""
    got, want = np.asarray(got), np.asarray(want)
    err = np.abs(got - want)
    lim = tol * np.maximum(np.abs(want) if scale is None else scale, 1.0)
    assert np.all(err <= lim), (float(np.max(err - lim)), float(err.max()))


def _ah(g):
    return gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))


def _bf16_W(torch, th, F):
    out = th.copy()
    o = 3 * F
    out[o:o + 2 * F * F] = torch.tensor(out[o:o + 2 * F * F], dtype=torch.float32).to(torch.bfloat16).double().numpy()
    return out


def test_graph_without_bonds(torch):
    g = W.Graph(1, np.zeros((0, 2), dtype=np.int32), np.zeros(0), "single")
    F, L = 8, 2
    th = W.random_theta(F, L, seed=1, scale=0.5)
    graph = gna.Graph.from_workload(g, L)
    model = gna.Model(F, L, gna.PREC_FP64)
    theta = torch.tensor(th, device="cuda")
    s = np.array([[1], [-1]], dtype=np.int8)
    st = torch.tensor(s, device="cuda")
    _close(gna.forward(graph, model, theta, st).cpu().numpy(), gcn.logpsi(th, F, L, _ah(g), s), 1e-12)
    for mode in (gna.ELOC_FULL, gna.ELOC_INCREMENTAL):
        assert np.all(gna.local_energy(graph, model, theta, st, mode).cpu().numpy() == 0.0)
    with pytest.raises(gna.GnaError) as ei:
        gna.metropolis_sweep(graph, model, theta, st.clone(), 1, 0, 1, 0)
    assert ei.value.status == gna.GNA_ERR_INVALID_ARG


@pytest.mark.parametrize("prec", [gna.PREC_FP64, gna.PREC_FP32])
def test_isolated_site(torch, prec):
    ring = W.ring(9)
    g = W.Graph(10, ring.edges, ring.J, "ring9_plus_isolated")  # site 9 has no bond
    F, L = 16, 3
    th = W.random_theta(F, L, seed=2, scale=0.6)
    graph = gna.Graph.from_workload(g, L)
    model = gna.Model(F, L, prec)
    theta = torch.tensor(th, dtype=model.theta_dtype(), device="cuda")
    th = theta.double().cpu().numpy()
    Ah = _ah(g)
    assert np.all(Ah[9] == 0.0)
    s = W.random_spins(g.n_sites, 13, seed=3)
    st = torch.tensor(s, device="cuda")
    tol = 1e-10 if prec == gna.PREC_FP64 else 1e-5
    _close(gna.forward(graph, model, theta, st).cpu().numpy(), gcn.logpsi(th, F, L, Ah, s), tol,
           SC.logpsi_scale(th, F, L, Ah, s))
    want = hz.local_energy(lambda x: gcn.logpsi_complex(th, F, L, Ah, x), g.edges, g.J, s)
    for mode in (gna.ELOC_FULL, gna.ELOC_INCREMENTAL):
        E = gna.local_energy(graph, model, theta, st, mode).cpu().numpy()
        _close(E[:, 0] + 1j * E[:, 1], want, tol, SC.eloc_scale(th, F, L, Ah, g.edges, g.J, s))
    cot = np.random.default_rng(4).normal(size=(13, 2))
    got = gna.backward(graph, model, theta, st, torch.tensor(cot, device="cuda")).cpu().numpy()
    _close(got, isgo.backward(th, F, L, Ah, s, cot), tol, SC.grad_scale(th, F, L, Ah, s, cot))
    ch = st.clone()
    gna.metropolis_sweep(graph, model, theta, ch, 2, 0, 5, 0)
    c = ch.cpu().numpy()
    assert np.array_equal(c[:, 9], s[:, 9])  # no bond reaches the isolated site
    assert np.array_equal((c > 0).sum(1), (s > 0).sum(1))


@pytest.mark.parametrize("prec", [gna.PREC_FP64, gna.PREC_FP32, gna.PREC_BF16])
def test_odd_number_of_sites(torch, prec):
    g = W.erdos_renyi(33, 4.0 / 32, seed=1001, J_range=(0.5, 1.5))
    assert g.n_sites % 2 == 1
    F, L = 16, 3
    scale = 0.1 if prec == gna.PREC_BF16 else 0.5
    th = W.random_theta(F, L, seed=5, scale=scale)
    graph = gna.Graph.from_workload(g, L)
    model = gna.Model(F, L, prec)
    theta = torch.tensor(th, dtype=model.theta_dtype(), device="cuda")
    th = theta.double().cpu().numpy()
    if prec == gna.PREC_BF16:
        th = _bf16_W(torch, th, F)
    Ah = _ah(g)
    s = W.random_spins(g.n_sites, 9, seed=6)
    assert np.all((s > 0).sum(1) == 16)
    st = torch.tensor(s, device="cuda")
    tol = {gna.PREC_FP64: 1e-10, gna.PREC_FP32: 1e-5, gna.PREC_BF16: 2e-2}[prec]
    _close(gna.forward(graph, model, theta, st).cpu().numpy(), gcn.logpsi(th, F, L, Ah, s), tol)
    E = gna.local_energy(graph, model, theta, st, gna.ELOC_INCREMENTAL).cpu().numpy()
    want = hz.local_energy(lambda x: gcn.logpsi_complex(th, F, L, Ah, x), g.edges, g.J, s)
    rel = np.abs(E[:, 0] + 1j * E[:, 1] - want) / np.abs(want).clip(1.0)
    assert rel.max() <= {gna.PREC_FP64: 1e-9, gna.PREC_FP32: 1e-4, gna.PREC_BF16: 1e-3}[prec], rel.max()
    ch = torch.tensor(W.random_spins(g.n_sites, 64, seed=7), device="cuda")
    gna.metropolis_sweep(graph, model, theta, ch, 3, 0, 9, 0)
    assert np.all((ch.cpu().numpy() > 0).sum(1) == 16)


@pytest.mark.parametrize("prec", [gna.PREC_FP64, gna.PREC_BF16])
def test_largest_model_on_a_fully_covered_graph(torch, prec):
    # L = 8, F = 64 on the triangular 4x4 torus: from layer 2 on every bond's ball is the whole graph
    g = W.triangular(4, 4)
    F, L = 64, 8
    assert np.all(gna.ball_sizes_host(g.n_sites, g.edges, L)[:, 2:] == g.n_sites)
    scale = 0.1
    th = W.random_theta(F, L, seed=8, scale=scale)
    graph = gna.Graph.from_workload(g, L)
    model = gna.Model(F, L, prec)
    theta = torch.tensor(th, dtype=model.theta_dtype(), device="cuda")
    th = theta.double().cpu().numpy()
    if prec == gna.PREC_BF16:
        th = _bf16_W(torch, th, F)
    Ah = _ah(g)
    s = W.random_spins(g.n_sites, 7, seed=9)
    st = torch.tensor(s, device="cuda")
    tol_lp = 1e-10 if prec == gna.PREC_FP64 else 2e-2
    _close(gna.forward(graph, model, theta, st).cpu().numpy(), gcn.logpsi(th, F, L, Ah, s), tol_lp)
    E = gna.local_energy(graph, model, theta, st, gna.ELOC_INCREMENTAL).cpu().numpy()
    want = hz.local_energy(lambda x: gcn.logpsi_complex(th, F, L, Ah, x), g.edges, g.J, s)
    rel = np.abs(E[:, 0] + 1j * E[:, 1] - want) / np.abs(want).clip(1.0)
    assert rel.max() <= (1e-9 if prec == gna.PREC_FP64 else 1e-3), rel.max()
    cot = np.random.default_rng(10).normal(size=(7, 2))
    got = gna.backward(graph, model, theta, st, torch.tensor(cot, device="cuda")).cpu().numpy()
    want_g = isgo.backward(th, F, L, Ah, s, cot)
    if prec == gna.PREC_FP64:
        _close(got, want_g, 1e-10)
    else:
        assert np.abs(got - want_g).max() <= 5e-3 * np.abs(want_g).max()


def test_largest_graph_4096_sites(torch):
    # triangular 64x64 (4096 sites, 12288 bonds), F = 16, L = 2: FP32 and BF16 forward against
    # the oracle, and the BF16 incremental per-bond Delta of sampled bonds against oracle
    # forwards of the exchanged configurations; the BF16 local energy against the FP32 one
    g = W.triangular(64, 64)
    F, L = 16, 2
    th = W.random_theta(F, L, seed=11, scale=0.1)
    graph = gna.Graph.from_workload(g, L)
    Ah = _ah(g)
    s = W.random_spins(g.n_sites, 2, seed=12)
    st = torch.tensor(s, device="cuda")
    m32 = gna.Model(F, L, gna.PREC_FP32)
    m16 = gna.Model(F, L, gna.PREC_BF16)
    theta = torch.tensor(th, dtype=torch.float32, device="cuda")
    th32 = theta.double().cpu().numpy()
    th16 = _bf16_W(torch, th32, F)
    _close(gna.forward(graph, m32, theta, st).cpu().numpy(), gcn.logpsi(th32, F, L, Ah, s), 1e-5)
    _close(gna.forward(graph, m16, theta, st).cpu().numpy(), gcn.logpsi(th16, F, L, Ah, s), 2e-2)
    E16, d16 = gna.local_energy(graph, m16, theta, st, gna.ELOC_INCREMENTAL, bonds=True)
    E32 = gna.local_energy(graph, m32, theta, st, gna.ELOC_INCREMENTAL).cpu().numpy()
    E16 = E16.cpu().numpy()
    assert np.abs(E16 - E32).max() <= 1e-3 * np.abs(E32).max()
    d16 = d16.cpu().numpy()
    lp = gcn.logpsi(th16, F, L, Ah, s[:1])[0, 0]
    rng = np.random.default_rng(13)
    anti = np.nonzero(s[0, g.edges[:, 0]] != s[0, g.edges[:, 1]])[0]
    for e in rng.choice(anti, size=4, replace=False):
        x = s[:1].copy()
        i, j = g.edges[e]
        x[0, [i, j]] = x[0, [j, i]]
        want = gcn.logpsi(th16, F, L, Ah, x)[0, 0] - lp
        assert abs(d16[0, e] - want) <= 2e-3 * max(1.0, abs(want)), (e, d16[0, e], want)
