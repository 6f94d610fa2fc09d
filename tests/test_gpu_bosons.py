"""GPU parity of the XXZ bond coefficients (gna_graph_create_xxz) against the FP64 oracle:
the local energy of the hard-core bosons of the numerical-experiments section,
H = -t sum (b+_i b_j + h.c.) + V sum n_i n_j, i.e. per bond (Jz, Jxy, hz, c) =
(V, -2t, V/2, V/4), and of random XXZ bonds, in full and incremental form at FP64 / FP32 and
on the BF16 tensor-core path, and the ISGO gradient built on it.  Tolerances as the
Heisenberg tests: 1e-10 (FP64), 1e-5 (FP32), BF16 per-sample 1e-3 at weight scale 0.1."""
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


def _random_xxz(E, seed):
    r = np.random.default_rng(seed)
    return (r.uniform(-1.5, 1.5, E), r.uniform(-1.5, 1.5, E), r.uniform(-0.7, 0.7, E), r.uniform(-0.5, 0.5, E))


def _case(name):
    g = {"kagome2": W.kagome(2), "tri34": W.triangular(3, 4), "er12": W.erdos_renyi(12, 0.5, seed=7)}[name]
    E = g.edges.shape[0]
    return g, {"bosons": hz.hardcore_bosons(E, 1.0, 2.5), "random": _random_xxz(E, 3)}


def _close(got, want, tol, scale=None):
    """Element by element: |got - want| <= tol * max(scale, 1), scale = |want| unless given (the
    magnitude of the terms the value is summed from, tests/scales.py)."""
    got, want = np.asarray(got), np.asarray(want)
    err = np.abs(got - want)
    lim = tol * np.maximum(np.abs(want) if scale is None else scale, 1.0)
    assert np.all(err <= lim), (float(np.max(err - lim)), float(err.max()))


@pytest.mark.parametrize("prec", [gna.PREC_FP64, gna.PREC_FP32])
@pytest.mark.parametrize("mode", [gna.ELOC_FULL, gna.ELOC_INCREMENTAL])
@pytest.mark.parametrize("name", ["kagome2", "tri34", "er12"])
@pytest.mark.parametrize("kind", ["bosons", "random"])
def test_xxz_local_energy_parity(torch, prec, mode, name, kind):
    g, coeffs = _case(name)
    xxz = coeffs[kind]
    F, L = 16, 2
    th = W.random_theta(F, L, seed=1, scale=0.6)
    graph = gna.Graph(g.n_sites, g.edges, g.J, L, xxz=xxz)
    model = gna.Model(F, L, prec)
    theta = torch.tensor(th, dtype=model.theta_dtype(), device="cuda")
    th_used = theta.double().cpu().numpy()
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    # half filling and a doped sector (the boson number is the number of up spins)
    for n_up in (g.n_sites // 2, g.n_sites // 3):
        s = W.random_spins(g.n_sites, 17, seed=n_up, n_up=n_up)
        E = gna.local_energy(graph, model, theta, torch.tensor(s, device="cuda"), mode).cpu().numpy()
        want = hz.local_energy(lambda x: gcn.logpsi_complex(th_used, F, L, Ah, x), g.edges, None, s, xxz)
        _close(E[:, 0] + 1j * E[:, 1], want, 1e-10 if prec == gna.PREC_FP64 else 1e-5,
               SC.eloc_scale(th_used, F, L, Ah, g.edges, None, s, xxz=xxz))


def test_heisenberg_coefficients_reproduce_the_heisenberg_graph(torch):
    # (Jz, Jxy, hz, c) = (J, J, 0, 0) through gna_graph_create_xxz gives the bits of gna_graph_create
    g = W.erdos_renyi(20, 0.2, seed=5, J_range=(0.5, 1.5))
    F, L = 16, 2
    th = W.random_theta(F, L, seed=2, scale=0.5)
    theta = torch.tensor(th, device="cuda")
    model = gna.Model(F, L, gna.PREC_FP64)
    s = torch.tensor(W.random_spins(g.n_sites, 11, seed=1), device="cuda")
    a = gna.local_energy(gna.Graph(g.n_sites, g.edges, g.J, L), model, theta, s).cpu().numpy()
    b = gna.local_energy(gna.Graph(g.n_sites, g.edges, None, L, xxz=(g.J, g.J, 0.0, 0.0)), model, theta,
                         s).cpu().numpy()
    assert np.array_equal(a, b)


def test_xxz_bf16_local_energy_kagome108(torch):
    # BF16 tensor-core incremental local energy of the hard-core bosons, Kagome 6x6x3, L = 4,
    # F = 32, weight scale 0.1; the oracle runs on W rounded to BF16
    g = W.kagome(6)
    F, L = 32, 4
    xxz = hz.hardcore_bosons(g.edges.shape[0], 1.0, 2.5)
    th = W.random_theta(F, L, seed=0, scale=0.1)
    graph = gna.Graph(g.n_sites, g.edges, None, L, xxz=xxz)
    model = gna.Model(F, L, gna.PREC_BF16)
    theta = torch.tensor(th, dtype=torch.float32, device="cuda")
    th_or = theta.double().cpu().numpy()
    o = 3 * F
    th_or[o:o + 2 * F * F] = torch.tensor(th_or[o:o + 2 * F * F], dtype=torch.float32).to(
        torch.bfloat16).double().numpy()
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    s = W.random_spins(g.n_sites, 4, seed=5)
    E = gna.local_energy(graph, model, theta, torch.tensor(s, device="cuda"), gna.ELOC_INCREMENTAL).cpu().numpy()
    want = hz.local_energy(lambda x: gcn.logpsi_complex(th_or, F, L, Ah, x), g.edges, None, s, xxz)
    rel = np.abs(E[:, 0] + 1j * E[:, 1] - want) / np.abs(want).clip(1.0)
    assert rel.max() <= 1e-3, rel.max()


@pytest.mark.parametrize("prec", [gna.PREC_FP64, gna.PREC_FP32])
def test_xxz_isgo_grad_parity(torch, prec):
    # Kagome 2x2x3 hard-core bosons at t/V = 0.4
    g = W.kagome(2)
    F, L = 16, 2
    xxz = hz.hardcore_bosons(g.edges.shape[0], 1.0, 2.5)
    th = W.random_theta(F, L, seed=0, scale=0.5)
    graph = gna.Graph(g.n_sites, g.edges, None, L, xxz=xxz)
    model = gna.Model(F, L, prec)
    theta = torch.tensor(th, dtype=model.theta_dtype(), device="cuda")
    th = theta.double().cpu().numpy()
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    th0 = th - W.random_theta(F, L, seed=9, scale=0.02)
    s = W.random_spins(g.n_sites, 64, seed=8)
    lp0 = gcn.logpsi(th0, F, L, Ah, s)
    grad, stats = gna.isgo_grad(graph, model, theta, torch.tensor(s, device="cuda"), torch.tensor(lp0, device="cuda"))
    g_o, Ebar, var, ess, E, p = isgo.isgo_gradient(th, F, L, Ah, g.edges, None, s, lp0[:, 0] + 1j * lp0[:, 1],
                                                   xxz=xxz)
    tol = 1e-10 if prec == gna.PREC_FP64 else 1e-5
    _close(grad.cpu().numpy(), g_o, tol, SC.grad_scale(th, F, L, Ah, s, isgo.cotangents(p, E, Ebar)))
    _close(stats.cpu().numpy()[:2], [Ebar.real, Ebar.imag], tol,
           float((p * SC.eloc_scale(th, F, L, Ah, g.edges, None, s, xxz=xxz)).sum()))
