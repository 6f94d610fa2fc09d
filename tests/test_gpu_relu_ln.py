"""GPU parity of the ReLU + layer-norm nonlinearity (GNA_ACT_RELU_LN, the paper's f) against
the FP64 oracle on the same seeded inputs: log Psi, the local energy of the hard-core bosons
(full and incremental), the Metropolis sampler's trajectories, the backward and the ISGO
gradient, at FP64 (1e-10) and FP32 (1e-5; gradients 1e-4), and the refusal of BF16."""
import numpy as np
import pytest

from oracle import gcn, heisenberg as hz, isgo, sampler
from paper_2011_12453_gb300 import build as B, gna, workloads as W

import scales as SC

pytestmark = pytest.mark.gpu
ACT = "relu_ln"
TOL = {gna.PREC_FP64: 1e-10, gna.PREC_FP32: 1e-5}


@pytest.fixture(scope="module")
def torch():
    import torch as t

    B.build()
    t.cuda.set_device(0)
    return t


def _setup(torch, g, F, L, prec, shared=True, seed=0, scale=0.5, xxz=None):
    th = W.random_theta(F, L, seed=seed, scale=scale, shared=shared)
    graph = gna.Graph(g.n_sites, g.edges, g.J, L, xxz=xxz)
    model = gna.Model(F, L, prec, shared, act=gna.ACT_RELU_LN)
    theta = torch.tensor(th, dtype=model.theta_dtype(), device="cuda")
    th_used = theta.double().cpu().numpy()
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    return graph, model, theta, th_used, Ah


def _geoms():
    return {"kagome2": W.kagome(2), "tri34": W.triangular(3, 4), "random12": W.erdos_renyi(12, 0.5, seed=7),
            "kagome6": W.kagome(6)}


def _close(got, want, tol, scale=None):
    """Element by element: |got - want| <= tol * max(scale, 1), scale = |want| unless given (the
    magnitude of the terms the value is summed from, tests/scales.py)."""
    got, want = np.asarray(got), np.asarray(want)
    err = np.abs(got - want)
    lim = tol * np.maximum(np.abs(want) if scale is None else scale, 1.0)
    assert np.all(err <= lim), (float(np.max(err - lim)), float(err.max()))


@pytest.mark.parametrize("prec", [gna.PREC_FP64, gna.PREC_FP32])
@pytest.mark.parametrize("geom", ["kagome2", "tri34", "random12", "kagome6"])
@pytest.mark.parametrize("shared", [True, False])
def test_forward_parity(torch, prec, geom, shared):
    g = _geoms()[geom]
    F, L = (16, 3) if geom != "kagome6" else (32, 4)
    graph, model, theta, th, Ah = _setup(torch, g, F, L, prec, shared)
    for Bn in (29, 1):
        s = W.random_spins(g.n_sites, Bn, seed=Bn)
        got = gna.forward(graph, model, theta, torch.tensor(s, device="cuda")).cpu().numpy()
        _close(got, gcn.logpsi(th, F, L, Ah, s, shared, ACT), TOL[prec], SC.logpsi_scale(th, F, L, Ah, s, shared, ACT))


@pytest.mark.parametrize("prec", [gna.PREC_FP64, gna.PREC_FP32])
@pytest.mark.parametrize("mode", [gna.ELOC_FULL, gna.ELOC_INCREMENTAL])
@pytest.mark.parametrize("geom", ["kagome2", "tri34", "random12"])
def test_boson_local_energy_parity(torch, prec, mode, geom):
    # the paper's model: hard-core bosons at t/V = 0.5 with ReLU + layer norm, 3 layers, F = 16
    g = _geoms()[geom]
    F, L = 16, 3
    xxz = hz.hardcore_bosons(g.edges.shape[0], 0.5, 1.0)
    graph, model, theta, th, Ah = _setup(torch, g, F, L, prec, xxz=xxz)
    s = W.random_spins(g.n_sites, 21, seed=4)
    E, dl = gna.local_energy(graph, model, theta, torch.tensor(s, device="cuda"), mode, bonds=True)
    E = E.cpu().numpy()
    lp_fn = lambda x: gcn.logpsi_complex(th, F, L, Ah, x, True, ACT)  # noqa: E731
    _close(E[:, 0] + 1j * E[:, 1], hz.local_energy(lp_fn, g.edges, None, s, xxz), TOL[prec],
           SC.eloc_scale(th, F, L, Ah, g.edges, None, s, act=ACT, xxz=xxz))
    d = hz.bond_log_ratios(lp_fn, g.edges, s)
    want_d = np.where(np.isnan(d.real), 0.0, d.real)
    assert np.all(np.abs(dl.cpu().numpy() - want_d) <= TOL[prec] * np.maximum(SC.delta_scale(
        th, F, L, Ah, g.edges, s, act=ACT), 1.0) + 2.0 ** -24 * np.abs(want_d))


def test_metropolis_fp64_trajectories_match_oracle(torch):
    g = W.kagome(2)
    F, L = 16, 3
    graph, model, theta, th, Ah = _setup(torch, g, F, L, gna.PREC_FP64, scale=0.8)
    C, sweeps, seed, step0 = 10, 3, 4321, 5
    s0 = W.random_spins(g.n_sites, C, seed=2)
    ch = torch.tensor(s0, device="cuda")
    samples, lpo, acc, tr = gna.metropolis_sweep(graph, model, theta, ch, sweeps, 1, seed, step0, trace=True)
    lp_fn = lambda x: gcn.logpsi_complex(th, F, L, Ah, x, True, ACT)  # noqa: E731
    s_o, samp_o, lp_o, acc_o, tr_o = sampler.run_chains(lp_fn, g.edges, s0, seed, step0, sweeps, 1)
    tr = tr.cpu().numpy()
    assert np.array_equal(tr[:, :, 0], tr_o[:, :, 0])
    m = ~np.isnan(tr_o[:, :, 2])
    assert np.array_equal(np.isnan(tr[:, :, 2]), ~m)
    assert np.abs(tr[:, :, 2][m] - tr_o[:, :, 2][m]).max() < 1e-10
    assert np.array_equal(tr[:, :, 1], tr_o[:, :, 1])
    assert np.array_equal(samples.cpu().numpy(), samp_o)
    assert np.array_equal(ch.cpu().numpy(), s_o)
    assert np.array_equal(acc.cpu().numpy(), acc_o)
    lpo = lpo.cpu().numpy()
    _close(lpo[..., 0] + 1j * lpo[..., 1], lp_o, 1e-10)


@pytest.mark.parametrize("prec", [gna.PREC_FP64, gna.PREC_FP32])
@pytest.mark.parametrize("shared", [True, False])
def test_backward_parity(torch, prec, shared):
    g = W.erdos_renyi(20, 0.2, seed=5)
    F, L = 16, 3
    graph, model, theta, th, Ah = _setup(torch, g, F, L, prec, shared)
    s = W.random_spins(g.n_sites, 37, seed=6)
    cot = np.random.default_rng(1).normal(size=(37, 2))
    got = gna.backward(graph, model, theta, torch.tensor(s, device="cuda"), torch.tensor(cot, device="cuda"))
    want = isgo.backward(th, F, L, Ah, s, cot, shared, ACT)
    _close(got.cpu().numpy(), want, TOL[prec], SC.grad_scale(th, F, L, Ah, s, cot, shared, ACT))


@pytest.mark.parametrize("prec", [gna.PREC_FP64, gna.PREC_FP32])
def test_boson_isgo_grad_parity(torch, prec):
    g = W.kagome(2)
    F, L = 16, 3
    xxz = hz.hardcore_bosons(g.edges.shape[0], 0.5, 1.0)
    graph, model, theta, th, Ah = _setup(torch, g, F, L, prec, xxz=xxz)
    th0 = th - W.random_theta(F, L, seed=9, scale=0.02)
    s = W.random_spins(g.n_sites, 64, seed=8)
    lp0 = gcn.logpsi(th0, F, L, Ah, s, True, ACT)
    grad, stats = gna.isgo_grad(graph, model, theta, torch.tensor(s, device="cuda"), torch.tensor(lp0, device="cuda"))
    g_o, Ebar, var, ess, E, p = isgo.isgo_gradient(th, F, L, Ah, g.edges, None, s, lp0[:, 0] + 1j * lp0[:, 1],
                                                   xxz=xxz, act=ACT)
    tol = TOL[prec]
    _close(grad.cpu().numpy(), g_o, tol, SC.grad_scale(th, F, L, Ah, s, isgo.cotangents(p, E, Ebar), act=ACT))
    _close(stats.cpu().numpy()[:2], [Ebar.real, Ebar.imag], tol,
           float((p * SC.eloc_scale(th, F, L, Ah, g.edges, None, s, act=ACT, xxz=xxz)).sum()))


def test_bf16_relu_ln_is_unsupported(torch):
    g = W.kagome(2)
    graph = gna.Graph.from_workload(g, 2)
    model = gna.Model(16, 2, gna.PREC_BF16, act=gna.ACT_RELU_LN)
    theta = torch.zeros(model.num_params, dtype=torch.float32, device="cuda")
    s = torch.tensor(W.random_spins(g.n_sites, 2, seed=1), device="cuda")
    with pytest.raises(gna.GnaError) as ei:
        gna.forward(graph, model, theta, s)
    assert ei.value.status == gna.GNA_ERR_UNSUPPORTED
