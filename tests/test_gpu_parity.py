"""GPU parity of the CUDA path (through the C ABI) against the FP64 CPU oracle on the
same seeded inputs: log Psi (Eq. gcn), the Heisenberg local energy (full and incremental),
the Metropolis sampler (bit-exact bookkeeping and decisions), the backward VJP and the
ISGO weights and gradient (Eq. isgo).

Tolerances, element by element: |got - want| <= tol * max(scale, 1) with tol = 1e-10 for
FP64 paths and 1e-5 for FP32, scale = the magnitude of the terms the value is summed from
(tests/scales.py: equal to |want| wherever the sum does not cancel, larger where it does --
the imaginary part of a local energy, a gradient entry whose samples' contributions nearly
cancel).  The per-bond Delta log Psi is returned as float32 by the ABI, so its FP64 check
allows the float32 rounding of the value (2^-24 relative)."""
import numpy as np
import pytest

from oracle import gcn, heisenberg as hz, isgo, sampler
from paper_2011_12453_gb300 import build as B, gna, workloads as W

import scales as SC

pytestmark = pytest.mark.gpu

TOL = {gna.PREC_FP64: 1e-10, gna.PREC_FP32: 1e-5}


@pytest.fixture(scope="module")
def torch():
    import torch as t

    B.build()
    t.cuda.set_device(0)
    return t


def _setup(torch, g, F, L, prec, shared=True, seed=0, scale=0.1, max_layers=None):
    th = W.random_theta(F, L, seed=seed, scale=scale, shared=shared)
    graph = gna.Graph.from_workload(g, L if max_layers is None else max_layers)
    model = gna.Model(F, L, prec, shared)
    theta = torch.tensor(th, dtype=model.theta_dtype(), device="cuda")
    th_used = theta.double().cpu().numpy()  # the values the device sees (fp32-rounded for FP32)
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    return graph, model, theta, th_used, Ah


def _geoms():
    return {"kagome2": W.kagome(2), "tri34": W.triangular(3, 4), "er20": W.erdos_renyi(20, 0.2, seed=5),
            "er_dense12": W.erdos_renyi(12, 0.5, seed=7)}


def _close(got, want, tol, scale=None):
    """Element by element: |got - want| <= tol * max(scale, 1), scale = |want| unless given (the
    magnitude of the terms the value is summed from, tests/scales.py)."""
    got, want = np.asarray(got), np.asarray(want)
    err = np.abs(got - want)
    lim = tol * np.maximum(np.abs(want) if scale is None else scale, 1.0)
    assert np.all(err <= lim), (float(np.max(err - lim)), float(err.max()))


# ---------------------------------------------------------------------------------
# Philox
# ---------------------------------------------------------------------------------

def test_philox_bit_exact(torch):
    rng = np.random.default_rng(0)
    n = 257
    keys = rng.integers(0, 2**63, size=(n, 2), dtype=np.int64)
    ctrs = rng.integers(0, 2**63, size=(n, 4), dtype=np.int64)
    keys[0] = [-1, -1]  # all-ones words
    out = gna.philox(torch.tensor(keys, device="cuda"), torch.tensor(ctrs, device="cuda")).cpu().numpy()
    for i in range(n):
        k = tuple(int(x) & (2**64 - 1) for x in keys[i])
        c = tuple(int(x) & (2**64 - 1) for x in ctrs[i])
        assert [int(x) & (2**64 - 1) for x in out[i]] == list(sampler.philox4x64_10(k, c))


# ---------------------------------------------------------------------------------
# forward
# ---------------------------------------------------------------------------------

@pytest.mark.parametrize("prec", [gna.PREC_FP64, gna.PREC_FP32])
@pytest.mark.parametrize("geom", ["kagome2", "tri34", "er20", "er_dense12"])
@pytest.mark.parametrize("shared", [True, False])
def test_forward_parity(torch, prec, geom, shared):
    g = _geoms()[geom]
    F, L = 16, 3
    graph, model, theta, th, Ah = _setup(torch, g, F, L, prec, shared, scale=0.5)
    for Bn in (37, 1):
        s = W.random_spins(g.n_sites, Bn, seed=Bn)
        got = gna.forward(graph, model, theta, torch.tensor(s, device="cuda")).cpu().numpy()
        _close(got, gcn.logpsi(th, F, L, Ah, s, shared), TOL[prec], SC.logpsi_scale(th, F, L, Ah, s, shared))


def test_forward_empty_batch_and_L0(torch):
    g = W.kagome(2)
    graph, model, theta, th, Ah = _setup(torch, g, 8, 0, gna.PREC_FP64, shared=False, scale=0.5)
    s = W.random_spins(g.n_sites, 5, seed=1)
    got = gna.forward(graph, model, theta, torch.tensor(s, device="cuda")).cpu().numpy()
    _close(got, gcn.logpsi(th, 8, 0, Ah, s, False), 1e-12)
    out = gna.forward(graph, model, theta, torch.empty((0, g.n_sites), dtype=torch.int8, device="cuda"))
    assert out.shape == (0, 2)


@pytest.mark.parametrize("F", [32, 48, 64])
def test_forward_wide_features(torch, F):
    g = W.triangular(6, 6)
    L = 4
    graph, model, theta, th, Ah = _setup(torch, g, F, L, gna.PREC_FP32, scale=0.2)
    s = W.random_spins(g.n_sites, 19, seed=2)
    got = gna.forward(graph, model, theta, torch.tensor(s, device="cuda")).cpu().numpy()
    _close(got, gcn.logpsi(th, F, L, Ah, s), TOL[gna.PREC_FP32], SC.logpsi_scale(th, F, L, Ah, s))


# ---------------------------------------------------------------------------------
# local energy
# ---------------------------------------------------------------------------------

def _oracle_eloc(th, F, L, Ah, g, s, shared=True):
    return hz.local_energy(lambda x: gcn.logpsi_complex(th, F, L, Ah, x, shared), g.edges, g.J, s)


@pytest.mark.parametrize("prec", [gna.PREC_FP64, gna.PREC_FP32])
@pytest.mark.parametrize("mode", [gna.ELOC_FULL, gna.ELOC_INCREMENTAL])
@pytest.mark.parametrize("geom", ["kagome2", "tri34", "er20", "er_dense12"])
def test_local_energy_parity(torch, prec, mode, geom):
    g = _geoms()[geom]
    if geom == "er20":
        g = W.erdos_renyi(20, 0.2, seed=5, J_range=(0.5, 1.5))
    F, L = 16, 2
    graph, model, theta, th, Ah = _setup(torch, g, F, L, prec, scale=0.6, max_layers=3)
    s = W.random_spins(g.n_sites, 23, seed=4)
    E, dl = gna.local_energy(graph, model, theta, torch.tensor(s, device="cuda"), mode, bonds=True)
    E = E.cpu().numpy()
    want = _oracle_eloc(th, F, L, Ah, g, s)
    _close(E[:, 0] + 1j * E[:, 1], want, TOL[prec], SC.eloc_scale(th, F, L, Ah, g.edges, g.J, s))
    # per-bond Re Delta (float32 output), 0 on parallel bonds
    d = hz.bond_log_ratios(lambda x: gcn.logpsi_complex(th, F, L, Ah, x), g.edges, s)
    want_d = np.where(np.isnan(d.real), 0.0, d.real)
    assert np.all(np.abs(dl.cpu().numpy() - want_d) <= TOL[prec] * SC.delta_scale(th, F, L, Ah, g.edges, s) +
                  2.0 ** -24 * np.abs(want_d) + TOL[prec])


def test_local_energy_unshared_weights(torch):
    g = W.erdos_renyi(16, 0.3, seed=9)
    F, L = 8, 3
    graph, model, theta, th, Ah = _setup(torch, g, F, L, gna.PREC_FP64, shared=False, scale=0.5)
    s = W.random_spins(g.n_sites, 9, seed=3)
    for mode in (gna.ELOC_FULL, gna.ELOC_INCREMENTAL):
        E = gna.local_energy(graph, model, theta, torch.tensor(s, device="cuda"), mode).cpu().numpy()
        _close(E[:, 0] + 1j * E[:, 1], _oracle_eloc(th, F, L, Ah, g, s, False), 1e-10)


def test_two_site_gcn_local_energy_is_quarter(torch):
    g = W.two_site()
    graph, model, theta, th, Ah = _setup(torch, g, 4, 2, gna.PREC_FP64, scale=1.0)
    s = torch.tensor([[1, -1], [-1, 1]], dtype=torch.int8, device="cuda")
    for mode in (gna.ELOC_FULL, gna.ELOC_INCREMENTAL):
        E = gna.local_energy(graph, model, theta, s, mode).cpu().numpy()
        assert np.abs(E[:, 0] - 0.25).max() < 1e-15 and np.abs(E[:, 1]).max() < 1e-15


def test_incremental_matches_full_fp32_kagome108(torch):
    # Kagome 6x6x3, L = 4, F = 32: incremental vs full re-evaluation, and the oracle on a subset
    g = W.kagome(6)
    F, L = 32, 4
    graph, model, theta, th, Ah = _setup(torch, g, F, L, gna.PREC_FP32, scale=0.1)
    s = W.random_spins(g.n_sites, 300, seed=1)
    st = torch.tensor(s, device="cuda")
    Ei = gna.local_energy(graph, model, theta, st, gna.ELOC_INCREMENTAL).cpu().numpy()
    Ef = gna.local_energy(graph, model, theta, st, gna.ELOC_FULL).cpu().numpy()
    want = _oracle_eloc(th, F, L, Ah, g, s[:6])
    _close(Ei[:6, 0] + 1j * Ei[:6, 1], want, 1e-5, SC.eloc_scale(th, F, L, Ah, g.edges, g.J, s[:6]))
    # two FP32 paths, each within 1e-5 of the terms' magnitude (from the kernel's own Delta)
    _, dl = gna.local_energy(graph, model, theta, st, gna.ELOC_INCREMENTAL, bonds=True)
    dl = dl.cpu().numpy()
    anti = s[:, g.edges[:, 0]] != s[:, g.edges[:, 1]]
    sc = (0.25 * np.abs(g.J)[None, :]).sum(axis=1)[:, None] + (anti * 0.5 * np.exp(dl)).sum(axis=1)[:, None]
    _close(Ei, Ef, 2e-5, sc)
    assert abs(Ei[:, 0].mean() - Ef[:, 0].mean()) <= 1e-4 * abs(Ef[:, 0].mean())


# ---------------------------------------------------------------------------------
# Metropolis
# ---------------------------------------------------------------------------------

def test_metropolis_fp64_trajectories_match_oracle(torch):
    g = W.kagome(2)
    F, L = 16, 2
    graph, model, theta, th, Ah = _setup(torch, g, F, L, gna.PREC_FP64, scale=0.8)
    C, sweeps, seed, step0 = 12, 3, 1234, 7
    s0 = W.random_spins(g.n_sites, C, seed=2)
    ch = torch.tensor(s0, device="cuda")
    samples, lpo, acc, tr = gna.metropolis_sweep(graph, model, theta, ch, sweeps, 1, seed, step0, trace=True)
    lp_fn = lambda x: gcn.logpsi_complex(th, F, L, Ah, x)  # noqa: E731
    s_o, samp_o, lp_o, acc_o, tr_o = sampler.run_chains(lp_fn, g.edges, s0, seed, step0, sweeps, 1)
    tr = tr.cpu().numpy()
    # near-ties |u - exp(2 Re Delta)| < 1e-12 would make the decision precision-dependent: expect none
    assert np.array_equal(tr[:, :, 0], tr_o[:, :, 0])  # bonds
    assert np.array_equal(np.isnan(tr[:, :, 2]), np.isnan(tr_o[:, :, 2]))
    m = ~np.isnan(tr_o[:, :, 2])
    assert np.abs(tr[:, :, 2][m] - tr_o[:, :, 2][m]).max() < 1e-10
    assert np.array_equal(tr[:, :, 1], tr_o[:, :, 1])  # decisions
    assert np.array_equal(samples.cpu().numpy(), samp_o)
    assert np.array_equal(ch.cpu().numpy(), s_o)
    assert np.array_equal(acc.cpu().numpy(), acc_o)
    lpo = lpo.cpu().numpy()
    _close(lpo[..., 0] + 1j * lpo[..., 1], lp_o, 1e-10)


@pytest.mark.parametrize("prec", [gna.PREC_FP32, gna.PREC_FP64])
def test_metropolis_decisions_given_uniforms_and_ratios(torch, prec):
    # every step: bond = hi64(r0 * E) of the oracle's Philox, decision = u < exp(2 Re Delta)
    # evaluated by the oracle in the kernel's precision on the kernel's own Re Delta
    g = W.triangular(4, 4)
    F, L = 16, 2
    graph, model, theta, th, Ah = _setup(torch, g, F, L, prec, scale=1.0)
    C, sweeps, seed, step0 = 9, 2, 99, 1000
    s0 = W.random_spins(g.n_sites, C, seed=3)
    ch = torch.tensor(s0, device="cuda")
    _, _, acc, tr = gna.metropolis_sweep(graph, model, theta, ch, sweeps, 0, seed, step0, trace=True)
    tr = tr.cpu().numpy()
    pname = "fp64" if prec == gna.PREC_FP64 else "fp32"
    s = s0.copy()
    near = 0
    for c in range(C):
        for k in range(tr.shape[1]):
            w = sampler.step_words(seed, c, step0 + k)
            e = sampler.bond_index(w[0], g.n_edges)
            assert int(tr[c, k, 0]) == e
            i, j = g.edges[e]
            if s[c, i] == s[c, j]:
                assert np.isnan(tr[c, k, 2]) and tr[c, k, 1] == 0
                continue
            u = sampler.uniform(w[1], pname)
            dre = tr[c, k, 2]
            if abs(float(u) - np.exp(2 * dre)) < 1e-6:
                near += 1
                continue
            assert bool(tr[c, k, 1]) == sampler.accept(u, dre, pname)
            if tr[c, k, 1]:
                s[c, [i, j]] = s[c, [j, i]]
    assert near <= 2
    assert np.array_equal(ch.cpu().numpy(), s)
    assert np.all((s > 0).sum(1) == g.n_sites // 2)
    assert acc.cpu().numpy().sum() == tr[:, :, 1].sum()


@pytest.mark.parametrize("prec", [gna.PREC_FP32, gna.PREC_FP64])
def test_metropolis_kagome108_records_match_forward(torch, prec):
    # Kagome 6x6x3, L = 4, F = 32: the sampler's recorded log Psi (from its incrementally
    # updated pre-activations) equals a fresh forward of the recorded configurations
    g = W.kagome(6)
    F, L = 32, 4
    graph, model, theta, th, Ah = _setup(torch, g, F, L, prec, scale=0.3)
    ch = torch.tensor(W.random_spins(g.n_sites, 40, seed=9), device="cuda")
    samples, lpo, acc, tr = gna.metropolis_sweep(graph, model, theta, ch, 3, 1, 11, 0, trace=True)
    x = samples.cpu().numpy()
    assert np.all((x > 0).sum(-1) == g.n_sites // 2)
    assert acc.cpu().numpy().sum() > 0
    for r in range(3):
        want = gna.forward(graph, model, theta, samples[r].contiguous()).cpu().numpy()
        _close(lpo[r].cpu().numpy(), want, 1e-10 if prec == gna.PREC_FP64 else 1e-5)
    if prec == gna.PREC_FP64:
        # and the oracle on a few of them
        _close(lpo[-1].cpu().numpy()[:3], gcn.logpsi(th, F, L, Ah, x[-1][:3]), 1e-10)


def test_metropolis_resume_is_bit_identical(torch):
    # counter-based randomness: 2 sweeps then 3 sweeps from step0 + 2N equals 5 sweeps at once
    g = W.kagome(2)
    graph, model, theta, th, Ah = _setup(torch, g, 16, 2, gna.PREC_FP32, scale=0.8)
    s0 = torch.tensor(W.random_spins(g.n_sites, 20, seed=5), device="cuda")
    a = s0.clone()
    gna.metropolis_sweep(graph, model, theta, a, 5, 0, 7, 0)
    b = s0.clone()
    gna.metropolis_sweep(graph, model, theta, b, 2, 0, 7, 0)
    gna.metropolis_sweep(graph, model, theta, b, 3, 0, 7, 2 * g.n_sites)
    assert torch.equal(a, b)


# ---------------------------------------------------------------------------------
# backward and ISGO
# ---------------------------------------------------------------------------------

@pytest.mark.parametrize("prec", [gna.PREC_FP64, gna.PREC_FP32])
@pytest.mark.parametrize("shared", [True, False])
def test_backward_parity(torch, prec, shared):
    g = W.erdos_renyi(18, 0.25, seed=2)
    F, L = 16, 3
    graph, model, theta, th, Ah = _setup(torch, g, F, L, prec, shared, scale=0.5)
    s = W.random_spins(g.n_sites, 41, seed=6)
    cot = np.random.default_rng(1).normal(size=(41, 2))
    got = gna.backward(graph, model, theta, torch.tensor(s, device="cuda"),
                       torch.tensor(cot, device="cuda")).cpu().numpy()
    want = isgo.backward(th, F, L, Ah, s, cot, shared)
    _close(got, want, TOL[prec], SC.grad_scale(th, F, L, Ah, s, cot, shared))


def test_backward_matches_finite_differences_triangular144(torch):
    # triangular 12x12, L = 4, F = 48, FP64: the hand-written backward against central
    # differences (h = 1e-6) of sum_x cot_x . log Psi_x computed by the forward kernel
    g = W.triangular(12, 12)
    F, L = 48, 4
    graph, model, theta, th, Ah = _setup(torch, g, F, L, gna.PREC_FP64, scale=0.2)
    s = torch.tensor(W.random_spins(g.n_sites, 6, seed=3), device="cuda")
    cot = torch.tensor(np.random.default_rng(2).normal(size=(6, 2)), device="cuda")
    grad = gna.backward(graph, model, theta, s, cot).cpu().numpy()
    idx = np.random.default_rng(5).choice(model.num_params, 24, replace=False)
    h = 1e-6
    for k in idx:
        tp = theta.clone()
        tp[k] += h
        tm = theta.clone()
        tm[k] -= h
        fp = (gna.forward(graph, model, tp, s) * cot).sum().item()
        fm = (gna.forward(graph, model, tm, s) * cot).sum().item()
        fd = (fp - fm) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, grad[k])


def test_autograd_function_uses_library_backward(torch):
    g = W.kagome(2)
    F, L = 8, 2
    graph, model, theta, th, Ah = _setup(torch, g, F, L, gna.PREC_FP64, scale=0.5)
    s = torch.tensor(W.random_spins(g.n_sites, 7, seed=1), device="cuda")
    t = theta.clone().requires_grad_(True)
    lp = gna.gcn_logpsi(t, s, graph, model)
    w = torch.randn(7, 2, dtype=torch.float64, device="cuda")
    (lp * w).sum().backward()
    want = isgo.backward(th, F, L, Ah, s.cpu().numpy(), w.cpu().numpy())
    _close(t.grad.cpu().numpy(), want, 1e-10)


def test_isgo_weights_parity(torch):
    rng = np.random.default_rng(3)
    Bn = 5000
    lp = rng.normal(size=(Bn, 2)) * 3
    lp0 = rng.normal(size=(Bn, 2)) * 3
    E = rng.normal(size=(Bn, 2))
    counts = rng.integers(1, 5, size=Bn).astype(float)
    T = lambda x: torch.tensor(x, device="cuda")  # noqa: E731
    cot, stats = gna.isgo_weights(T(lp), T(lp0), T(E), T(counts))
    p = isgo.weights(lp[:, 0] + 1j * lp[:, 1], lp0[:, 0] + 1j * lp0[:, 1], counts)
    Ebar, var, ess = isgo.statistics(p, E[:, 0] + 1j * E[:, 1], counts)
    st = stats.cpu().numpy()
    _close(st, [Ebar.real, Ebar.imag, var, ess], 1e-12)
    _close(cot.cpu().numpy(), isgo.cotangents(p, E[:, 0] + 1j * E[:, 1], Ebar), 1e-12)


@pytest.mark.parametrize("prec", [gna.PREC_FP64, gna.PREC_FP32])
def test_isgo_grad_parity(torch, prec):
    g = W.kagome(2)
    F, L = 16, 2
    graph, model, theta, th, Ah = _setup(torch, g, F, L, prec, scale=0.5)
    th0 = th - W.random_theta(F, L, seed=9, scale=0.02)
    s = W.random_spins(g.n_sites, 64, seed=8)
    lp0 = gcn.logpsi(th0, F, L, Ah, s)
    grad, stats = gna.isgo_grad(graph, model, theta, torch.tensor(s, device="cuda"), torch.tensor(lp0, device="cuda"))
    g_o, Ebar, var, ess, E, p = isgo.isgo_gradient(th, F, L, Ah, g.edges, g.J, s, lp0[:, 0] + 1j * lp0[:, 1])
    tol = TOL[prec]
    _close(grad.cpu().numpy(), g_o, tol, SC.grad_scale(th, F, L, Ah, s, isgo.cotangents(p, E, Ebar)))
    st = stats.cpu().numpy()
    _close(st[:2], [Ebar.real, Ebar.imag], tol, float((p * SC.eloc_scale(th, F, L, Ah, g.edges, g.J, s)).sum()))
    assert abs(st[3] - ess) <= tol * ess


def test_isgo_reuse_loop_replays_oracle_fp64(torch):
    # Kagome 2x2x3, F = 16, L = 2: ten reuse steps (isgo_grad + SGD) on fixed samples give
    # the oracle's theta trajectory (isgo_gradient + sgd in FP64).  Bound: each FP64 gradient
    # is within 1e-9 relative of the oracle's (the gradient parity bound), so ten steps of
    # lr = 0.02 move theta apart by at most 10 * 0.02 * 1e-9 * |g|, below 1e-9 * max|theta|
    g = W.kagome(2)
    F, L = 16, 2
    graph, model, theta, th, Ah = _setup(torch, g, F, L, gna.PREC_FP64, scale=0.5)
    s = W.random_spins(g.n_sites, 256, seed=21)
    lp0 = gcn.logpsi(th, F, L, Ah, s)
    st, l0 = torch.tensor(s, device="cuda"), torch.tensor(lp0, device="cuda")
    th_o = th.copy()
    for _ in range(10):
        grad, _ = gna.isgo_grad(graph, model, theta, st, l0)
        gna.sgd_update(model, theta, grad, 0.02)
        g_o = isgo.isgo_gradient(th_o, F, L, Ah, g.edges, g.J, s, lp0[:, 0] + 1j * lp0[:, 1])[0]
        th_o = isgo.sgd(th_o, g_o, 0.02)
    _close(theta.cpu().numpy(), th_o, 1e-9)


def test_isgo_training_kagome12_respects_the_variational_bound(torch):
    # Kagome 2x2x3 (S_z = 0 sector of 924 states, ED E0 = -5.4449), F = 16, L = 2, FP64,
    # 1024 chains: ISGO iterations (2 sweeps, K = 10 reuse steps) from weight scale 0.5 lower
    # the exact enumerated energy E_v(theta) far below its start, E_v stays >= E0, and the
    # chains' weighted mean agrees with E_v
    from paper_2011_12453_gb300 import vmc

    g = W.kagome(2)
    F, L = 16, 2
    graph, model, theta, th, Ah = _setup(torch, g, F, L, gna.PREC_FP64, scale=0.5)
    Hs, codes = hz.sector_hamiltonian(g.n_sites, g.edges, g.J)
    sall = hz.codes_to_spins(codes, g.n_sites)
    E0 = np.linalg.eigvalsh(Hs.toarray())[0]

    def exact(t):
        return hz.variational_energy(gcn.logpsi_complex(t, F, L, Ah, sall), Hs).real

    Ev_start = exact(th)
    ch = vmc.Chains(graph, model, theta, W.random_spins(g.n_sites, 1024, seed=2), seed=3)
    ch.sweep(20)
    for _ in range(30):
        st = vmc.isgo_iteration(ch, K=10, lr=0.01, sweeps=2)
    Ev = exact(theta.cpu().numpy())
    assert Ev >= E0 - 1e-9
    assert Ev < Ev_start - 2.0, (Ev_start, Ev)
    samples, _, _, _ = ch.sweep(40, record_every=2)
    E = gna.local_energy(graph, model, theta, samples.reshape(-1, g.n_sites).contiguous(),
                         gna.ELOC_FULL).cpu().numpy()[:, 0].reshape(20, 1024)
    m = E.mean(axis=0)
    assert abs(m.mean() - Ev) < 5 * m.std() / np.sqrt(len(m)) + 1e-3, (m.mean(), Ev)
    print("kagome12 ISGO: E_v start %.4f -> %.4f, chains %.4f, ED %.4f" % (Ev_start, Ev, m.mean(), E0))


def test_sgd_update(torch):
    m = gna.Model(16, 2, gna.PREC_FP32)
    th = torch.randn(m.num_params, device="cuda")
    gr = torch.randn(m.num_params, dtype=torch.float64, device="cuda")
    want = (th.double() - 0.01 * gr).float()
    gna.sgd_update(m, th, gr, 0.01)
    assert torch.allclose(th, want, rtol=0, atol=1e-7)


def test_workspace_too_small_is_an_error(torch):
    g = W.kagome(6)
    graph, model, theta, th, Ah = _setup(torch, g, 64, 4, gna.PREC_FP64)  # cache does not fit smem
    s = torch.tensor(W.random_spins(g.n_sites, 4, seed=1), device="cuda")
    need = gna.workspace_size(graph, model, gna.OP_ELOC_INCR, 4)
    assert need > 0
    E = torch.empty((4, 2), dtype=torch.float64, device="cuda")
    st = gna.lib().gna_local_energy(graph.handle, gna.ctypes.byref(model.desc), theta.data_ptr(), s.data_ptr(), 4,
                                    gna.ELOC_INCREMENTAL, E.data_ptr(), None, None, 0, None)
    assert st == gna.GNA_ERR_WORKSPACE
