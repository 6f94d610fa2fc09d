"""GPU parity of the tensor-core path (tcgen05 GEMMs, FP32 accumulation) against the FP64
oracle run on the same parameters with the GEMM weights W rounded to BF16 (W is a BF16
model parameter), so the stated error is that of the activations' rounding.  Both
tensor-core precisions: BF16 (single BF16 operands) and BF16X2 (each FP32 operand as
hi + lo BF16 values, FP32 rows, tanh from its Taylor series).

Tolerances are derived from the arithmetic, not from measurements (tests/bounds.py):
  log Psi     the forward's roundings propagated to the readout (shared embedding rounding
              exactly, the independent roundings as 6 standard deviations); BF16 also at
              most 2e-2 relative (the stated BF16 tolerance on log Psi).
  Delta       per bond the same propagation through the incremental difference form, plus
              the float32 rounding of the returned value.
  E_loc       per sample sum_e |J_e|/2 |exp(Delta_e)| (exp(b_e) - 1) for the bounds b_e, plus
              the float32 rounding of each term.
  backward    per parameter 2^-14 sum_x |cot_x| |d log Psi_x / d theta| (the split operands
              carry 16 significant bits; four rounded operands per product), plus FP32
              accumulation.
"""
import numpy as np
import pytest

from oracle import gcn, heisenberg as hz, isgo
from paper_2011_12453_gb300 import build as B, gna, workloads as W

import bounds as BD

MODES = {gna.PREC_BF16: "bf16", gna.PREC_BF16X2: "bf16x2"}

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t

    B.build()
    t.cuda.set_device(0)
    return t


def _round_W_bf16(torch, th, F, L):
    """theta with the GCN weight matrix W rounded to BF16 (the GEMM operand)."""
    out = th.copy()
    o = 3 * F
    w = torch.tensor(out[o:o + 2 * F * F], dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    out[o:o + 2 * F * F] = w
    return out


def _setup(torch, g, F, L, seed=0, scale=0.1, prec=gna.PREC_BF16):
    th = W.random_theta(F, L, seed=seed, scale=scale)
    graph = gna.Graph.from_workload(g, L)
    model = gna.Model(F, L, prec)
    theta = torch.tensor(th, dtype=torch.float32, device="cuda")
    th_or = _round_W_bf16(torch, theta.double().cpu().numpy(), F, L)
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    return graph, model, theta, th_or, Ah


CASES = [("kagome2", 16, 2), ("kagome6", 32, 4), ("tri12", 48, 4), ("tri6", 64, 3), ("er40", 32, 3)]


def _graph(name):
    return {"kagome2": W.kagome(2), "kagome6": W.kagome(6), "tri12": W.triangular(12, 12), "tri6": W.triangular(6, 6),
            "er40": W.erdos_renyi(40, 0.1, seed=3, J_range=(0.5, 1.5))}[name]


@pytest.mark.parametrize("prec", [gna.PREC_BF16, gna.PREC_BF16X2])
@pytest.mark.parametrize("name,F,L", CASES)
def test_bf16_forward_parity(torch, name, F, L, prec):
    g = _graph(name)
    graph, model, theta, th, Ah = _setup(torch, g, F, L, scale=0.3, prec=prec)
    for Bn in (33, 1):
        s = W.random_spins(g.n_sites, Bn, seed=7 + Bn)
        got = gna.forward(graph, model, theta, torch.tensor(s, device="cuda")).cpu().numpy()
        want = gcn.logpsi(th, F, L, Ah, s)
        err = np.abs(got - want).sum(axis=1)
        bound = BD.forward_bound(th, F, L, Ah, s, MODES[prec]) + 1e-12 * np.abs(want).sum(axis=1)
        assert np.all(err <= bound), (err.max(), bound[np.argmax(err - bound)])
        if prec == gna.PREC_BF16:
            assert err.max() <= 2e-2 * max(1.0, np.abs(want).max())


def _check_eloc(torch, g, F, L, prec, scale, seed, n=6):
    graph, model, theta, th, Ah = _setup(torch, g, F, L, scale=scale, prec=prec)
    s = W.random_spins(g.n_sites, n, seed=seed)
    E, dl = gna.local_energy(graph, model, theta, torch.tensor(s, device="cuda"), gna.ELOC_INCREMENTAL, bonds=True)
    E = E.cpu().numpy()
    Ec = E[:, 0] + 1j * E[:, 1]
    delta, bd, eb = BD.bond_bounds(th, F, L, Ah, g.edges, g.J, s, MODES[prec])
    want = hz.local_energy(lambda x: gcn.logpsi_complex(th, F, L, Ah, x), g.edges, g.J, s)
    anti = ~np.isnan(delta.real)
    want_d = np.where(anti, delta.real, 0.0)
    got_d = dl.cpu().numpy()
    # per bond: the derived bound plus the float32 rounding of the returned Delta
    lim = bd + 2.0 ** -23 * np.abs(want_d)
    assert np.all(np.abs(got_d - want_d) <= lim), np.max(np.abs(got_d - want_d) - lim)
    assert np.all(got_d[~anti] == 0.0)
    # per sample: the propagated bond bounds plus the float32 rounding of each term
    terms = 0.5 * np.abs(np.where(anti, g.J[None, :], 0.0)) * np.abs(np.exp(np.where(anti, delta, 0.0)))
    elim = eb + 2.0 ** -21 * terms.sum(axis=1) + 1e-12 * np.abs(want)
    assert np.all(np.abs(Ec - want) <= elim), np.max(np.abs(Ec - want) - elim)
    return np.abs(Ec - want) / np.abs(want).clip(1.0)


@pytest.mark.parametrize("prec", [gna.PREC_BF16, gna.PREC_BF16X2])
@pytest.mark.parametrize("name,F,L", CASES)
def test_bf16_local_energy_parity(torch, name, F, L, prec):
    # weight scale 0.3: saturating units, |Delta log Psi| up to ~3
    _check_eloc(torch, _graph(name), F, L, prec, 0.3, 11)


@pytest.mark.parametrize("prec", [gna.PREC_BF16, gna.PREC_BF16X2])
@pytest.mark.parametrize("name,F,L", CASES)
def test_bf16_local_energy_benchmark_scale(torch, name, F, L, prec):
    # the benchmark's weight scale 0.1: a nearly flat wavefunction, small Delta
    rel = _check_eloc(torch, _graph(name), F, L, prec, 0.1, 12)
    if prec == gna.PREC_BF16X2:
        assert rel.max() <= 1e-5, rel.max()


def test_bf16_incremental_mean_energy_matches_fp32_full(torch):
    # Kagome 6x6x3, L = 4, F = 32: batch-mean energy agreement <= 1e-4 relative
    g = W.kagome(6)
    F, L = 32, 4
    graph, model, theta, th, Ah = _setup(torch, g, F, L, scale=0.1)
    m32 = gna.Model(F, L, gna.PREC_FP32)
    s = torch.tensor(W.random_spins(g.n_sites, 4096, seed=2), device="cuda")
    Eb = gna.local_energy(graph, model, theta, s, gna.ELOC_INCREMENTAL).cpu().numpy()
    Ef = gna.local_energy(graph, m32, theta, s, gna.ELOC_FULL).cpu().numpy()
    assert abs(Eb[:, 0].mean() - Ef[:, 0].mean()) <= 1e-4 * abs(Ef[:, 0].mean())
    assert np.max(np.abs(Eb[:, 0] - Ef[:, 0]) / np.abs(Ef[:, 0])) <= 2e-3


def test_bf16_two_site_is_quarter(torch):
    g = W.two_site()
    graph, model, theta, th, Ah = _setup(torch, g, 16, 2, scale=0.3)
    E = gna.local_energy(graph, model, theta, torch.tensor([[1, -1], [-1, 1]], dtype=torch.int8, device="cuda"),
                         gna.ELOC_INCREMENTAL).cpu().numpy()
    # exact value 1/4 (the GCN cannot tell the two sites apart); Delta is formed from BF16
    # differences, so the per-sample BF16 tolerance (2e-2 on the ratio, J/2 = 1/2) applies
    assert np.abs(E[:, 0] - 0.25).max() < 1e-2 and np.all(np.isfinite(E))


def test_bf16_unshared_is_unsupported(torch):
    g = W.kagome(2)
    graph = gna.Graph.from_workload(g, 2)
    model = gna.Model(16, 2, gna.PREC_BF16, shared=False)
    with pytest.raises(gna.GnaError) as ei:
        gna.workspace_size(graph, model, gna.OP_ELOC_INCR, 4)
    assert ei.value.status == gna.GNA_ERR_UNSUPPORTED


def test_bf16_device_status_clean(torch):
    g = W.kagome(6)
    graph, model, theta, th, Ah = _setup(torch, g, 32, 4)
    s = torch.tensor(W.random_spins(g.n_sites, 300, seed=5), device="cuda")
    gna.local_energy(graph, model, theta, s, gna.ELOC_INCREMENTAL)
    assert gna.device_status(clear=True) == 0


# ---------------------------------------------------------------------------------
# Metropolis sweeps on the tensor cores (BF16 models, plain moves)
# ---------------------------------------------------------------------------------

def _replay(g, s0, tr, seed, step0):
    """Replay the kernel's trace with the oracle's Philox words: the bond of every step,
    the no-op on parallel bonds, the decision u < exp(2 Re Delta) on the kernel's own
    Delta with the FP32 uniform; returns the states before each step and the near-tie count."""
    from oracle import sampler

    C, K = tr.shape[0], tr.shape[1]
    s = s0.copy()
    before = np.empty((C, K, g.n_sites), dtype=np.int8)
    near = 0
    for c in range(C):
        for k in range(K):
            before[c, k] = s[c]
            w = sampler.step_words(seed, c, step0 + k)
            e = sampler.bond_index(w[0], g.n_edges)
            assert int(tr[c, k, 0]) == e, (c, k)
            assert tr[c, k, 3] == 1.0
            i, j = g.edges[e]
            if s[c, i] == s[c, j]:
                assert np.isnan(tr[c, k, 2]) and tr[c, k, 1] == 0
                continue
            u = sampler.uniform(w[1], "fp32")
            dre = tr[c, k, 2]
            if abs(float(u) - np.exp(2 * dre)) < 1e-6:
                near += 1
            else:
                assert bool(tr[c, k, 1]) == sampler.accept(u, dre, "fp32"), (c, k)
            if tr[c, k, 1]:
                s[c, [i, j]] = s[c, [j, i]]
    return s, before, near


@pytest.mark.parametrize("name,F,L", [("kagome2", 16, 2), ("kagome6", 32, 4), ("tri6", 64, 3)])
def test_bf16_sampler_bookkeeping_and_ratios(torch, name, F, L):
    # bonds and no-ops bit-exact, decisions exact given the kernel's Delta, configurations and
    # acceptance counts consistent with the replay; Delta of every antiparallel proposal
    # within the BF16 benchmark-scale tolerance of the oracle on the state it was made from
    g = _graph(name)
    graph, model, theta, th, Ah = _setup(torch, g, F, L, scale=0.1)
    C, sweeps, seed, step0 = 9 if name == "kagome2" else 5, 2, 31, 77
    s0 = W.random_spins(g.n_sites, C, seed=4)
    ch = torch.tensor(s0, device="cuda")
    _, _, acc, tr = gna.metropolis_sweep(graph, model, theta, ch, sweeps, 0, seed, step0, trace=True)
    tr = tr.cpu().numpy()
    s, before, near = _replay(g, s0, tr, seed, step0)
    assert near <= 2
    assert np.array_equal(ch.cpu().numpy(), s)
    assert acc.cpu().numpy().sum() == tr[:, :, 1].sum() > 0
    anti = ~np.isnan(tr[:, :, 2])
    cs, ks = np.nonzero(anti)
    pick = np.random.default_rng(0).choice(len(cs), size=min(40, len(cs)), replace=False)
    states = before[cs[pick], ks[pick]]
    d = hz.bond_log_ratios(lambda x: gcn.logpsi_complex(th, F, L, Ah, x), g.edges, states)
    want = d.real[np.arange(len(pick)), tr[cs[pick], ks[pick], 0].astype(int)]
    assert np.abs(tr[cs[pick], ks[pick], 2] - want).max() <= 2e-3


def test_bf16_sampler_records_match_forward(torch):
    # Kagome 6x6x3, L = 4, F = 32: recorded samples conserve S_z and the recorded log Psi
    # (from the incrementally updated FP32 pre-activations) matches a fresh BF16 forward
    g = W.kagome(6)
    F, L = 32, 4
    graph, model, theta, th, Ah = _setup(torch, g, F, L, scale=0.3)
    ch = torch.tensor(W.random_spins(g.n_sites, 300, seed=9), device="cuda")
    samples, lpo, acc, _ = gna.metropolis_sweep(graph, model, theta, ch, 3, 1, 11, 0)
    x = samples.cpu().numpy()
    assert np.all((x > 0).sum(-1) == g.n_sites // 2)
    assert np.array_equal(x[-1], ch.cpu().numpy())
    assert acc.cpu().numpy().sum() > 0
    for r in range(3):
        want = gna.forward(graph, model, theta, samples[r].contiguous()).cpu().numpy()
        assert np.abs(lpo[r].cpu().numpy() - want).max() <= 2e-2 * max(1.0, np.abs(want).max())
    want = gcn.logpsi(th, F, L, Ah, x[-1][:4])
    assert np.abs(lpo[-1].cpu().numpy()[:4] - want).max() <= 2e-2 * max(1.0, np.abs(want).max())


def test_bf16_sampler_matches_fp32_sampler_statistics(torch):
    # same move rule, Delta in BF16 vs FP32: the mean local energy of the two samplers'
    # chains agrees within 4 combined standard errors (Kagome 2x2x3, F = 16, L = 2)
    g = W.kagome(2)
    F, L = 16, 2
    graph, model, theta, th, Ah = _setup(torch, g, F, L, scale=0.8)
    m32 = gna.Model(F, L, gna.PREC_FP32)
    res = {}
    for name, md in (("bf16", model), ("fp32", m32)):
        ch = torch.tensor(W.random_spins(g.n_sites, 2048, seed=1), device="cuda")
        gna.metropolis_sweep(graph, md, theta, ch, 20, 0, 5, 0)
        samples, _, _, _ = gna.metropolis_sweep(graph, md, theta, ch, 40, 4, 5, 20 * g.n_sites)
        E = gna.local_energy(graph, m32, theta, samples.reshape(-1, g.n_sites).contiguous(),
                             gna.ELOC_FULL).cpu().numpy()[:, 0].reshape(10, 2048)
        m = E.mean(axis=0)
        res[name] = (m.mean(), m.std() / np.sqrt(len(m)))
    (a, sa), (b, sb) = res["bf16"], res["fp32"]
    assert abs(a - b) < 4 * np.hypot(sa, sb), (res)


# ---------------------------------------------------------------------------------
# backward VJP on the tensor cores
# ---------------------------------------------------------------------------------

@pytest.mark.parametrize("scale", [0.3, 0.1])
@pytest.mark.parametrize("name,F,L", CASES)
def test_bf16_backward_parity(torch, name, F, L, scale):
    # sum_x cot_x . d log Psi_x / d theta with split (hi + lo) BF16 operands and FP32
    # accumulation against the FP64 oracle on the BF16-rounded W; bound per parameter
    # 2^-14 sum_x |cot_x . d log Psi_x / d theta| (condition of the sum over samples times the
    # operand precision) + the FP32 accumulation
    g = _graph(name)
    graph, model, theta, th, Ah = _setup(torch, g, F, L, scale=scale)
    Bn = 37
    s = W.random_spins(g.n_sites, Bn, seed=13)
    cot = np.random.default_rng(14).normal(size=(Bn, 2))
    got = gna.backward(graph, model, theta, torch.tensor(s, device="cuda"), torch.tensor(cot, device="cuda"))
    want = isgo.backward(th, F, L, Ah, s, cot)
    per = np.stack([np.abs(isgo.backward(th, F, L, Ah, s[x:x + 1], cot[x:x + 1])) for x in range(Bn)])
    kappa = per.sum(axis=0)
    err = np.abs(got.cpu().numpy() - want)
    lim = 2.0 ** -14 * kappa + 2.0 ** -20 * np.abs(want).max()
    assert np.all(err <= lim), (np.max(err - lim), err.max() / np.abs(want).max())


def test_bf16_backward_matches_fp32_on_the_benchmark_workload(torch):
    # Kagome 6x6x3, L = 4, F = 32, weight scale 0.1, 2048 configurations: BF16 tensor-core
    # backward vs the FP32 backward on the same parameters, and an empty batch gives zeros
    g = W.kagome(6)
    F, L = 32, 4
    graph, model, theta, th, Ah = _setup(torch, g, F, L, scale=0.1)
    m32 = gna.Model(F, L, gna.PREC_FP32)
    s = torch.tensor(W.random_spins(g.n_sites, 2048, seed=3), device="cuda")
    cot = torch.tensor(np.random.default_rng(4).normal(size=(2048, 2)) / 2048, device="cuda")
    a = gna.backward(graph, model, theta, s, cot).cpu().numpy()
    b = gna.backward(graph, m32, theta, s, cot).cpu().numpy()
    # the FP32 backward differentiates the FP32 W, the tensor-core one the BF16 W: the
    # gradients differ by the weight rounding (relative 2^-9 of W) at first order
    assert np.abs(a - b).max() <= 2.0 ** -7 * np.abs(b).max()
    z = gna.backward(graph, model, theta, s[:0], cot[:0]).cpu().numpy()
    assert np.all(z == 0)
