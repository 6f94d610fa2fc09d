"""Pins of the oracle's ISGO gradient (Eq. isgo of arXiv:2011.12453, read as the
textbook covariance gradient) and of its hand-written backward: finite differences of
log Psi, the exact gradient of the enumerated variational energy, reduction to plain VMC
(Eq. vmc), duplicate grouping with counts, and exact zero-gradient invariants."""
import numpy as np
import pytest

from oracle import gcn, heisenberg as hz, isgo
from paper_2011_12453_gb300 import workloads as W


@pytest.mark.parametrize("shared", [True, False])
def test_backward_matches_central_differences(shared):
    g = W.erdos_renyi(9, 0.4, seed=1)
    F, L = 3, 3
    th = W.random_theta(F, L, seed=2, scale=0.6, shared=shared)
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    s = W.random_spins(g.n_sites, 4, seed=3)
    cot = np.random.default_rng(4).normal(size=(4, 2))
    grad = isgo.backward(th, F, L, Ah, s, cot, shared)

    def f(t):
        return (gcn.logpsi(t, F, L, Ah, s, shared) * cot).sum()

    h = 1e-6
    fd = np.empty_like(th)
    for k in range(th.size):
        e = np.zeros_like(th)
        e[k] = h
        fd[k] = (f(th + e) - f(th - e)) / (2 * h)
    np.testing.assert_allclose(grad, fd, rtol=1e-6, atol=1e-8)


def _exact_setup(F=3, L=2):
    g = W.kagome(2)
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    Hs, codes = hz.sector_hamiltonian(g.n_sites, g.edges, g.J)
    s = hz.codes_to_spins(codes, g.n_sites)
    return g, Ah, Hs, s


def test_isgo_gradient_equals_exact_gradient():
    F, L = 3, 2
    g, Ah, Hs, s = _exact_setup(F, L)
    th0 = W.random_theta(F, L, seed=10, scale=0.8)
    th = th0 + W.random_theta(F, L, seed=11, scale=0.05)  # moved parameters: reweighting matters
    lp0 = gcn.logpsi_complex(th0, F, L, Ah, s)
    # all sector states as samples, counts proportional to |Psi^0|^2 (fractional counts)
    counts = np.exp(2 * (lp0.real - lp0.real.max()))
    grad, Ebar, var, ess, E, p = isgo.isgo_gradient(th, F, L, Ah, g.edges, g.J, s, lp0, counts)

    def Ev(t):
        return hz.variational_energy(gcn.logpsi_complex(t, F, L, Ah, s), Hs).real

    assert abs(Ebar - hz.variational_energy(gcn.logpsi_complex(th, F, L, Ah, s), Hs)) < 1e-12
    h = 1e-6
    fd = np.array([(Ev(th + h * e) - Ev(th - h * e)) / (2 * h) for e in np.eye(th.size)])
    scale = np.abs(fd).max()
    np.testing.assert_allclose(grad, fd, rtol=0, atol=1e-7 * max(scale, 1e-3))


def test_reduces_to_vmc_at_theta0():
    F, L = 3, 2
    g = W.kagome(2)
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    th = W.random_theta(F, L, seed=3, scale=0.5)
    s = W.random_spins(g.n_sites, 40, seed=5)
    lp = gcn.logpsi_complex(th, F, L, Ah, s)
    grad, Ebar, var, ess, E, p = isgo.isgo_gradient(th, F, L, Ah, g.edges, g.J, s, lp)
    np.testing.assert_allclose(p, 1.0 / 40, rtol=1e-14)
    assert abs(ess - 40) < 1e-9
    # Eq. (vmc) with uniform weights: 2 Re[<E* O> - <E>* <O>] using per-sample log-derivatives
    O = np.stack([isgo.backward(th, F, L, Ah, s[b:b + 1], np.array([[1.0, 0.0]])) +
                  1j * isgo.backward(th, F, L, Ah, s[b:b + 1], np.array([[0.0, 1.0]])) for b in range(40)])
    want = 2 * ((np.conj(E)[:, None] * O).mean(0) - np.conj(E.mean()) * O.mean(0)).real
    np.testing.assert_allclose(grad, want, rtol=1e-10, atol=1e-12)


def test_grouping_duplicates_with_counts():
    F, L = 3, 2
    g = W.kagome(2)
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    th0 = W.random_theta(F, L, seed=6, scale=0.5)
    th = th0 + W.random_theta(F, L, seed=7, scale=0.05)
    uniq = W.random_spins(g.n_sites, 7, seed=8)
    reps = np.array([1, 3, 2, 1, 5, 1, 2])
    dup = np.repeat(uniq, reps, axis=0)
    lp0u = gcn.logpsi_complex(th0, F, L, Ah, uniq)
    lp0d = gcn.logpsi_complex(th0, F, L, Ah, dup)
    a = isgo.isgo_gradient(th, F, L, Ah, g.edges, g.J, uniq, lp0u, reps.astype(float))
    b = isgo.isgo_gradient(th, F, L, Ah, g.edges, g.J, dup, lp0d)
    np.testing.assert_allclose(a[0], b[0], rtol=1e-10, atol=1e-12)
    assert abs(a[1] - b[1]) < 1e-13 and abs(a[2] - b[2]) < 1e-13
    assert abs(a[3] - b[3]) < 1e-9 * a[3]  # the IS-ESS is defined per copy, so grouping keeps it


def test_zero_gradient_invariants():
    # b_r shifts log Psi by a constant (normalisation / global phase), and the one-hot
    # readout rows see the constant (N_up, N_down) of the sector: their gradient is zero.
    F, L = 4, 2
    g = W.triangular(3, 4)
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    th0 = W.random_theta(F, L, seed=1, scale=0.7)
    th = th0 + W.random_theta(F, L, seed=2, scale=0.1)
    s = W.random_spins(g.n_sites, 30, seed=3)
    lp0 = gcn.logpsi_complex(th0, F, L, Ah, s)
    grad = isgo.isgo_gradient(th, F, L, Ah, g.edges, g.J, s, lp0)[0]
    P = grad.size
    b_r = grad[P - 2:]
    onehot_rows = grad[P - 2 - 2 * (F + 2) + 2 * F:P - 2]
    assert np.abs(b_r).max() < 1e-13
    assert np.abs(onehot_rows).max() < 1e-12
    assert np.abs(grad).max() > 1e-6  # the rest is not trivially zero


def test_weights_are_overflow_safe():
    lp = np.array([1000.0 + 0j, 999.0 + 0j, -1000.0 + 0j])
    p = isgo.weights(lp, np.zeros(3, complex))
    assert np.all(np.isfinite(p)) and abs(p.sum() - 1) < 1e-15
    np.testing.assert_allclose(p[1] / p[0], np.exp(-2.0), rtol=1e-14)
