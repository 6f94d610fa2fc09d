"""Pins of the oracle's local energy, sector Hamiltonian and ED (local energy
E_x = sum_x' H_xx' Psi_x'/Psi_x of the scaling section, arXiv:2011.12453, on the
Heisenberg model) against closed forms, an independent Kronecker-product Hamiltonian,
the zero-variance property and the variational principle."""
import json
import os

import numpy as np
import pytest

from oracle import gcn, heisenberg as hz
from paper_2011_12453_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _closed_forms():
    with open(os.path.join(GOLDEN, "heisenberg_closed_forms.json")) as f:
        return json.load(f)


def test_two_site_spectrum():
    cf = _closed_forms()["two_site"]
    g = W.two_site()
    w, _, _ = hz.ground_state(2, g.edges, g.J, k=2)
    np.testing.assert_allclose(w, [cf["singlet"], cf["triplet_m0"]], atol=1e-14)


def test_ring4():
    g = W.ring(4)
    w, _, _ = hz.ground_state(4, g.edges, g.J)
    assert abs(w[0] - _closed_forms()["ring4"]) < 1e-13


@pytest.mark.parametrize("n", [4, 6, 8, 10, 12])
def test_complete_graph_closed_form(n):
    # H = J/2 (S_tot^2 - sum S_i^2) -> E0 = -3 n J / 8 for even n (S_tot = 0)
    g = W.complete(n)
    w, _, _ = hz.ground_state(n, g.edges, g.J)
    assert abs(w[0] + 3.0 * n / 8.0) < 1e-12


@pytest.mark.parametrize("a,b", [(2, 2), (3, 5), (1, 5), (4, 6)])
def test_complete_bipartite_closed_form(a, b):
    # H = J S_A . S_B = J/2 (S^2 - S_A^2 - S_B^2), ground state S_A = a/2, S_B = b/2, S = |a-b|/2
    g = W.complete_bipartite(a, b)
    w, _, _ = hz.ground_state(a + b, g.edges, g.J)
    SA, SB = a / 2, b / 2
    S = abs(SA - SB)
    want = 0.5 * (S * (S + 1) - SA * (SA + 1) - SB * (SB + 1))
    assert abs(w[0] - want) < 1e-12


def _kron_hamiltonian(n, edges, J):
    sx = np.array([[0, 1], [1, 0]]) / 2.0
    sy = np.array([[0, -1j], [1j, 0]]) / 2.0
    sz = np.array([[1, 0], [0, -1]]) / 2.0

    def op(o, site):
        # basis index bit v = 1 <=> site v up, site 0 the least significant bit of the kron order;
        # the matrices above use (up, down) order, so conjugate by the bit flip to get (down, up)
        flip = np.array([[0, 1], [1, 0]])
        mats = [flip @ o @ flip if v == site else np.eye(2) for v in range(n)]
        out = np.array([[1.0]])
        for v in reversed(range(n)):
            out = np.kron(out, mats[v])
        return out

    H = np.zeros((2 ** n, 2 ** n), dtype=np.complex128)
    for (i, j), Jij in zip(edges.tolist(), J.tolist()):
        for o in (sx, sy, sz):
            H += Jij * op(o, i) @ op(o, j)
    return H


@pytest.mark.parametrize("graph", ["ring6", "er7"])
def test_sector_hamiltonian_matches_kronecker(graph):
    g = W.ring(6) if graph == "ring6" else W.erdos_renyi(7, 0.5, seed=2, J_range=(0.5, 1.5))
    n = g.n_sites
    Hs, codes = hz.sector_hamiltonian(n, g.edges, g.J)
    Hk = _kron_hamiltonian(n, g.edges, g.J)
    sub = Hk[np.ix_(codes, codes)]
    assert np.abs(sub.imag).max() < 1e-14
    np.testing.assert_allclose(Hs.toarray(), sub.real, atol=1e-14)
    # no matrix element leaves the sector
    mask = np.ones(2 ** n, bool)
    mask[codes] = False
    assert np.abs(Hk[np.ix_(mask, codes)]).max() < 1e-14


def test_zero_variance_with_exact_ground_state():
    g = W.kagome(2)
    w, v, codes = hz.ground_state(g.n_sites, g.edges, g.J)
    table = {int(c): v[k] for k, c in enumerate(codes)}

    def lp_fn(s):
        vals = np.array([table[int(c)] for c in hz.spins_to_codes(s)], dtype=np.complex128)
        with np.errstate(divide="ignore"):
            return np.log(vals)

    s = hz.codes_to_spins(codes, g.n_sites)
    keep = np.abs(v) > 1e-6 * np.abs(v).max()
    E = hz.local_energy(lp_fn, g.edges, g.J, s[keep])
    np.testing.assert_allclose(E.real, w[0], rtol=0, atol=1e-9)
    assert np.abs(E.imag).max() < 1e-9


@pytest.mark.parametrize("sign,energy_key", [(-1.0, "singlet"), (1.0, "triplet_m0")])
def test_two_site_tabulated(sign, energy_key):
    cf = _closed_forms()["two_site"]
    g = W.two_site()
    table = {(1, -1): 1.0, (-1, 1): sign}

    def lp_fn(s):
        return np.log(np.array([table[tuple(int(a) for a in x)] for x in s], dtype=np.complex128))

    E = hz.local_energy(lp_fn, g.edges, g.J, np.array([[1, -1], [-1, 1]], dtype=np.int8))
    np.testing.assert_allclose(E, [cf[energy_key]] * 2, atol=1e-15)


def test_two_site_gcn_is_triplet():
    # sum-pooling is invariant under the site swap, so the GCN gives Psi(ud) = Psi(du): E_loc = +1/4
    g = W.two_site()
    F, L = 4, 2
    th = W.random_theta(F, L, seed=3, scale=1.0)
    Ah = gcn.norm_adjacency(gcn.adjacency(2, g.edges))
    E = hz.local_energy(lambda s: gcn.logpsi_complex(th, F, L, Ah, s), g.edges, g.J,
                        np.array([[1, -1], [-1, 1]], dtype=np.int8))
    np.testing.assert_allclose(E, [0.25, 0.25], atol=1e-15)


def _geoms():
    return [W.kagome(2), W.triangular(3, 4), W.erdos_renyi(12, 0.5, seed=7)]


@pytest.mark.parametrize("gi", [0, 1, 2])
def test_enumeration_identity_and_variational_bound(gi):
    g = _geoms()[gi]
    F, L = 4, 2
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    Hs, codes = hz.sector_hamiltonian(g.n_sites, g.edges, g.J)
    E0 = np.linalg.eigvalsh(Hs.toarray())[0]
    s = hz.codes_to_spins(codes, g.n_sites)
    for seed in range(3):
        th = W.random_theta(F, L, seed=seed, scale=0.8)

        def lp_fn(x):
            return gcn.logpsi_complex(th, F, L, Ah, x)

        lp = lp_fn(s)
        Ev = hz.variational_energy(lp, Hs)
        Eloc = hz.local_energy(lp_fn, g.edges, g.J, s)
        w = np.exp(2 * (lp.real - lp.real.max()))
        mean = (w * Eloc).sum() / w.sum()
        assert abs(mean - Ev) < 1e-12 * max(1.0, abs(Ev))
        assert Ev.real >= E0 - 1e-12
        assert abs(Ev.imag) < 1e-12


def test_local_energy_matches_matrix_row():
    g = W.erdos_renyi(8, 0.5, seed=4, J_range=(0.5, 1.5))
    F, L = 3, 2
    th = W.random_theta(F, L, seed=6, scale=1.0)
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    Hs, codes = hz.sector_hamiltonian(g.n_sites, g.edges, g.J)
    s = hz.codes_to_spins(codes, g.n_sites)
    psi = np.exp(gcn.logpsi_complex(th, F, L, Ah, s))
    want = (Hs @ psi) / psi
    got = hz.local_energy(lambda x: gcn.logpsi_complex(th, F, L, Ah, x), g.edges, g.J, s)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


def test_ed_golden_energies():
    with open(os.path.join(GOLDEN, "ed_energies.json")) as f:
        gold = json.load(f)
    g = W.kagome(2)
    w, _, _ = hz.ground_state(g.n_sites, g.edges, g.J, k=2)
    np.testing.assert_allclose(w, gold["kagome_2x2x3"]["E"][:2], atol=1e-12)
    t = W.triangular(3, 4)
    w, _, _ = hz.ground_state(t.n_sites, t.edges, t.J)
    assert abs(w[0] - gold["triangular_3x4"]["E"][0]) < 1e-12
