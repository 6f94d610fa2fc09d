"""Pins of the oracle's XXZ bonds and the hard-core boson model of the numerical-experiments
section (oracle/heisenberg.py): closed forms (two sites, free hard-core bosons on a ring via
the Jordan-Wigner mapping, the classical limit), the reduction to the Heisenberg bonds, an
independent Kronecker-product construction, and the local-energy identities."""
import numpy as np
import scipy.sparse as sp

from oracle import gcn, heisenberg as hz
from paper_2011_12453_gb300 import workloads as W


def _ring(n):
    return np.array([[i, (i + 1) % n] for i in range(n)], dtype=np.int32)


def test_two_sites_one_boson():
    # H = -t (b1^+ b2 + h.c.) + V n1 n2 with one particle: [[0, -t], [-t, 0]] -> E0 = -t
    e = np.array([[0, 1]], dtype=np.int32)
    for t, V in [(1.0, 0.0), (0.7, 3.0)]:
        w, _, _ = hz.ground_state(2, e, None, n_up=1, k=2, xxz=hz.hardcore_bosons(1, t, V))
        np.testing.assert_allclose(w, [-t, t], atol=1e-12)


def test_free_hardcore_bosons_on_a_ring_match_jordan_wigner_fermions():
    # V = 0: hard-core bosons on a ring are free fermions with periodic (odd particle
    # number) or antiperiodic (even) boundary conditions; E0 = -2t sum of the lowest cos k
    for n, npart in [(8, 4), (10, 5), (9, 3)]:
        t = 1.3
        w, _, _ = hz.ground_state(n, _ring(n), None, n_up=npart, xxz=hz.hardcore_bosons(n, t, 0.0))
        phase = 0.0 if npart % 2 == 1 else 0.5
        eps = np.sort(-2 * t * np.cos(2 * np.pi * (np.arange(n) + phase) / n))
        np.testing.assert_allclose(w[0], eps[:npart].sum(), atol=1e-10)


def test_classical_limit():
    # t = 0: diagonal; the best half filling of an even ring has no neighbouring pair
    n = 8
    w, _, _ = hz.ground_state(n, _ring(n), None, n_up=4, xxz=hz.hardcore_bosons(n, 0.0, 2.0))
    assert abs(w[0]) < 1e-12
    w, _, _ = hz.ground_state(n, _ring(n), None, n_up=5, xxz=hz.hardcore_bosons(n, 0.0, 2.0))
    # five particles and three holes: at most three runs of particles, so 5 - 3 = 2 pairs
    assert abs(w[0] - 2 * 2.0) < 1e-12


def test_xxz_with_heisenberg_coefficients_is_heisenberg():
    g = W.erdos_renyi(10, 0.35, seed=2, J_range=(0.5, 1.5))
    H1, _ = hz.sector_hamiltonian(g.n_sites, g.edges, g.J)
    H2, _ = hz.sector_hamiltonian(g.n_sites, g.edges, None, xxz=hz.heisenberg_xxz(g.J))
    assert abs(H1 - H2).max() < 1e-14


def test_sector_matrix_against_kronecker_construction():
    # boson H from creation/annihilation matrices on the full 2^n space, restricted to N
    n, t, V = 6, 0.8, 1.7
    e = _ring(n)
    bdag = sp.csr_matrix(np.array([[0.0, 0.0], [1.0, 0.0]]))  # |1><0| (occupied = up = bit 1)
    num = sp.csr_matrix(np.array([[0.0, 0.0], [0.0, 1.0]]))

    def site(op, k):
        mats = [sp.identity(2, format="csr")] * n
        mats[k] = op
        out = mats[n - 1]
        for m in reversed(mats[:-1]):
            out = sp.kron(out, m, format="csr")
        return out  # bit k of the basis index is site k

    H = sp.csr_matrix((1 << n, 1 << n))
    for i, j in e:
        hop = site(bdag, i) @ site(bdag.T, j)
        H = H - t * (hop + hop.T) + V * (site(num, i) @ site(num, j))
    Hs, codes = hz.sector_hamiltonian(n, e, None, n_up=3, xxz=hz.hardcore_bosons(n, t, V))
    ref = H.toarray()[np.ix_(codes, codes)]
    np.testing.assert_allclose(Hs.toarray(), ref, atol=1e-13)


def test_local_energy_identities_for_bosons():
    g = W.kagome(2)
    F, L, t, V = 8, 2, 1.0, 2.5
    xxz = hz.hardcore_bosons(g.n_edges, t, V)
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    th = W.random_theta(F, L, seed=3, scale=0.6)
    H, codes = hz.sector_hamiltonian(g.n_sites, g.edges, None, xxz=xxz)
    s = hz.codes_to_spins(codes, g.n_sites)
    lp = gcn.logpsi_complex(th, F, L, Ah, s)
    E = hz.local_energy(lambda x: gcn.logpsi_complex(th, F, L, Ah, x), g.edges, None, s, xxz=xxz)
    p = np.exp(2 * (lp.real - lp.real.max()))
    np.testing.assert_allclose((p * E).sum() / p.sum(), hz.variational_energy(lp, H), atol=1e-11)
    # zero variance with the ground state as Psi (positive: no sign problem for bosons)
    w, v, _ = hz.ground_state(g.n_sites, g.edges, None, xxz=xxz)
    assert np.all(v * np.sign(v[0]) > 0)
    table = dict(zip(codes.tolist(), np.log(np.abs(v)).tolist()))
    Eg = hz.local_energy(lambda x: np.array([table[c] for c in hz.spins_to_codes(x).tolist()], dtype=complex),
                         g.edges, None, s, xxz=xxz)
    np.testing.assert_allclose(Eg.real, w[0], atol=1e-10)
