"""Heisenberg local energy, S_z-sector Hamiltonian, ED and E_v.  TEST INFRASTRUCTURE ONLY.

The scaling section of arXiv:2011.12453 defines the local energy of a sampled state x
as E_x = sum_x' H_xx' Psi_x' / Psi_x, and the variational energy
E_v(w) = <Psi|H|Psi> / <Psi|Psi>.  The Hamiltonian used here is the antiferromagnetic
Heisenberg model H = sum_<ij> J_ij S_i . S_j with S = sigma/2.  In the basis of
S^z eigenstates (spins s = +-1) this gives, per bond (i, j):

* diagonal element J/4 * s_i * s_j;
* for an antiparallel pair, an off-diagonal element J/2 to the state with s_i and s_j
  exchanged (from (S+_i S-_j + S-_i S+_j)/2).

so E_loc(s) = sum_e J_e/4 s_i s_j + sum_{e: s_i != s_j} J_e/2 Psi(s^e)/Psi(s), with the
ratio taken as exp(log Psi(s^e) - log Psi(s)) for complex log Psi.  The local energy
below is the definition, evaluated by full re-evaluation of log Psi at every s^e.

Bond Hamiltonians of the XXZ family (the paper's hard-core bosons among them) are given
by per-bond coefficients xxz = (Jz, Jxy, hz, c):

  H_e = Jz S^z_i S^z_j + Jxy/2 (S^+_i S^-_j + S^-_i S^+_j) + hz (S^z_i + S^z_j) + c,

i.e. diagonal element Jz/4 s_i s_j + hz/2 (s_i + s_j) + c and off-diagonal element Jxy/2
for an antiparallel pair.  Heisenberg: (J, J, 0, 0).  Hard-core bosons
H = -t sum (b^+_i b_j + h.c.) + V sum n_i n_j (numerical-experiments section) with
n = (1 + s)/2 and b^+ <-> S^+: V n_i n_j = V/4 (1 + s_i + s_j + s_i s_j) and the hopping
is -t (S^+_i S^-_j + h.c.), so (Jz, Jxy, hz, c) = (V, -2t, V/2, V/4).
"""
from __future__ import annotations

from typing import Callable

import numpy as np
import scipy.sparse
import scipy.sparse.linalg


def heisenberg_xxz(J) -> tuple:
    """(Jz, Jxy, hz, c) of the Heisenberg bonds J."""
    J = np.asarray(J, dtype=np.float64)
    return J, J, np.zeros_like(J), np.zeros_like(J)


def hardcore_bosons(n_edges: int, t: float, V: float) -> tuple:
    """(Jz, Jxy, hz, c) of -t (b^+_i b_j + h.c.) + V n_i n_j on every bond."""
    one = np.ones(n_edges)
    return V * one, -2.0 * t * one, V / 2.0 * one, V / 4.0 * one


def _xxz(J, xxz):
    return heisenberg_xxz(J) if xxz is None else tuple(np.asarray(a, dtype=np.float64) for a in xxz)


def diagonal_energy(edges: np.ndarray, J: np.ndarray, spins: np.ndarray, xxz=None) -> np.ndarray:
    """sum_e [Jz_e/4 s_i s_j + hz_e/2 (s_i + s_j) + c_e] for each row of spins (B, n) -> (B,);
    with xxz None, the Heisenberg sum_e J_e/4 s_i s_j."""
    s = np.atleast_2d(spins).astype(np.float64)
    e = np.asarray(edges)
    Jz, _, hz, c = _xxz(J, xxz)
    si, sj = s[:, e[:, 0]], s[:, e[:, 1]]
    return (si * sj * (Jz / 4.0) + (si + sj) * (hz / 2.0) + c).sum(axis=1)


def local_energy(logpsi_fn: Callable[[np.ndarray], np.ndarray], edges: np.ndarray, J: np.ndarray,
                 spins: np.ndarray, xxz=None) -> np.ndarray:
    """Complex E_loc for each row of spins, by full re-evaluation of log Psi.

    logpsi_fn maps int8 (B, n) -> complex (B,).  Returns complex128 (B,).  The off-diagonal
    element of an antiparallel bond is Jxy/2 (J/2 for Heisenberg bonds).
    """
    s = np.atleast_2d(np.asarray(spins, dtype=np.int8))
    e = np.asarray(edges)
    _, Jxy, _, _ = _xxz(J, xxz)
    lp = logpsi_fn(s)
    out = diagonal_energy(e, J, s, xxz).astype(np.complex128)
    for k in range(e.shape[0]):
        i, j = int(e[k, 0]), int(e[k, 1])
        anti = s[:, i] != s[:, j]
        if not anti.any():
            continue
        sw = s[anti].copy()
        sw[:, [i, j]] = sw[:, [j, i]]
        out[anti] += Jxy[k] / 2.0 * np.exp(logpsi_fn(sw) - lp[anti])
    return out


def bond_log_ratios(logpsi_fn, edges, spins) -> np.ndarray:
    """log Psi(s^e) - log Psi(s) for every bond e (complex, NaN for parallel bonds): (B, E)."""
    s = np.atleast_2d(np.asarray(spins, dtype=np.int8))
    e = np.asarray(edges)
    lp = logpsi_fn(s)
    out = np.full((s.shape[0], e.shape[0]), np.nan + 0j)
    for k in range(e.shape[0]):
        i, j = int(e[k, 0]), int(e[k, 1])
        anti = s[:, i] != s[:, j]
        if anti.any():
            sw = s[anti].copy()
            sw[:, [i, j]] = sw[:, [j, i]]
            out[anti, k] = logpsi_fn(sw) - lp[anti]
    return out


# ---------------------------------------------------------------------------
# S_z-sector Hamiltonian from bit operations (independent of local_energy)
# ---------------------------------------------------------------------------

def sector_codes(n: int, n_up: int) -> np.ndarray:
    """Integer codes (bit v = 1 <=> site v up) with n_up set bits, increasing."""
    return np.array([c for c in range(1 << n) if bin(c).count("1") == n_up], dtype=np.int64)


def codes_to_spins(codes: np.ndarray, n: int) -> np.ndarray:
    bits = (codes[:, None] >> np.arange(n)[None, :]) & 1
    return np.where(bits == 1, 1, -1).astype(np.int8)


def spins_to_codes(spins: np.ndarray) -> np.ndarray:
    s = np.atleast_2d(spins)
    return ((s > 0).astype(np.int64) << np.arange(s.shape[1])[None, :]).sum(axis=1)


def sector_hamiltonian(n: int, edges: np.ndarray, J: np.ndarray, n_up: int | None = None, xxz=None):
    """Sparse H restricted to the sector with n_up up spins, and its basis codes (Heisenberg
    bonds J, or XXZ bonds (Jz, Jxy, hz, c))."""
    n_up = n // 2 if n_up is None else n_up
    codes = sector_codes(n, n_up)
    index = {int(c): k for k, c in enumerate(codes)}
    Jz, Jxy, hz, cc = (a.tolist() for a in _xxz(J, xxz))
    rows, cols, vals = [], [], []
    for k, c in enumerate(codes.tolist()):
        diag = 0.0
        for b, (i, j) in enumerate(np.asarray(edges).tolist()):
            zi, zj = 0.5 if (c >> i) & 1 else -0.5, 0.5 if (c >> j) & 1 else -0.5  # S^z eigenvalues
            diag += Jz[b] * zi * zj + hz[b] * (zi + zj) + cc[b]
            if zi != zj:
                flipped = c ^ ((1 << i) | (1 << j))
                rows.append(k)
                cols.append(index[flipped])
                vals.append(Jxy[b] / 2.0)
        rows.append(k)
        cols.append(k)
        vals.append(diag)
    M = len(codes)
    H = scipy.sparse.coo_matrix((vals, (rows, cols)), shape=(M, M)).tocsr()
    return H, codes


def ground_state(n: int, edges, J, n_up: int | None = None, k: int = 1, xxz=None):
    """Lowest k eigenvalues (ascending) and the ground-state vector in the sector."""
    H, codes = sector_hamiltonian(n, edges, J, n_up, xxz)
    if H.shape[0] <= 4000:
        w, v = np.linalg.eigh(H.toarray())
        return w[:k], v[:, 0], codes
    w, v = scipy.sparse.linalg.eigsh(H, k=max(k, 2), which="SA", tol=1e-13)
    order = np.argsort(w)
    return w[order][:k], v[:, order[0]], codes


def variational_energy(logpsi_values: np.ndarray, H) -> complex:
    """<Psi|H|Psi>/<Psi|Psi> for log Psi given on every basis state of the sector.

    The amplitudes are rescaled by the largest Re log Psi before exponentiation.
    """
    lp = np.asarray(logpsi_values, dtype=np.complex128)
    psi = np.exp(lp - lp.real.max())
    return complex(np.vdot(psi, H @ psi) / np.vdot(psi, psi))
