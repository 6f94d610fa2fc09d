"""Metropolis pair-exchange sampling of P ~ |Psi|^2.  TEST INFRASTRUCTURE ONLY.

The scaling section of arXiv:2011.12453 samples states with MCMC following
P_x ~ |Psi_x|^2; the paper does not give the move set.  Reading adopted here (a
Metropolis chain on the fixed-S_z sector):

* Random words come from Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
  numbers: as easy as 1, 2, 3", SC'11), restated below from that definition: key
  (seed, chain), counter (t, 0, 0, 0) for absolute step t of the chain, output
  (r0, r1, r2, r3).
* Bond choice e = floor(r0 * |E| / 2^64) (the high word of the 128-bit product), so
  every bond is proposed with probability 1/|E| up to a 2^-64 bias; the proposal is
  symmetric.
* A parallel bond is a rejected step.  For an antiparallel bond the move exchanges
  s_i and s_j and is accepted iff u < exp(2 Re(log Psi(s') - log Psi(s))), with
  u = (r1 >> 11) * 2^-53 in float64 or u = (r1 >> 40) * 2^-24 in float32.
* A sweep is n_sites steps; after each recorded sweep the chain's state and its
  log Psi are written out.
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
PHILOX_M0 = 0xD2E7470EE14C6C93
PHILOX_M1 = 0xCA5A826395121157
PHILOX_W0 = 0x9E3779B97F4A7C15
PHILOX_W1 = 0xBB67AE8584CAA73B


def philox4x64_10(key: tuple[int, int], ctr: tuple[int, int, int, int]) -> tuple[int, int, int, int]:
    """One Philox4x64 block with 10 rounds (the published SC'11 construction)."""
    c0, c1, c2, c3 = (int(x) & MASK64 for x in ctr)
    k0, k1 = (int(x) & MASK64 for x in key)
    for r in range(10):
        if r:
            k0 = (k0 + PHILOX_W0) & MASK64
            k1 = (k1 + PHILOX_W1) & MASK64
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> 64, p0 & MASK64
        hi1, lo1 = p1 >> 64, p1 & MASK64
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def step_words(seed: int, chain: int, t: int) -> tuple[int, int, int, int]:
    return philox4x64_10((seed, chain), (t, 0, 0, 0))


def bond_index(r0: int, n_edges: int) -> int:
    return (int(r0) * int(n_edges)) >> 64


def uniform(r1: int, precision: str = "fp64"):
    if precision == "fp64":
        return np.float64((int(r1) >> 11) * 2.0 ** -53)
    return np.float32((int(r1) >> 40) * 2.0 ** -24)


def accept(u, dre, precision: str = "fp64") -> bool:
    """Metropolis test for |Psi(s')|^2/|Psi(s)|^2 = exp(2 Re Delta), strict '<'."""
    if precision == "fp64":
        return bool(np.float64(u) < np.exp(2.0 * np.float64(dre)))
    with np.errstate(over="ignore"):
        return bool(np.float32(u) < np.exp(np.float32(2.0) * np.float32(dre)))


def run_chains(logpsi_fn, edges: np.ndarray, spins0: np.ndarray, seed: int, step0: int,
               n_sweeps: int, record_every: int = 1, precision: str = "fp64"):
    """Advance every chain by n_sweeps * n_sites steps, chains in lock step.

    logpsi_fn maps int8 (B, n) -> complex (B,).  Returns (final spins, samples
    [n_rec][C][n], logpsi of samples [n_rec][C] complex, accepted counts [C], trace) where
    trace[c][k] = (bond, accepted, Re Delta or NaN for a parallel bond).
    """
    s = np.array(spins0, dtype=np.int8, copy=True)
    C, n = s.shape
    e = np.asarray(edges)
    E = e.shape[0]
    lp = logpsi_fn(s)
    n_steps = n_sweeps * n
    samples, sample_lp = [], []
    acc = np.zeros(C, dtype=np.int64)
    trace = np.zeros((C, n_steps, 3))
    for k in range(n_steps):
        t = step0 + k
        words = [step_words(seed, c, t) for c in range(C)]
        bonds = np.array([bond_index(w[0], E) for w in words])
        i, j = e[bonds, 0], e[bonds, 1]
        anti = s[np.arange(C), i] != s[np.arange(C), j]
        trace[:, k, 0] = bonds
        trace[:, k, 2] = np.nan
        if anti.any():
            idx = np.nonzero(anti)[0]
            sw = s[idx].copy()
            sw[np.arange(len(idx)), i[idx]] = s[idx, j[idx]]
            sw[np.arange(len(idx)), j[idx]] = s[idx, i[idx]]
            lp_new = logpsi_fn(sw)
            delta = lp_new - lp[idx]
            for m, c in enumerate(idx):
                dre = delta[m].real
                if precision == "fp32":
                    dre = np.float32(dre)
                trace[c, k, 2] = dre
                if accept(uniform(words[c][1], precision), dre, precision):
                    s[c] = sw[m]
                    lp[c] = lp_new[m]
                    acc[c] += 1
                    trace[c, k, 1] = 1
        if (k + 1) % n == 0 and record_every > 0 and ((k + 1) // n) % record_every == 0:
            samples.append(s.copy())
            sample_lp.append(logpsi_fn(s))
    samples = np.array(samples, dtype=np.int8).reshape(-1, C, n)
    sample_lp = np.array(sample_lp).reshape(-1, C)
    return s, samples, sample_lp, acc, trace


def transition_matrix(logpsi_values: np.ndarray, codes: np.ndarray, edges: np.ndarray) -> np.ndarray:
    """Exact transition matrix of the plain pair-exchange chain on a sector basis.

    Bond proposed with probability 1/|E|; acceptance min(1, |Psi_b|^2/|Psi_a|^2).
    """
    lp = np.asarray(logpsi_values)
    index = {int(c): k for k, c in enumerate(np.asarray(codes).tolist())}
    M, E = len(codes), len(edges)
    T = np.zeros((M, M))
    for a, c in enumerate(np.asarray(codes).tolist()):
        for i, j in np.asarray(edges).tolist():
            if ((c >> i) & 1) == ((c >> j) & 1):
                T[a, a] += 1.0 / E
                continue
            b = index[c ^ ((1 << i) | (1 << j))]
            ratio = min(1.0, float(np.exp(2.0 * (lp[b].real - lp[a].real))))
            T[a, b] += ratio / E
            T[a, a] += (1.0 - ratio) / E
    return T
