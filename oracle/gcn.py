"""GCN wavefunction log Psi(s) in plain numpy float64.  TEST INFRASTRUCTURE ONLY.

Follows the GNA section of arXiv:2011.12453:

* Eq. (gcn):  H^(l+1) = f([D^-1/2 A D^-1/2 H^(l) ; H^(l)] W + b), W in R^{2F x F},
  b in R^F, with W and b shared across the GCN layers.
* The state is one-hot encoded per site and transformed by a dense layer and f into
  F-wide embeddings (H^0).
* Readout: the output H^L is concatenated with the one-hot input, summed over all
  sites and mapped by a dense layer to log Psi.  The dense layer has two units, read
  as (Re log Psi, Im log Psi): the two-head (amplitude, angle) form the conclusion
  proposes for complex wavefunctions.

Nonlinearity f (argument ``act``):
* "tanh": f = tanh applied elementwise (the configurations built here).
* "relu_ln": the paper's f, ReLU followed by a layer normalisation over the F features
  of each node row, r = max(y, 0), f(y) = (r - mean r) / sqrt(mean (r - mean r)^2 + eps).
  The paper gives neither eps nor an affine part: eps = 1e-6 (LN_EPS), no affine (the
  next layer's W and b, or the readout, absorb a per-feature scale and shift).

Readings where the paper is silent:
* The embedding's nonlinear transform is a dense layer followed by the same f.
* A is the binary adjacency (couplings J do not enter the network), without
  self-loops; an isolated site has an all-zero row in D^-1/2 A D^-1/2.
* onehot(+1) = (1, 0) and onehot(-1) = (0, 1); spin +1 is the occupied site
  n = (1 + s)/2 of the boson language.
* Flat parameter layout: [W_e (2 x F), b_e (F), {W (2F x F), b (F)} x (1 if shared
  else L), w_r ((F+2) x 2), b_r (2)], all row-major.  W rows 0..F-1 multiply the
  message D^-1/2 A D^-1/2 H and rows F..2F-1 multiply H, the concatenation order of
  Eq. (gcn).
"""
from __future__ import annotations

import numpy as np


def adjacency(n: int, edges: np.ndarray) -> np.ndarray:
    """Binary symmetric adjacency matrix A (n x n) of an edge list."""
    A = np.zeros((n, n), dtype=np.float64)
    for a, b in np.asarray(edges).tolist():
        if a == b:
            raise ValueError("self-loop")
        if A[a, b] != 0:
            raise ValueError("duplicate edge")
        A[a, b] = 1.0
        A[b, a] = 1.0
    return A


def norm_adjacency(A: np.ndarray) -> np.ndarray:
    """D^-1/2 A D^-1/2 with D the degree matrix (isolated sites give zero rows)."""
    d = A.sum(axis=1)
    inv = np.zeros_like(d)
    nz = d > 0
    inv[nz] = 1.0 / np.sqrt(d[nz])
    return inv[:, None] * A * inv[None, :]


def num_params(F: int, L: int, shared: bool = True) -> int:
    n_layers = 1 if shared else L
    return 2 * F + F + n_layers * (2 * F * F + F) + (F + 2) * 2 + 2


def unpack(theta: np.ndarray, F: int, L: int, shared: bool = True) -> dict:
    """Views into the flat parameter vector, following the layout in the module doc."""
    theta = np.asarray(theta, dtype=np.float64)
    if theta.shape != (num_params(F, L, shared),):
        raise ValueError(f"theta has shape {theta.shape}, expected ({num_params(F, L, shared)},)")
    o = 0

    def take(shape):
        nonlocal o
        size = int(np.prod(shape))
        out = theta[o:o + size].reshape(shape)
        o += size
        return out

    p = {"W_e": take((2, F)), "b_e": take((F,))}
    n_layers = 1 if shared else L
    Ws, bs = [], []
    for _ in range(n_layers):
        Ws.append(take((2 * F, F)))
        bs.append(take((F,)))
    if shared:
        Ws, bs = Ws * L, bs * L
    p["W"], p["b"] = Ws, bs
    p["w_r"] = take((F + 2, 2))
    p["b_r"] = take((2,))
    assert o == theta.size
    return p


def onehot(spins: np.ndarray) -> np.ndarray:
    """(..., n) of +-1 -> (..., n, 2): +1 -> (1, 0), -1 -> (0, 1)."""
    s = np.asarray(spins)
    return np.stack([(s > 0), (s < 0)], axis=-1).astype(np.float64)


LN_EPS = 1e-6
ACTS = ("tanh", "relu_ln")


def activation(Y: np.ndarray, act: str = "tanh") -> np.ndarray:
    """f applied to pre-activations Y (..., F): tanh, or ReLU then layer norm over the last axis."""
    if act == "tanh":
        return np.tanh(Y)
    if act != "relu_ln":
        raise ValueError(act)
    r = np.maximum(Y, 0.0)
    c = r - r.mean(axis=-1, keepdims=True)
    return c / np.sqrt((c * c).mean(axis=-1, keepdims=True) + LN_EPS)


def layers(theta, F: int, L: int, Ahat: np.ndarray, spins: np.ndarray, shared: bool = True, act: str = "tanh"):
    """All node-embedding layers [H^0, ..., H^L], each (B, n, F), for a batch of states."""
    p = unpack(theta, F, L, shared)
    x = onehot(np.atleast_2d(spins))
    H = activation(x @ p["W_e"] + p["b_e"], act)
    out = [H]
    for l in range(L):
        msg = np.einsum("vu,buf->bvf", Ahat, H)
        H = activation(np.concatenate([msg, H], axis=-1) @ p["W"][l] + p["b"][l], act)
        out.append(H)
    return out


def logpsi(theta, F: int, L: int, Ahat: np.ndarray, spins: np.ndarray, shared: bool = True,
           act: str = "tanh") -> np.ndarray:
    """(B, 2) float64: columns (Re log Psi, Im log Psi) for each state of the batch."""
    p = unpack(theta, F, L, shared)
    x = onehot(np.atleast_2d(spins))
    H = layers(theta, F, L, Ahat, spins, shared, act)[-1]
    z = np.concatenate([H, x], axis=-1).sum(axis=1)  # (B, F+2): sum-pool over sites
    return z @ p["w_r"] + p["b_r"]


def logpsi_complex(theta, F, L, Ahat, spins, shared=True, act="tanh") -> np.ndarray:
    lp = logpsi(theta, F, L, Ahat, spins, shared, act)
    return lp[:, 0] + 1j * lp[:, 1]


def _f_loops(row, act):
    """f of one node row (a list of F floats), written with scalar loops."""
    if act == "tanh":
        return [float(np.tanh(y)) for y in row]
    r = [y if y > 0.0 else 0.0 for y in row]
    mu = sum(r) / len(r)
    var = sum((x - mu) ** 2 for x in r) / len(r)
    inv = 1.0 / np.sqrt(var + LN_EPS)
    return [(x - mu) * inv for x in r]


def logpsi_loops(theta, F: int, L: int, n: int, edges: np.ndarray, spins_1d, shared: bool = True,
                 act: str = "tanh") -> np.ndarray:
    """Same function for ONE state, written with per-site loops over the edge list.

    An independent formulation (no dense adjacency matrix, no batched matmul) used to
    pin ``logpsi``.
    """
    p = unpack(theta, F, L, shared)
    nbrs = [[] for _ in range(n)]
    for a, b in np.asarray(edges).tolist():
        nbrs[a].append(b)
        nbrs[b].append(a)
    deg = [len(x) for x in nbrs]
    s = [int(v) for v in spins_1d]
    H = []
    for v in range(n):
        row = p["W_e"][0] if s[v] > 0 else p["W_e"][1]
        H.append(_f_loops([row[f] + p["b_e"][f] for f in range(F)], act))
    for l in range(L):
        W, b = p["W"][l], p["b"][l]
        newH = []
        for v in range(n):
            msg = [0.0] * F
            for u in nbrs[v]:
                c = 1.0 / np.sqrt(deg[v] * deg[u])
                for f in range(F):
                    msg[f] += c * H[u][f]
            row = []
            for g in range(F):
                acc = b[g]
                for f in range(F):
                    acc += msg[f] * W[f, g] + H[v][f] * W[F + f, g]
                row.append(acc)
            newH.append(_f_loops(row, act))
        H = newH
    out = np.array(p["b_r"], dtype=np.float64)
    for v in range(n):
        for f in range(F):
            out += H[v][f] * p["w_r"][f]
        out += p["w_r"][F] if s[v] > 0 else p["w_r"][F + 1]
    return out
