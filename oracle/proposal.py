"""Learned exchange proposal for Metropolis-Hastings.  TEST INFRASTRUCTURE ONLY.

Not part of arXiv:2011.12453, whose sampler is plain MCMC with P ~ |Psi|^2 (scaling
section).  Every choice below is a reading adopted here:

Policy.  Site i is drawn uniformly from the N sites.  Its candidates are the neighbours
j with s_j != s_i, in adjacency (CSR) order; j is drawn with probability
pi_i(j|s) = softmax over the candidates of logit(phi(i, j, s)).  No candidate: the step
is rejected.  With probability eps the step instead uses the plain move (uniform bond).

Exact proposal density of the exchange s -> s' of the pair {i, j} (reachable from
either endpoint or as a plain move):
    q(s -> s') = (1 - eps)/N [pi_i(j|s) + pi_j(i|s)] + eps/|E|
and the move is accepted with min(1, exp(2 Re Delta) q(s' -> s)/q(s -> s')), which keeps
|Psi|^2 stationary (detailed balance).

Features phi(i, j, s) (9 values), with n1(v) = sum of the neighbours' spins of v:
    s_i, s_j, J_ij, 1/d_i, 1/d_j,
    a_i = (n1(i) - s_j)/max(d_i - 1, 1),  a_j = (n1(j) - s_i)/max(d_j - 1, 1),
    b_i = mean over u in N(i) minus j of n1(u)/d_u (0 if empty),  b_j likewise.
Network: 9 -> 64 -> 64 -> 1 with tanh hidden units; flat parameters
    [W1 (9 x 64), b1 (64), W2 (64 x 64), b2 (64), w3 (64), b3 (1)].
Training target for a pair on bond e: min(0, 2 Re Delta_e), the log acceptance of the
plain exchange; loss = mean squared error over both orientations of every antiparallel
bond of the training configurations; Adam (Kingma & Ba 2015) updates.

Random words of step t (Philox4x64-10, as the plain sampler): r0 plain bond,
r1 acceptance uniform, r2 site i = hi64(r2 N), r3: plain-move coin (r3 >> 40) 2^-24 < eps
and categorical uniform (r3 mod 2^32) 2^-32.
"""
from __future__ import annotations

import numpy as np

from . import sampler

D_IN, HID = 9, 64
N_PARAMS = D_IN * HID + HID + HID * HID + HID + HID + 1


class Topology:
    """Neighbour lists (CSR order: edge-list order of insertion) and couplings."""

    def __init__(self, n: int, edges: np.ndarray, J: np.ndarray):
        self.n = n
        self.edges = np.asarray(edges)
        self.nbr = [[] for _ in range(n)]
        self.Jnb = [[] for _ in range(n)]
        for (a, b), j in zip(self.edges.tolist(), np.asarray(J).tolist()):
            self.nbr[a].append(b)
            self.Jnb[a].append(j)
            self.nbr[b].append(a)
            self.Jnb[b].append(j)
        self.deg = np.array([len(x) for x in self.nbr])
        self.bond = {}
        for e, (a, b) in enumerate(self.edges.tolist()):
            self.bond[(a, b)] = e
            self.bond[(b, a)] = e


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    o = 0

    def take(shape):
        nonlocal o
        size = int(np.prod(shape))
        out = p[o:o + size].reshape(shape)
        o += size
        return out

    W1 = take((D_IN, HID))
    b1 = take((HID,))
    W2 = take((HID, HID))
    b2 = take((HID,))
    w3 = take((HID,))
    b3 = take((1,))
    assert o == p.size == N_PARAMS
    return W1, b1, W2, b2, w3, b3


def features(top: Topology, s, i: int, j: int) -> np.ndarray:
    s = np.asarray(s, dtype=np.float64)
    n1 = np.array([s[top.nbr[v]].sum() for v in range(top.n)])
    Jij = top.Jnb[i][top.nbr[i].index(j)]
    di, dj = top.deg[i], top.deg[j]
    ai = (n1[i] - s[j]) / max(di - 1, 1)
    aj = (n1[j] - s[i]) / max(dj - 1, 1)
    oi = [u for u in top.nbr[i] if u != j]
    oj = [u for u in top.nbr[j] if u != i]
    bi = np.mean([n1[u] / top.deg[u] for u in oi]) if oi else 0.0
    bj = np.mean([n1[u] / top.deg[u] for u in oj]) if oj else 0.0
    return np.array([s[i], s[j], Jij, 1.0 / di, 1.0 / dj, ai, aj, bi, bj])


def mlp(params, phi):
    """Logits (and the hidden activations) for rows phi (R, 9)."""
    W1, b1, W2, b2, w3, b3 = unpack(params)
    phi = np.atleast_2d(phi)
    h1 = np.tanh(phi @ W1 + b1)
    h2 = np.tanh(h1 @ W2 + b2)
    return h2 @ w3 + b3[0], (phi, h1, h2)


def candidates(top: Topology, s, i: int):
    return [u for u in top.nbr[i] if s[u] != s[i]]


def policy(top: Topology, params, s, i: int):
    """(candidates of i, their probabilities pi_i(.|s)) in neighbour order."""
    c = candidates(top, s, i)
    if not c:
        return c, np.zeros(0)
    z, _ = mlp(params, np.stack([features(top, s, i, j) for j in c]))
    z = z - z.max()
    p = np.exp(z)
    return c, p / p.sum()


def pair_prob(top, params, s, i, j) -> float:
    """pi_i(j|s) + pi_j(i|s) for an antiparallel pair."""
    ci, pi = policy(top, params, s, i)
    cj, pj = policy(top, params, s, j)
    return float(pi[ci.index(j)] + pj[cj.index(i)])


def q_mix(top, params, s, i, j, eps: float) -> float:
    """Exact probability of proposing the exchange of the antiparallel pair {i, j} in s."""
    return (1.0 - eps) / top.n * pair_prob(top, params, s, i, j) + eps / len(top.edges)


def transition_matrix(logpsi_values, codes, top: Topology, params, eps: float) -> np.ndarray:
    lp = np.asarray(logpsi_values)
    index = {int(c): k for k, c in enumerate(np.asarray(codes).tolist())}
    n = top.n
    M = len(codes)
    T = np.zeros((M, M))
    for a, c in enumerate(np.asarray(codes).tolist()):
        s = np.array([1 if (c >> v) & 1 else -1 for v in range(n)])
        out = 0.0
        for (i, j) in top.edges.tolist():
            if s[i] == s[j]:
                continue
            b = index[c ^ ((1 << i) | (1 << j))]
            s2 = s.copy()
            s2[[i, j]] = s2[[j, i]]
            qf = q_mix(top, params, s, i, j, eps)
            qr = q_mix(top, params, s2, i, j, eps)
            acc = min(1.0, float(np.exp(2.0 * (lp[b].real - lp[a].real))) * qr / qf)
            T[a, b] += qf * acc
            out += qf * acc
        T[a, a] += 1.0 - out
    return T


def choose(cands, probs, uc: float):
    """First candidate whose cumulative probability exceeds uc (the last one otherwise)."""
    acc = 0.0
    for j, p in zip(cands, probs):
        acc += p
        if uc < acc:
            return j
    return cands[-1]


def run_chains(logpsi_fn, top: Topology, params, spins0, seed: int, step0: int, n_sweeps: int, eps: float):
    """Learned-proposal Metropolis-Hastings chains (float64).

    Returns (final spins, accepted [C], trace [C][steps][5]) with trace rows
    (move kind: 0 none / 1 plain / 2 learned, i, j, accepted, log acceptance ratio or NaN).
    """
    s_all = np.array(spins0, dtype=np.int8, copy=True)
    C, n = s_all.shape
    E = len(top.edges)
    steps = n_sweeps * n
    acc = np.zeros(C, dtype=np.int64)
    trace = np.full((C, steps, 5), np.nan)
    for c in range(C):
        s = s_all[c]
        lp = logpsi_fn(s[None])[0]
        for k in range(steps):
            r0, r1, r2, r3 = sampler.step_words(seed, c, step0 + k)
            coin = (r3 >> 40) * 2.0 ** -24
            trace[c, k, :4] = (0, -1, -1, 0)
            if coin < eps:
                e = sampler.bond_index(r0, E)
                i, j = (int(x) for x in top.edges[e])
                kind = 1
                if s[i] == s[j]:
                    trace[c, k, :4] = (1, i, j, 0)
                    continue
            else:
                i = (int(r2) * n) >> 64
                ci, pi = policy(top, params, s, i)
                if not ci:
                    trace[c, k, :4] = (2, i, -1, 0)
                    continue
                j = choose(ci, pi, (r3 & 0xFFFFFFFF) * 2.0 ** -32)
                kind = 2
            s2 = s.copy()
            s2[[i, j]] = s2[[j, i]]
            lp2 = logpsi_fn(s2[None])[0]
            qf = q_mix(top, params, s, i, j, eps)
            qr = q_mix(top, params, s2, i, j, eps)
            log_ratio = 2.0 * (lp2 - lp).real + np.log(qr) - np.log(qf)
            u = sampler.uniform(r1, "fp64")
            ok = bool(u < np.exp(log_ratio))
            trace[c, k] = (kind, i, j, int(ok), log_ratio)
            if ok:
                s[:] = s2
                lp = lp2
                acc[c] += 1
    return s_all, acc, trace


# ---------------------------------------------------------------------------------
# training
# ---------------------------------------------------------------------------------

def training_rows(top: Topology, spins, dlogpsi_re):
    """Features and targets of every antiparallel bond of every configuration, both
    orientations: (phi (R, 9), target (R,))."""
    rows, tgt = [], []
    for b, s in enumerate(np.asarray(spins)):
        for e, (i, j) in enumerate(top.edges.tolist()):
            if s[i] == s[j]:
                continue
            a = min(0.0, 2.0 * float(dlogpsi_re[b, e]))
            rows.append(features(top, s, i, j))
            tgt.append(a)
            rows.append(features(top, s, j, i))
            tgt.append(a)
    return np.array(rows).reshape(-1, D_IN), np.array(tgt)


def loss_and_grad(params, phi, target):
    """Mean squared error and its gradient (hand-derived reverse mode)."""
    W1, b1, W2, b2, w3, b3 = unpack(params)
    z, (x, h1, h2) = mlp(params, phi)
    R = x.shape[0]
    r = z - target
    loss = float((r * r).mean())
    dz = 2.0 * r / R
    gw3 = h2.T @ dz
    gb3 = np.array([dz.sum()])
    dh2 = np.outer(dz, w3)
    dz2 = dh2 * (1.0 - h2 * h2)
    gW2 = h1.T @ dz2
    gb2 = dz2.sum(axis=0)
    dh1 = dz2 @ W2.T
    dz1 = dh1 * (1.0 - h1 * h1)
    gW1 = x.T @ dz1
    gb1 = dz1.sum(axis=0)
    return loss, np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, gb3])


def adam_step(params, grad, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns (params, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
