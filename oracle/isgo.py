"""ISGO importance-reweighted energy gradient.  TEST INFRASTRUCTURE ONLY.

Eq. (isgo) of arXiv:2011.12453 reweights samples drawn from P^0 ~ |Psi^0|^2 to the
current wavefunction with I_x / I^0 = C |Psi_x|^2 / |Psi^0_x|^2, normalised so that
the weights sum to one, and forms the covariance of E_x with d ln Psi_x.

The printed normalisation of Eq. (vmc)/(isgo) is not self-consistent (with I^0 = 2/N
the two terms differ by a factor 2).  Reading adopted: the textbook covariance
gradient that the equation approximates, for complex log Psi and real parameters w:

  w_x  = count_x * |Psi_x|^2 / |Psi^0_x|^2,     p_x = w_x / sum_x w_x
  Ebar = sum_x p_x E_x
  g_k  = 2 Re sum_x p_x (E_x - Ebar)^* d log Psi_x / d w_k
       = sum_x [ 2 p_x Re(E_x - Ebar) d Re log Psi_x/d w_k
                + 2 p_x Im(E_x - Ebar) d Im log Psi_x/d w_k ]

i.e. one vector-Jacobian product of log Psi with the cotangents
(2 p Re(E - Ebar), 2 p Im(E - Ebar)).  E_x is evaluated under the current parameters
and the weights use log Psi^0 stored at sampling time.  With w = w^0 and unit counts
this is plain VMC (Eq. vmc).  Counts group duplicate states (scaling section).
"""
from __future__ import annotations

import numpy as np

from . import gcn


def weights(logpsi, logpsi0, counts=None) -> np.ndarray:
    """Normalised importance weights p_x (float64), via a max-shifted log-sum-exp."""
    lp = np.asarray(logpsi)
    lp0 = np.asarray(logpsi0)
    re = lp.real if np.iscomplexobj(lp) else lp[:, 0]
    re0 = lp0.real if np.iscomplexobj(lp0) else lp0[:, 0]
    logw = 2.0 * (re - re0)
    if counts is not None:
        logw = logw + np.log(np.asarray(counts, dtype=np.float64))
    m = logw.max()
    w = np.exp(logw - m)
    return w / w.sum()


def statistics(p: np.ndarray, E: np.ndarray, counts=None):
    """(Ebar complex, variance sum p |E - Ebar|^2, importance-sampling ESS).

    ESS = (sum_x c_x w_x)^2 / sum_x c_x w_x^2 = 1 / sum_x p_x^2 / c_x with w_x the
    per-copy weight |Psi_x|^2/|Psi^0_x|^2, so that grouping duplicates into counts c_x
    leaves it unchanged; with unit counts it is 1 / sum p^2.
    """
    E = np.asarray(E, dtype=np.complex128)
    c = np.ones_like(p) if counts is None else np.asarray(counts, dtype=np.float64)
    Ebar = complex((p * E).sum())
    var = float((p * np.abs(E - Ebar) ** 2).sum())
    ess = float(1.0 / (p * p / c).sum())
    return Ebar, var, ess


def cotangents(p: np.ndarray, E: np.ndarray, Ebar: complex) -> np.ndarray:
    """(B, 2): (2 p Re(E - Ebar), 2 p Im(E - Ebar))."""
    d = np.asarray(E, dtype=np.complex128) - Ebar
    return np.stack([2.0 * p * d.real, 2.0 * p * d.imag], axis=1)


def _act_vjp(G, H, Y, act):
    """Cotangent of the pre-activation Y of f, given the cotangent G of H = f(Y).

    tanh: G (1 - H^2).  ReLU then layer norm (r = max(Y, 0), H = (r - mean r)/sigma,
    sigma = sqrt(var r + eps)): dr = (G - mean G - H mean(G H)) / sigma over each row,
    then dY = dr where Y > 0 and 0 elsewhere."""
    if act == "tanh":
        return G * (1.0 - H * H)
    r = np.maximum(Y, 0.0)
    c = r - r.mean(axis=-1, keepdims=True)
    sigma = np.sqrt((c * c).mean(axis=-1, keepdims=True) + gcn.LN_EPS)
    dr = (G - G.mean(axis=-1, keepdims=True) - H * (G * H).mean(axis=-1, keepdims=True)) / sigma
    return np.where(Y > 0.0, dr, 0.0)


def backward(theta, F: int, L: int, Ahat: np.ndarray, spins: np.ndarray, cot: np.ndarray,
             shared: bool = True, act: str = "tanh") -> np.ndarray:
    """sum_x [cot_x0 d Re log Psi_x/d theta + cot_x1 d Im log Psi_x/d theta] (flat, float64).

    Reverse-mode derivative of gcn.logpsi, derived by hand from the chain rule:
    readout -> L GCN layers (f' of _act_vjp; the message term transposes
    D^-1/2 A D^-1/2, which is symmetric) -> embedding.
    """
    p = gcn.unpack(theta, F, L, shared)
    s = np.atleast_2d(spins)
    cot = np.atleast_2d(np.asarray(cot, dtype=np.float64))
    Hs = gcn.layers(theta, F, L, Ahat, s, shared, act)
    x = gcn.onehot(s)
    g = {"W_e": np.zeros((2, F)), "b_e": np.zeros(F), "w_r": np.zeros((F + 2, 2)), "b_r": np.zeros(2)}
    gW = [np.zeros((2 * F, F)) for _ in range(L)]
    gb = [np.zeros(F) for _ in range(L)]
    # readout: log Psi_k = sum_v [H^L_v, x_v] . w_r[:, k] + b_r[k]
    z = np.concatenate([Hs[L], x], axis=-1).sum(axis=1)  # (B, F+2)
    g["w_r"] += z.T @ cot
    g["b_r"] += cot.sum(axis=0)
    G = np.broadcast_to((cot @ p["w_r"][:F].T)[:, None, :], Hs[L].shape).copy()  # dL/dH^L
    for l in range(L, 0, -1):
        Hp, Hl = Hs[l - 1], Hs[l]
        X = np.concatenate([np.einsum("vu,buf->bvf", Ahat, Hp), Hp], axis=-1)  # (B, n, 2F)
        dY = _act_vjp(G, Hl, X @ p["W"][l - 1] + p["b"][l - 1], act)
        gW[l - 1] += np.einsum("bvk,bvg->kg", X, dY)
        gb[l - 1] += dY.sum(axis=(0, 1))
        dX = dY @ p["W"][l - 1].T  # (B, n, 2F)
        G = np.einsum("uv,buf->bvf", Ahat, dX[..., :F]) + dX[..., F:]
    dY0 = _act_vjp(G, Hs[0], x @ p["W_e"] + p["b_e"], act)
    g["W_e"] += np.einsum("bvc,bvf->cf", x, dY0)
    g["b_e"] += dY0.sum(axis=(0, 1))
    parts = [g["W_e"].ravel(), g["b_e"]]
    if shared:
        parts += [sum(gW).ravel(), sum(gb)]
    else:
        for l in range(L):
            parts += [gW[l].ravel(), gb[l]]
    parts += [g["w_r"].ravel(), g["b_r"]]
    return np.concatenate(parts)


def isgo_gradient(theta, F, L, Ahat, edges, J, spins, logpsi0, counts=None, shared=True, xxz=None,
                  act="tanh"):
    """Full ISGO step quantities: (gradient, Ebar, variance, ESS, E_loc, p).  Heisenberg
    bonds J, or XXZ bonds xxz = (Jz, Jxy, hz, c) (hard-core bosons)."""
    from . import heisenberg

    def lp_fn(s):
        return gcn.logpsi_complex(theta, F, L, Ahat, s, shared, act)

    s = np.atleast_2d(spins)
    lp = lp_fn(s)
    E = heisenberg.local_energy(lp_fn, edges, J, s, xxz)
    p = weights(lp, logpsi0, counts)
    Ebar, var, ess = statistics(p, E, counts)
    cot = cotangents(p, E, Ebar)
    grad = backward(theta, F, L, Ahat, s, cot, shared, act)
    return grad, Ebar, var, ess, E, p


def sgd(theta, grad, lr: float) -> np.ndarray:
    """w <- w - alpha dE_v/dw (scaling section)."""
    return np.asarray(theta) - lr * np.asarray(grad)
