"""Magnitudes of the terms that the checked quantities are summed from (test helper; FP64
oracle).  A floating-point sum is accurate relative to the sum of the absolute values of
its terms, not relative to its result when the terms cancel (the imaginary part of a local
energy, a gradient entry whose samples' contributions nearly cancel), so the FP32 and FP64
parity tests hold each value to tol * max(scale, 1) with:

  log Psi        sum_v sum_f |H^L_vf w_r[f]| + sum_v |onehot_v . w_r[F:]| + |b_r|, per part
  E_loc          sum_e |diagonal element of bond e| + sum_{antiparallel e} |c_e/2| |exp(Delta_e)|
                 (c_e the exchange coupling), for both parts
  Delta_e        the log Psi scales of the state and of the exchanged state (real part)
  grad_k         sum_x |cot_x . d log Psi_x / d theta_k| (per-sample derivatives)
"""
from __future__ import annotations

import numpy as np

from oracle import gcn, heisenberg as hz, isgo


def logpsi_scale(th, F, L, Ah, spins, shared=True, act="tanh"):
    p = gcn.unpack(th, F, L, shared)
    spins = np.atleast_2d(spins)
    HL = gcn.layers(th, F, L, Ah, spins, shared, act)[-1]
    x = gcn.onehot(spins)
    sc = np.abs(HL[..., None] * p["w_r"][None, None, :F, :]).sum(axis=(1, 2))
    sc += np.abs(x[..., None] * p["w_r"][None, None, F:, :]).sum(axis=(1, 2))
    return sc + np.abs(p["b_r"])[None, :]


def delta_scale(th, F, L, Ah, edges, spins, shared=True, act="tanh"):
    """[B][E]: Re log Psi scales of s and s^e (antiparallel bonds; 0 elsewhere)."""
    spins = np.atleast_2d(spins)
    B, N = spins.shape
    out = np.zeros((B, len(edges)))
    base = logpsi_scale(th, F, L, Ah, spins, shared, act)[:, 0]
    for b in range(B):
        s = spins[b]
        anti = np.nonzero(s[edges[:, 0]] != s[edges[:, 1]])[0]
        if len(anti) == 0:
            continue
        sx = np.repeat(s[None, :], len(anti), axis=0)
        r = np.arange(len(anti))
        i, j = edges[anti, 0], edges[anti, 1]
        sx[r, i], sx[r, j] = s[j], s[i]
        out[b, anti] = base[b] + logpsi_scale(th, F, L, Ah, sx, shared, act)[:, 0]
    return out


def eloc_scale(th, F, L, Ah, edges, J, spins, shared=True, act="tanh", xxz=None):
    spins = np.atleast_2d(spins)
    d = hz.bond_log_ratios(lambda x: gcn.logpsi_complex(th, F, L, Ah, x, shared, act), edges, spins)
    si, sj = spins[:, edges[:, 0]].astype(float), spins[:, edges[:, 1]].astype(float)
    if xxz is None:
        Jz, Jxy, hzv, c = np.asarray(J), np.asarray(J), 0.0, 0.0
    else:
        Jz, Jxy, hzv, c = (np.asarray(v) for v in xxz)
    diag = np.abs(Jz / 4 * si * sj + hzv / 2 * (si + sj) + c)
    off = np.where(np.isnan(d.real), 0.0, 0.5 * np.abs(Jxy) * np.abs(np.exp(np.where(np.isnan(d), 0.0, d))))
    return diag.sum(axis=1) + off.sum(axis=1)


def grad_scale(th, F, L, Ah, spins, cot, shared=True, act="tanh"):
    spins = np.atleast_2d(spins)
    cot = np.atleast_2d(cot)
    return sum(np.abs(isgo.backward(th, F, L, Ah, spins[x:x + 1], cot[x:x + 1], shared, act))
               for x in range(spins.shape[0]))
