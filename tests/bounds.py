"""Error bounds of the tensor-core incremental local energy, derived from its arithmetic
(test helper; uses the FP64 oracle for the exact values the bounds are built from).

The incremental ratio of a bond e propagates the change dH^l of the node features caused
by exchanging s_i and s_j (Eq. gcn, layer by layer).  Per layer the tensor-core path
rounds (a) the stored rows of dH^{l-1} that the gather reads and (b) the gathered rows
dX^l = [A_hat dH^{l-1} ; dH^{l-1}] that the MMA multiplies by W (W itself is the BF16
model parameter and exact); it evaluates tanh(dY) with a relative error u_t; and it takes
the derivative of tanh at the pre-activation Y^l of the cached forward, which carries the
forward's own rounding.

Each rounding of a value x to a grid of relative spacing 2u (round to nearest) makes an
error uniform in [-u|x|, u|x|], of variance u^2 x^2 / 3; errors of different values are
independent.  Their variances propagate through the difference propagation to first order
(squares of the linear maps):

  v^0      = u_s^2/3 |dH^0|^2
  vX^l     = [A_hat^2 v^{l-1} ; v^{l-1}] + u_a^2/3 [A_hat dH^{l-1} ; dH^{l-1}]^2
  v^l      = (1 - tanh^2(Y^l + dY^l))^2 (vX^l W^2) + (u_t^2 + u_s^2 [l < L]) / 3 |dH^l|^2
  sigma_e  = sqrt(sum_v v^L_v . w_r[:, 0]^2 + sum_v v^L_v . w_r[:, 1]^2)

The cached forward's pre-activations Y^l carry two kinds of error.  The two embedding rows
are rounded once and shared by every site of a spin, so that error is not independent
across sites: it is computed exactly (the forward run from the rounded rows, minus the
exact one) and propagated as a signed first-order change.  The forward's other roundings
(its gathered rows X^l, its stored rows H^l, its tanh) are independent and enter as
variances, v_f^l = [A_hat^2 v_fH ; v_fH] W^2 + u_a^2/3 X^2 W^2, v_fH = tanh'(Y)^2 v_f + (u_t^2 +
u_s^2)/3 H^2.  A pre-activation error eps changes dH^l by (tanh'(Y^l + dY^l) - tanh'(Y^l)) eps,
which joins the propagation above (signed for the shared part, as variance for the rest).
The bound on |err Delta_e| is |signed part| + 6 sigma_e; per sample,
|err E_loc| <= sum_e |J_e|/2 |exp(Delta_e)| (exp(b_e) - 1).

Unit roundoffs: BF16 (8 significant bits) u_s = u_a = 2^-8 and the approximate hardware
tanh u_t = 2^-10.5; BF16X2 operands as hi + lo pairs u_a = 2^-16, FP32 rows u_s = 2^-24,
tanh from its Taylor series u_t = 2^-22.
"""
from __future__ import annotations

import numpy as np

from oracle import gcn

UNITS = {"bf16": (2.0 ** -8, 2.0 ** -8, 2.0 ** -10.5), "bf16x2": (2.0 ** -24, 2.0 ** -16, 2.0 ** -22)}


def bf16_round(x):
    """Round to the nearest BF16 value (ties to even), through float32."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _layers_and_pre(th, F, L, Ah, spins):
    """[H^0..H^L] and [Y^1..Y^L] (B, N, F) of the oracle's GCN (shared weights)."""
    p = gcn.unpack(th, F, L)
    H = gcn.layers(th, F, L, Ah, spins)
    Y = []
    for l in range(L):
        X = np.concatenate([np.einsum("vu,buf->bvf", Ah, H[l]), H[l]], axis=-1)
        Y.append(X @ p["W"][l] + p["b"][l])
    return H, Y


def bond_bounds(th, F, L, Ah, edges, J, spins, mode, parts=False):
    """For each sample and bond: the exact Delta = log Psi(s^e) - log Psi(s) (complex, NaN on
    parallel bonds), the bound on |err Delta| and the per-sample bound on |err E_loc|; with
    parts=True also, per sample, the local-energy error's shared part (an absolute bound)
    and the standard deviation of its independent part, to first order."""
    u_s, u_a, u_t = UNITS[mode]
    p = gcn.unpack(th, F, L)
    wr = p["w_r"][:F]
    spins = np.atleast_2d(spins)
    B, N = spins.shape
    E = len(edges)
    H, Y = _layers_and_pre(th, F, L, Ah, spins)
    # errors of the cached forward's pre-activations: the shared rounding of the embedding
    # rows (signed, exact first order) and the independent ones (variance)
    W = p["W"][0]
    Hr = bf16_round(H[0]) if u_s > 2.0 ** -12 else H[0]
    fdet = [None] * (L + 1)
    vf = [None] * (L + 1)
    Hd, vH = Hr, (u_t ** 2 + u_s ** 2) / 3.0 * H[0] ** 2 * 0.0
    for l in range(1, L + 1):
        Xd = np.concatenate([np.einsum("vu,buf->bvf", Ah, Hd), Hd], axis=-1)
        Yd = Xd @ W + p["b"][0]
        fdet[l] = Yd - Y[l - 1]
        X = np.concatenate([np.einsum("vu,buf->bvf", Ah, H[l - 1]), H[l - 1]], axis=-1)
        vX = np.concatenate([np.einsum("vu,buf->bvf", Ah ** 2, vH), vH], axis=-1) + u_a ** 2 / 3.0 * X ** 2
        vf[l] = vX @ W ** 2
        vH = (1.0 - H[l] ** 2) ** 2 * vf[l] + (u_t ** 2 + u_s ** 2) / 3.0 * H[l] ** 2
        Hd = np.tanh(Yd)
    delta = np.full((B, E), np.nan + 0j)
    bound = np.zeros((B, E))
    e_bound = np.zeros(B)
    e_shared = np.zeros(B)
    e_sigma = np.zeros(B)
    for b in range(B):
        s = spins[b]
        anti = np.nonzero(s[edges[:, 0]] != s[edges[:, 1]])[0]
        if len(anti) == 0:
            continue
        sx = np.repeat(s[None, :], len(anti), axis=0)
        i, j = edges[anti, 0], edges[anti, 1]
        r = np.arange(len(anti))
        sx[r, i], sx[r, j] = s[j], s[i]
        Hx, Yx = _layers_and_pre(th, F, L, Ah, sx)
        dH = [Hx[l] - H[l][b][None] for l in range(L + 1)]
        var = u_s ** 2 / 3.0 * dH[0] ** 2
        sgn = np.zeros_like(dH[0])  # signed first-order error from the shared embedding rounding
        for l in range(1, L + 1):
            dX = np.concatenate([np.einsum("vu,buf->bvf", Ah, dH[l - 1]), dH[l - 1]], axis=-1)
            vX = np.concatenate([np.einsum("vu,buf->bvf", Ah ** 2, var), var], axis=-1) + u_a ** 2 / 3.0 * dX ** 2
            sX = np.concatenate([np.einsum("vu,buf->bvf", Ah, sgn), sgn], axis=-1)
            g_new = 1.0 - Hx[l] ** 2
            dg = g_new - (1.0 - H[l][b][None] ** 2)
            var = (g_new ** 2 * (vX @ W ** 2) + dg ** 2 * vf[l][b][None] +
                   (u_t ** 2 + (u_s ** 2 if l < L else 0.0)) / 3.0 * dH[l] ** 2)
            sgn = g_new * (sX @ W) + dg * fdet[l][b][None]
        d = dH[L].sum(axis=1) @ wr  # the one-hot readout rows cancel (same N_up)
        sig = np.sqrt((var.sum(axis=1) @ wr ** 2).sum(axis=1))
        bd = np.abs(sgn.sum(axis=1) @ wr).sum(axis=1) + 6.0 * sig
        delta[b, anti] = d[:, 0] + 1j * d[:, 1]
        bound[b, anti] = bd
        amp = np.abs(np.exp(d[:, 0] + 1j * d[:, 1]))
        e_bound[b] = float((0.5 * np.abs(np.asarray(J)[anti]) * amp * np.expm1(bd)).sum())
        # the sample's local-energy error as a shared part (bounded in absolute value, summed
        # over bonds) and an independent part (standard deviation, added in quadrature)
        shr = np.abs(sgn.sum(axis=1) @ wr).sum(axis=1)
        w = 0.5 * np.abs(np.asarray(J)[anti]) * amp
        e_shared[b] = float((w * shr).sum())
        e_sigma[b] = float(np.sqrt(((w * sig) ** 2).sum()))
    if parts:
        return delta, bound, e_bound, e_shared, e_sigma
    return delta, bound, e_bound


def forward_bound(th, F, L, Ah, spins, mode):
    """Bound on |err log Psi| (Re and Im together) of the tensor-core forward: the shared
    rounding of the embedding rows propagated exactly (signed), the independent roundings of
    the gathered rows X^l, the stored rows H^l (l < L) and their tanh by variance (6 sigma);
    the forward-only call keeps H^L in FP32 from an accurate tanh."""
    u_s, u_a, u_t = UNITS[mode]
    p = gcn.unpack(th, F, L)
    W = p["W"][0]
    wr = p["w_r"][:F]
    spins = np.atleast_2d(spins)
    H, Y = _layers_and_pre(th, F, L, Ah, spins)
    Hd = bf16_round(H[0]) if u_s > 2.0 ** -12 else H[0]
    vH = np.zeros_like(H[0])
    for l in range(1, L + 1):
        Yd = np.concatenate([np.einsum("vu,buf->bvf", Ah, Hd), Hd], axis=-1) @ W + p["b"][0]
        X = np.concatenate([np.einsum("vu,buf->bvf", Ah, H[l - 1]), H[l - 1]], axis=-1)
        vX = np.concatenate([np.einsum("vu,buf->bvf", Ah ** 2, vH), vH], axis=-1) + u_a ** 2 / 3.0 * X ** 2
        vY = vX @ W ** 2
        last = l == L
        vH = (1.0 - H[l] ** 2) ** 2 * vY + ((2.0 ** -22) ** 2 if last else u_t ** 2 + u_s ** 2) / 3.0 * H[l] ** 2
        Hd = np.tanh(Yd)
    det = np.abs((Hd - H[L]).sum(axis=1) @ wr).sum(axis=1)
    sig = np.sqrt((vH.sum(axis=1) @ wr ** 2).sum(axis=1))
    return det + 6.0 * sig
