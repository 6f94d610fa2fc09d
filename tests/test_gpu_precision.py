"""Error of the reduced-precision paths against the FP64 oracle for each of the quantities an
ISGO step produces -- the mean energy E, its variance sigma^2(E) and the gradient -- on
the Kagome 6x6x3 workload (L = 4, F = 32), on the same 48 chain samples, at the benchmark
weight scale 0.1 (a nearly flat wavefunction: E_loc varies by 1.6e-4 of E across samples,
and the gradient is a small covariance of nearly equal per-sample derivatives) and at 0.3.
The tensor-core precisions are compared with the oracle on W rounded to BF16 (W is a BF16
model parameter), so the error is that of the activations' rounding; FP32 with the oracle
on the same FP32 parameters.  The gradient error is also split into the part that comes
from the local energies (oracle backward, device E_loc) and the part from d log Psi /
d theta (device backward, oracle E_loc).

Bounds for the tensor-core precisions are derived from the arithmetic, per sample
(tests/bounds.py for the local energies; the backward as in test_gpu_bf16.py).  Each
sample's local-energy error eps_x = a_x + r_x has a part a_x shared with the other samples
through the cached forward (|a_x| <= A_x) and an independent part r_x of standard deviation
s_x (the operand roundings of its own difference propagations).  With p the weights
(uniform here: log Psi^0 is the forward's own value), O_x the oracle's per-sample
derivatives and Obar = sum p O, and since sum_x p_x (eps_x - epsbar) = 0,
  err Ebar   = sum p eps                           <= sum p A + 6 sqrt(sum p^2 s^2)
  err sigma^2 = 2 sum p Re((E - Ebar)^* (eps - epsbar)) + sum p |eps - epsbar|^2
             <= 2 sum p |E - Ebar| 2A + 6 sqrt(sum (2 p |E - Ebar|)^2 s^2)
                + sum p (2A)^2 + 2 sum p 2A 3s + sum p s^2 + 6 sqrt(2 sum p^2 s^4)
  err g_k    = sum 2 p (eps - epsbar) (O_x,k - Obar_k)
             <= sum 2 p 2A |O - Obar| + 6 sqrt(sum (2 p |O - Obar|)^2 s^2)
plus, for the gradient, 2^-14 sum_x |cot_x . d log Psi_x / d theta_k| (split-operand
backward); |O| sums the real and imaginary parts.  BF16X2, the precision the benchmark
runs, must also meet the accuracy targets outright: E within 1e-4, sigma^2 within 1e-3 and
the gradient within 1e-3 of its largest component.
FP32 is held to E 1e-6, sigma^2 1e-4 and gradient 1e-3 of its largest component."""
import numpy as np
import pytest

from oracle import gcn, isgo
from paper_2011_12453_gb300 import build as B, gna, workloads as W

import bounds as BD

pytestmark = pytest.mark.gpu

TARGETS = {gna.PREC_BF16X2: (1e-4, 1e-3, 1e-3), gna.PREC_FP32: (1e-6, 1e-4, 1e-3)}


@pytest.fixture(scope="module")
def torch():
    import torch as t

    B.build()
    t.cuda.set_device(0)
    return t


def _derived_bounds(th, F, L, Ah, g, x, E_o, cot_o, mode):
    """(E, sigma^2, gradient) error bounds of the tensor-core path, relative as tested."""
    Bn = x.shape[0]
    p = np.full(Bn, 1.0 / Bn)
    _, _, _, A, sg = BD.bond_bounds(th, F, L, Ah, g.edges, g.J, x, mode, parts=True)
    Ebar = (p * E_o).sum()
    dE = np.abs(E_o - Ebar)
    var = float((p * dE ** 2).sum())
    bE = ((p * A).sum() + 6.0 * np.sqrt((p * p * sg * sg).sum())) / abs(Ebar.real)
    # second order: sum p |a + r - abar - rbar|^2 <= sum p (2A)^2 + 2 sum p 2A 3s + sum p r^2, the
    # last a sum of independent squares: its mean sum p s^2 plus 6 of its standard deviations
    second = ((p * (2.0 * A) ** 2).sum() + 2.0 * (p * 2.0 * A * 3.0 * sg).sum() + (p * sg ** 2).sum() +
              6.0 * np.sqrt(2.0 * (p * p * sg ** 4).sum()))
    bV = (2.0 * (p * dE * 2.0 * A).sum() + 6.0 * np.sqrt(((2.0 * p * dE) ** 2 * sg ** 2).sum()) + second) / var
    one, two = np.array([[1.0, 0.0]]), np.array([[0.0, 1.0]])
    O = np.stack([isgo.backward(th, F, L, Ah, x[k:k + 1], one) for k in range(Bn)])
    Oi = np.stack([isgo.backward(th, F, L, Ah, x[k:k + 1], two) for k in range(Bn)])
    dO = np.abs(O - (p[:, None] * O).sum(0)) + np.abs(Oi - (p[:, None] * Oi).sum(0))
    gE = (2.0 * p[:, None] * 2.0 * A[:, None] * dO).sum(0) + 6.0 * np.sqrt(((2.0 * p[:, None] * dO) ** 2 *
                                                                            sg[:, None] ** 2).sum(0))
    gO = sum(np.abs(isgo.backward(th, F, L, Ah, x[k:k + 1], cot_o[k:k + 1])) for k in range(Bn))
    return bE, bV, gE + 2.0 ** -14 * gO


@pytest.mark.parametrize("scale", [0.1, 0.3])
@pytest.mark.parametrize("prec", [gna.PREC_BF16, gna.PREC_BF16X2, gna.PREC_FP32])
def test_energy_variance_gradient_errors(torch, prec, scale):
    g = W.kagome(6)
    F, L, Bn = 32, 4, 48
    graph = gna.Graph.from_workload(g, L)
    model = gna.Model(F, L, prec)
    theta = torch.tensor(W.random_theta(F, L, seed=0, scale=scale), dtype=torch.float32, device="cuda")
    th = theta.double().cpu().numpy()
    tensor = prec in (gna.PREC_BF16, gna.PREC_BF16X2)
    if tensor:
        o = 3 * F
        th[o:o + 2 * F * F] = torch.tensor(th[o:o + 2 * F * F], dtype=torch.float32).to(torch.bfloat16).double().numpy()
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    ch = torch.tensor(W.random_spins(g.n_sites, Bn, seed=1), device="cuda")
    samples, _, _, _ = gna.metropolis_sweep(graph, model, theta, ch, 4, 4, 3, 0)
    s = samples[-1].contiguous()
    lp0 = gna.forward(graph, model, theta, s)
    grad, stats = gna.isgo_grad(graph, model, theta, s, lp0)
    grad, stats = grad.cpu().numpy(), stats.cpu().numpy()
    x = s.cpu().numpy()
    lp_o = gcn.logpsi_complex(th, F, L, Ah, x)
    g_o, Ebar, var, ess, E_o, p = isgo.isgo_gradient(th, F, L, Ah, g.edges, g.J, x, lp_o)
    err_E = abs(stats[0] - Ebar.real) / abs(Ebar.real)
    err_var = abs(stats[2] - var) / var
    gmax = np.abs(g_o).max()
    err = np.abs(grad - g_o)
    err_g = err.max() / gmax
    # attribution: device local energies with the oracle's derivatives, and the reverse
    E_d = gna.local_energy(graph, model, theta, s).cpu().numpy()
    E_d = E_d[:, 0] + 1j * E_d[:, 1]
    pu = np.full(Bn, 1.0 / Bn)
    from_E = isgo.backward(th, F, L, Ah, x, isgo.cotangents(pu, E_d, E_d.mean()))
    cot_np = isgo.cotangents(pu, E_o, E_o.mean())
    from_O = gna.backward(graph, model, theta, s, torch.tensor(cot_np, device="cuda")).cpu().numpy()
    err_gE = np.abs(from_E - g_o).max() / gmax
    err_gO = np.abs(from_O - g_o).max() / gmax
    name = {gna.PREC_BF16: "BF16", gna.PREC_BF16X2: "BF16X2", gna.PREC_FP32: "FP32"}[prec]
    print(f"\n{name} scale {scale}: E {Ebar.real:.5f} (sigma_E {np.sqrt(var):.2e}) rel err {err_E:.2e}; sigma^2 rel err "
          f"{err_var:.2e}; gradient err / max {err_g:.2e} (from E_loc {err_gE:.2e}, from d log Psi {err_gO:.2e})")
    if tensor:
        bE, bV, bG = _derived_bounds(th, F, L, Ah, g, x, E_o, cot_np, "bf16" if prec == gna.PREC_BF16 else "bf16x2")
        print(f"  derived bounds: E {bE:.2e}, sigma^2 {bV:.2e}, gradient {bG.max() / gmax:.2e} of max")
        assert err_E <= bE and err_var <= bV, (err_E, bE, err_var, bV)
        assert np.all(err <= bG), float(np.max(err - bG))
    if prec in TARGETS:
        tE, tV, tG = TARGETS[prec]
        assert err_E <= tE and err_var <= tV and err_g <= tG, (err_E, err_var, err_g)
