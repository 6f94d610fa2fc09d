"""Error of the reduced-precision paths against the FP64 oracle for each of the quantities an
ISGO step produces -- the mean energy E, its variance sigma^2(E) and the gradient -- on
the Kagome 6x6x3 workload (L = 4, F = 32), on the same 48 chain samples, at the benchmark
weight scale 0.1 (a nearly flat wavefunction: E_loc varies by 1.6e-4 of E across samples)
and at 0.3.  BF16 (tensor-core GEMMs, FP32 activations and ratios, FP64 reductions) is
compared with the oracle on W rounded to BF16, so the error is that of the activation
rounding; FP32 with the oracle on the same FP32 parameters.  The gradient error is also
split into the part that comes from the local energies (oracle backward, device E_loc)
and the part from d log Psi / d theta (device backward, oracle E_loc).

Bounds, from the measured errors with margin: BF16 at scale 0.1 E 1e-4, sigma^2 5e-2,
gradient 0.6 of its largest component -- the covariance gradient of a nearly flat state is
a small difference of per-sample derivatives, and the BF16 operand rounding of the
backward's activations (relative 2^-9 of the full derivatives, not of their small
variation) is of the same size as that difference; at scale 0.3 (saturating units, bond
ratios exp(Delta) up to ~20, which amplify the BF16 rounding of O(1) differences) E 5e-3,
sigma^2 2e-2, gradient 5e-2.  FP32: E 1e-6, sigma^2 1e-4, gradient 1e-3."""
import numpy as np
import pytest

from oracle import gcn, isgo
from paper_2011_12453_gb300 import build as B, gna, workloads as W

pytestmark = pytest.mark.gpu

BOUNDS = {(gna.PREC_BF16, 0.1): (1e-4, 5e-2, 0.6), (gna.PREC_BF16, 0.3): (5e-3, 2e-2, 5e-2),
          (gna.PREC_BF16X2, 0.1): (1e-4, 1e-3, 1e-3), (gna.PREC_BF16X2, 0.3): (1e-4, 1e-3, 1e-3),
          (gna.PREC_FP32, 0.1): (1e-6, 1e-4, 1e-3), (gna.PREC_FP32, 0.3): (1e-6, 1e-4, 1e-3)}


@pytest.fixture(scope="module")
def torch():
    import torch as t

    B.build()
    t.cuda.set_device(0)
    return t


@pytest.mark.parametrize("scale", [0.1, 0.3])
@pytest.mark.parametrize("prec", [gna.PREC_BF16, gna.PREC_BF16X2, gna.PREC_FP32])
def test_energy_variance_gradient_errors(torch, prec, scale):
    g = W.kagome(6)
    F, L, Bn = 32, 4, 48
    graph = gna.Graph.from_workload(g, L)
    model = gna.Model(F, L, prec)
    theta = torch.tensor(W.random_theta(F, L, seed=0, scale=scale), dtype=torch.float32, device="cuda")
    th = theta.double().cpu().numpy()
    if prec in (gna.PREC_BF16, gna.PREC_BF16X2):
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
    err_g = np.abs(grad - g_o).max() / gmax
    # attribution: device local energies with the oracle's derivatives, and the reverse
    E_d = gna.local_energy(graph, model, theta, s).cpu().numpy()
    E_d = E_d[:, 0] + 1j * E_d[:, 1]
    pu = np.full(Bn, 1.0 / Bn)
    from_E = isgo.backward(th, F, L, Ah, x, isgo.cotangents(pu, E_d, E_d.mean()))
    cot_o = torch.tensor(isgo.cotangents(pu, E_o, E_o.mean()), device="cuda")
    from_O = gna.backward(graph, model, theta, s, cot_o).cpu().numpy()
    err_gE = np.abs(from_E - g_o).max() / gmax
    err_gO = np.abs(from_O - g_o).max() / gmax
    name = {gna.PREC_BF16: "BF16", gna.PREC_BF16X2: "BF16X2", gna.PREC_FP32: "FP32"}[prec]
    print(f"\n{name} scale {scale}: E {Ebar.real:.5f} (sigma_E {np.sqrt(var):.2e}) rel err {err_E:.2e}; sigma^2 rel err "
          f"{err_var:.2e}; gradient err / max {err_g:.2e} (from E_loc {err_gE:.2e}, from d log Psi {err_gO:.2e})")
    bE, bV, bG = BOUNDS[(prec, scale)]
    assert err_E <= bE and err_var <= bV and err_g <= bG, (err_E, err_var, err_g)
