"""The tensor-core backward (split BF16 operands, the benchmark's default) at the benchmark's
size and launch configuration: Kagome 6x6x3, F = 32, L = 4, 16384 configurations per call,
parameters from the benchmark's seed (weight scale 0.1).  The cotangent is zero except on 64
configurations drawn at random, so the gradient is the vector-Jacobian product of those 64
alone, which the FP64 oracle computes sample by sample (on the BF16 W the model holds).  The
tensor-core backward accumulates each block's samples in FP32 from operands exact to 2^-16:
every component within 2 x 2^-14 sum_x |cot_x . d log Psi_x / d theta| of the oracle (the
bound of the allocation-free backward's test).  The other 16320 configurations, with zero
cotangent, must add nothing."""
import numpy as np
import pytest

from bounds import bf16_round
from oracle import gcn, isgo
from paper_2011_12453_gb300 import build as B, gna, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t

    B.build()
    t.cuda.set_device(0)
    return t


def test_split_backward_at_benchmark_size(torch):
    g = W.kagome(6)
    F, L, C = 32, 4, 16384
    graph = gna.Graph.from_workload(g, L)
    model = gna.Model(F, L, gna.PREC_BF16X2)
    theta = torch.tensor(W.random_theta(F, L, 0), dtype=torch.float32, device="cuda")
    spins = W.random_spins(g.n_sites, C, 1)
    rng = np.random.default_rng(5)
    pick = rng.choice(C, size=64, replace=False)
    cot = np.zeros((C, 2))
    cot[pick] = rng.normal(size=(64, 2))
    gna.device_status(clear=True)  # the status word is sticky: start from a clean one
    got = gna.backward(graph, model, theta, torch.tensor(spins, device="cuda"),
                       torch.tensor(cot, device="cuda")).cpu().numpy()
    assert gna.device_status(clear=True) == 0
    th = theta.double().cpu().numpy()
    th[3 * F:3 * F + 2 * F * F] = bf16_round(th[3 * F:3 * F + 2 * F * F])
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    parts = [isgo.backward(th, F, L, Ah, spins[k:k + 1], cot[k:k + 1]) for k in pick]
    want = np.sum(parts, axis=0)
    kappa = np.sum(np.abs(parts), axis=0)
    lim = 2.0 * 2.0 ** -14 * kappa
    assert np.all(np.abs(got - want) <= lim), float(np.max(np.abs(got - want) - lim))
