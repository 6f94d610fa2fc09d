"""gna_local_energy_logpsi -- the incremental local energy and log Psi in one call (on the
tensor cores the local-energy kernel's own forward gives log Psi) -- must return exactly what
gna_local_energy (incremental) and gna_forward return, in every precision, and isgo_grad,
which now uses it, exactly what the composition forward -> local energy -> weights ->
backward gives."""
import numpy as np
import pytest

from paper_2011_12453_gb300 import build as B, gna, workloads as W

pytestmark = pytest.mark.gpu

PRECS = {"fp64": gna.PREC_FP64, "fp32": gna.PREC_FP32, "bf16": gna.PREC_BF16, "bf16x2": gna.PREC_BF16X2}
CASES = [("kagome6", 32, 4, 600), ("tri12", 48, 4, 300)]


@pytest.fixture(scope="module")
def torch():
    import torch as t

    B.build()
    t.cuda.set_device(0)
    return t


def _setup(torch, name, F, L, Bn, prec):
    g = {"kagome6": W.kagome(6), "tri12": W.triangular(12, 12)}[name]
    graph = gna.Graph.from_workload(g, L)
    model = gna.Model(F, L, prec)
    theta = torch.tensor(W.random_theta(F, L, 0, scale=0.3), dtype=model.theta_dtype(), device="cuda")
    s = torch.tensor(W.random_spins(g.n_sites, Bn, 7), device="cuda")
    return graph, model, theta, s


@pytest.mark.parametrize("prec_name", list(PRECS))
@pytest.mark.parametrize("name,F,L,Bn", CASES)
def test_fused_equals_separate_calls(torch, name, F, L, Bn, prec_name):
    graph, model, theta, s = _setup(torch, name, F, L, Bn, PRECS[prec_name])
    gna.device_status(clear=True)  # the status word is sticky: start from a clean one
    E, lp = gna.local_energy_logpsi(graph, model, theta, s)
    E_ref = gna.local_energy(graph, model, theta, s, gna.ELOC_INCREMENTAL)
    lp_ref = gna.forward(graph, model, theta, s)
    assert gna.device_status(clear=True) == 0
    assert np.array_equal(E.cpu().numpy(), E_ref.cpu().numpy())
    assert np.array_equal(lp.cpu().numpy(), lp_ref.cpu().numpy())
    # B = 0 is a no-op
    gna.local_energy_logpsi(graph, model, theta, s[:0])


@pytest.mark.parametrize("prec_name", list(PRECS))
def test_isgo_grad_equals_composition(torch, prec_name):
    graph, model, theta, s = _setup(torch, "kagome6", 32, 4, 400, PRECS[prec_name])
    lp0 = gna.forward(graph, model, theta, s) + 0.01 * torch.randn(400, 2, dtype=torch.float64, device="cuda")
    grad, stats = gna.isgo_grad(graph, model, theta, s, lp0)
    lp = gna.forward(graph, model, theta, s)
    E = gna.local_energy(graph, model, theta, s, gna.ELOC_INCREMENTAL)
    cot, st = gna.isgo_weights(lp, lp0, E)
    g_ref = gna.backward(graph, model, theta, s, cot)
    assert np.array_equal(stats.cpu().numpy(), st.cpu().numpy())
    assert np.array_equal(grad.cpu().numpy(), g_ref.cpu().numpy())
