"""Failure detection without a GPU fault: the conditions kernels record in the device status
word (read by gna_device_status), each made on the host or by a launch argument.

* Degenerate importance weights (the failure the paper warns of when samples are reused
  too long: a few samples carry the weights): one sample's weight dominates, so the
  effective sample size falls below 1% of the batch -> bit 4, GNA_WARN_DEGENERATE_WEIGHTS.
* A non-finite parameter injected on the host -> bit 2, GNA_ERR_NONFINITE.
* A bounded MMA wait given a limit of 0 iterations (a launch argument, not a fault): the
  wait gives up, the kernel waits for the MMAs it issued, frees its tensor memory and
  returns -> bit 1, GNA_ERR_TIMEOUT; the context stays usable and the next call with the
  default limit gives the normal result."""
import numpy as np
import pytest

from paper_2011_12453_gb300 import build as B, gna, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t

    B.build()
    t.cuda.set_device(0)
    gna.device_status(clear=True)
    yield t
    gna.debug_wait_limit(None)
    gna.device_status(clear=True)


def test_degenerate_weights_warning(torch):
    Bn = 1000
    rng = np.random.default_rng(0)
    E = torch.tensor(rng.normal(size=(Bn, 2)), device="cuda")
    lp0 = torch.zeros((Bn, 2), dtype=torch.float64, device="cuda")
    # balanced weights: no condition
    lp = torch.tensor(rng.normal(scale=0.1, size=(Bn, 2)), device="cuda")
    _, stats = gna.isgo_weights(lp, lp0, E)
    flags, st = gna.device_status(clear=True, with_status=True)
    assert flags == 0 and st == gna.GNA_OK and float(stats[3]) > 0.5 * Bn
    # one sample carries the weights: ESS ~ 1 < 0.01 * 1000
    lp[0, 0] = 20.0
    _, stats = gna.isgo_weights(lp, lp0, E)
    flags, st = gna.device_status(clear=True, with_status=True)
    assert float(stats[3]) < 0.01 * Bn
    assert flags == 4 and st == gna.GNA_WARN_DEGENERATE_WEIGHTS
    # with counts the threshold is 1% of the copies
    counts = torch.full((Bn,), 3.0, dtype=torch.float64, device="cuda")
    lp[0, 0] = 0.0
    gna.isgo_weights(lp, lp0, E, counts)
    assert gna.device_status(clear=True) == 0


@pytest.mark.parametrize("prec", [gna.PREC_FP64, gna.PREC_BF16X2])
def test_nonfinite_parameter_is_flagged(torch, prec):
    g = W.kagome(2)
    F, L = 16, 2
    graph = gna.Graph.from_workload(g, L)
    model = gna.Model(F, L, prec)
    theta = torch.tensor(W.random_theta(F, L, seed=0, scale=0.3), dtype=model.theta_dtype(), device="cuda")
    s = torch.tensor(W.random_spins(g.n_sites, 32, seed=1), device="cuda")
    lp0 = gna.forward(graph, model, theta, s)
    gna.isgo_grad(graph, model, theta, s, lp0)
    assert gna.device_status(clear=True) == 0
    bad = theta.clone()
    bad[3 * F + 5] = float("nan")  # one entry of W
    gna.isgo_grad(graph, model, bad, s, lp0)
    flags, st = gna.device_status(clear=True, with_status=True)
    assert flags & 2 and st == gna.GNA_ERR_NONFINITE


def test_wait_timeout_is_reported_and_the_context_stays_usable(torch):
    g = W.kagome(6)
    F, L = 32, 4
    graph = gna.Graph.from_workload(g, L)
    model = gna.Model(F, L, gna.PREC_BF16)
    theta = torch.tensor(W.random_theta(F, L, seed=0, scale=0.1), dtype=torch.float32, device="cuda")
    s = torch.tensor(W.random_spins(g.n_sites, 600, seed=2), device="cuda")
    want = gna.local_energy(graph, model, theta, s, gna.ELOC_INCREMENTAL).cpu().numpy()
    assert gna.device_status(clear=True) == 0
    try:
        gna.debug_wait_limit(0)
        gna.local_energy(graph, model, theta, s, gna.ELOC_INCREMENTAL)
        torch.cuda.synchronize()
    finally:
        gna.debug_wait_limit(None)
    flags, st = gna.device_status(clear=True, with_status=True)
    assert flags & 1 and st == gna.GNA_ERR_TIMEOUT
    again = gna.local_energy(graph, model, theta, s, gna.ELOC_INCREMENTAL).cpu().numpy()
    assert gna.device_status(clear=True) == 0
    assert np.array_equal(again, want)
