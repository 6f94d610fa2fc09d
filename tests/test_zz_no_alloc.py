"""gna_backward_static -- the backward for callers that cannot allocate device memory --
must give the same gradient as gna_backward (which takes a caller-supplied workspace).

It is called twice in a row on each case: every call reuses the library's one fixed
scratch array, so the second call also shows that nothing left there by the first one
leaks into the result.  Collected last (file name), so a stop-at-first-failure run has
already run every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

from paper_2011_12453_gb300 import build as B, gna, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t

    B.build()
    t.cuda.set_device(0)
    return t


CASES = [
    # (graph, F, L, precision, shared, batch, tolerance)
    ("kagome2", 16, 2, gna.PREC_FP64, True, 37, 1e-10),
    ("er18", 16, 3, gna.PREC_FP64, False, 41, 1e-10),
    ("kagome6", 32, 4, gna.PREC_FP32, True, 256, 1e-5),
    ("tri12", 48, 4, gna.PREC_FP32, True, 64, 1e-5),  # features do not fit in shared memory
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] + ("_fp64" if c[3] == 0 else "_fp32") for c in CASES])
def test_backward_static_matches_backward(torch, case):
    name, F, L, prec, shared, Bn, tol = case
    g = {"kagome2": W.kagome(2), "er18": W.erdos_renyi(18, 0.25, seed=2), "kagome6": W.kagome(6),
         "tri12": W.triangular(12, 12)}[name]
    graph = gna.Graph.from_workload(g, L)
    model = gna.Model(F, L, prec, shared)
    theta = torch.tensor(W.random_theta(F, L, seed=4, scale=0.3, shared=shared), dtype=model.theta_dtype(),
                         device="cuda")
    s = torch.tensor(W.random_spins(g.n_sites, Bn, seed=5), device="cuda")
    cot = torch.tensor(np.random.default_rng(6).normal(size=(Bn, 2)), device="cuda")
    want = gna.backward(graph, model, theta, s, cot).cpu().numpy()
    scale = max(1.0, np.abs(want).max())
    for _ in range(2):
        got = gna.backward_static(graph, model, theta, s, cot).cpu().numpy()
        assert np.abs(got - want).max() <= tol * scale
