"""gna_backward_static -- the backward for callers that cannot allocate device memory --
must give the gradient of gna_backward (which takes a caller-supplied workspace).

It is called twice in a row on each case: every call reuses the library's one fixed
scratch array, so the second call also shows that nothing left there by the first one
leaks into the result.  Cases cover the FP64/FP32 SIMT backward and the tensor-core
backward of BF16 and BF16X2 models, each with a grid as large as gna_backward's and with a
grid reduced to fit the array (triangular 12x12 at F = 48: about 0.5 MB of per-block
storage in FP64, 0.24 MB for the tensor-core kernel, so fewer blocks than SMs fit in the
32 MiB array and each block takes several samples).  A block never needs the whole array
with the library's limits (n_sites <= 4096, F <= 64, L <= 8: at most 27.4 MB per block), so
the GNA_ERR_WORKSPACE branch cannot be reached with a valid model.

Collected last (file name), so a stop-at-first-failure run has already run every other
test; it also passes alone in a fresh process."""
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
    # (graph, F, L, precision, shared, batch, tolerance against gna_backward; the tensor-core
    # cases use the bound below)
    ("kagome2", 16, 2, gna.PREC_FP64, True, 37, 1e-10),
    ("er18", 16, 3, gna.PREC_FP64, False, 41, 1e-10),
    ("kagome6", 32, 4, gna.PREC_FP32, True, 256, 1e-5),
    ("tri12", 48, 4, gna.PREC_FP32, True, 64, 1e-5),    # features do not fit in shared memory
    ("tri12", 48, 4, gna.PREC_FP64, True, 300, 1e-10),  # grid reduced to fit the array
    ("kagome6", 32, 4, gna.PREC_BF16, True, 256, 1e-5),
    ("tri12", 48, 4, gna.PREC_BF16X2, True, 300, 1e-5),  # tensor-core backward, grid reduced
]
NAMES = {gna.PREC_FP64: "fp64", gna.PREC_FP32: "fp32", gna.PREC_BF16: "bf16", gna.PREC_BF16X2: "bf16x2"}


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}_{NAMES[c[3]]}_B{c[5]}" for c in CASES])
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
    lim = tol * np.maximum(np.abs(want), 1.0)
    if prec in (gna.PREC_BF16, gna.PREC_BF16X2):
        # the tensor-core backward accumulates each block's samples in FP32, and the two calls
        # group the samples into blocks differently (the static call may have fewer blocks):
        # both are within 2^-14 sum_x |cot_x . d log Psi_x / d theta| of the exact gradient
        from oracle import gcn, isgo

        th = theta.double().cpu().numpy()
        o = 3 * F
        th[o:o + 2 * F * F] = torch.tensor(th[o:o + 2 * F * F], dtype=torch.float32).to(torch.bfloat16).double().numpy()
        Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
        x, c = s.cpu().numpy(), cot.cpu().numpy()
        kappa = sum(np.abs(isgo.backward(th, F, L, Ah, x[k:k + 1], c[k:k + 1])) for k in range(Bn))
        lim = 2.0 * 2.0 ** -14 * kappa
    for _ in range(2):
        got = gna.backward_static(graph, model, theta, s, cot).cpu().numpy()
        assert np.all(np.abs(got - want) <= lim), float(np.max(np.abs(got - want) - lim))
