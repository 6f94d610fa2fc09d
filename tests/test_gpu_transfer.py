"""Transfer of a trained GNA to a larger system and another geometry (the paper's
experiments: a GNA pretrained on 12 sites speeds up convergence on a larger Kagome lattice,
also when the pretraining geometry differs).  The GCN's parameters do not depend on the
number of sites (W, b shared over sites and layers), so parameters trained on a 12-site
graph apply unchanged to the Kagome 6x6x3 lattice (108 sites).

Hard-core bosons at t/V = 0.5, half filling; ReLU + layer norm, L = 3, F = 16, real head.
Pretraining: 40 ISGO iterations on Kagome 2x2x3 or triangular 3x4 (FP64).  Target: Kagome
6x6x3, FP32, 1024 chains, ISGO with K = 10 reuse steps, from the pretrained parameters and
from random ones.  Checked: without any training on the large lattice the pretrained
parameters already give an energy within 10 % of the best either run finds (the random
start is far from it), and after 30 iterations the pretrained run is at least as low as the
random one.  The iterations each run needs to come within 1 % of that best energy are
printed: with 1024 chains the random start also converges in a few iterations here, unlike
the gradient explosions the paper reports for random starts on 432 sites."""
import numpy as np
import pytest

from oracle import heisenberg as hz
from paper_2011_12453_gb300 import build as B, gna, vmc, workloads as W

pytestmark = pytest.mark.gpu

F, L, TV = 16, 3, 0.5


@pytest.fixture(scope="module")
def torch():
    import torch as t

    B.build()
    t.cuda.set_device(0)
    return t


def _real_theta(seed, scale=0.3):
    th = W.random_theta(F, L, seed=seed, scale=scale)
    P = th.size
    o_r = P - (F + 2) * 2 - 2
    th[o_r + 1:P - 2:2] = 0.0
    th[P - 1] = 0.0
    return th


def _train(torch, g, th, prec, iters, C, lr, seed):
    xxz = hz.hardcore_bosons(g.edges.shape[0], TV, 1.0)
    graph = gna.Graph(g.n_sites, g.edges, None, L, xxz=xxz)
    model = gna.Model(F, L, prec, act=gna.ACT_RELU_LN)
    theta = torch.tensor(th, dtype=model.theta_dtype(), device="cuda")
    chains = vmc.Chains(graph, model, theta, W.random_spins(g.n_sites, C, seed=seed), seed=seed)
    chains.sweep(4)  # burn-in
    traj = []
    for _ in range(iters):
        st = vmc.isgo_iteration(chains, 10, lr, sweeps=2)
        traj.append(st[0, 0] / g.n_sites)  # energy per site at the sampling parameters
    return theta.double().cpu().numpy(), np.array(traj)


def _iters_to(traj, target, tol=0.01):
    ok = np.nonzero(np.abs(traj - target) <= tol * abs(target))[0]
    return int(ok[0]) if ok.size else len(traj)


@pytest.mark.parametrize("source", ["kagome2", "tri34"])
def test_pretrained_parameters_transfer_to_kagome108(torch, source):
    g_small = {"kagome2": W.kagome(2), "tri34": W.triangular(3, 4)}[source]
    th_pre, traj_small = _train(torch, g_small, _real_theta(0), gna.PREC_FP64, 40, 1024, 0.05, 1)
    big = W.kagome(6)
    lr = 0.05 * 12 / big.n_sites  # the gradient of the total energy grows with the number of sites
    iters = 30
    _, traj_pre = _train(torch, big, th_pre, gna.PREC_FP32, iters, 1024, lr, 2)
    _, traj_rnd = _train(torch, big, _real_theta(3), gna.PREC_FP32, iters, 1024, lr, 2)
    best = min(traj_pre.min(), traj_rnd.min())
    n_pre, n_rnd = _iters_to(traj_pre, best), _iters_to(traj_rnd, best)
    print(f"\n{source} -> kagome108: small E/N {traj_small[-1]:.5f}; start E/N pretrained {traj_pre[0]:.5f} "
          f"random {traj_rnd[0]:.5f}; best {best:.5f}; iterations to 1%: pretrained {n_pre} random {n_rnd}")
    print("pretrained", np.array2string(traj_pre, precision=4, max_line_width=200))
    print("random    ", np.array2string(traj_rnd, precision=4, max_line_width=200))
    assert np.all(np.isfinite(traj_pre)) and np.all(np.isfinite(traj_rnd))
    assert abs(traj_pre[0] - best) <= 0.1 * abs(best)
    assert abs(traj_rnd[0] - best) > 0.5 * abs(best)
    # energies per site are negative here: "as low" with a margin of 0.1 % for sampling noise
    assert traj_pre[-5:].mean() <= traj_rnd[-5:].mean() + 1e-3 * abs(best)


@pytest.mark.parametrize("source", ["kagome2", "tri34"])
def test_pretrained_parameters_transfer_to_kagome432(torch, source):
    # the paper's scale: Kagome 12x12x3 (432 sites) from parameters pretrained on 12 sites
    # (Kagome 2x2x3, or triangular 3x4: another geometry), against a random start, both with the same ISGO schedule (1024 chains, 2 sweeps and
    # K = 10 per iteration, the learning rate scaled by 12 / N as above).  Checked: the
    # transferred parameters start within 10 % of the best energy either run finds and much
    # closer to it than the random start.  Printed, not asserted: the trajectories and the
    # iterations each run needs to come within 1 % of the best (whether a run destabilises
    # on the way is what this measures, and it depends on the pretraining geometry).
    g_small = {"kagome2": W.kagome(2), "tri34": W.triangular(3, 4)}[source]
    th_pre, traj_small = _train(torch, g_small, _real_theta(0), gna.PREC_FP64, 40, 1024, 0.05, 1)
    big = W.kagome(12)
    lr = 0.05 * 12 / big.n_sites
    iters = 40
    _, traj_pre = _train(torch, big, th_pre, gna.PREC_FP32, iters, 1024, lr, 2)
    _, traj_rnd = _train(torch, big, _real_theta(3), gna.PREC_FP32, iters, 1024, lr, 2)
    assert np.all(np.isfinite(traj_pre)) and np.all(np.isfinite(traj_rnd))
    best = min(traj_pre.min(), traj_rnd.min())
    n_pre, n_rnd = _iters_to(traj_pre, best), _iters_to(traj_rnd, best)
    print(f"\n{source} -> kagome432: small E/N {traj_small[-1]:.5f}; start E/N pretrained {traj_pre[0]:.5f} "
          f"random {traj_rnd[0]:.5f}; best {best:.5f}; iterations to 1%: pretrained {n_pre} random {n_rnd}")
    print("pretrained", np.array2string(traj_pre, precision=4, max_line_width=200))
    print("random    ", np.array2string(traj_rnd, precision=4, max_line_width=200))
    assert abs(traj_pre[0] - best) <= 0.1 * abs(best)
    assert abs(traj_pre[0] - best) < 0.5 * abs(traj_rnd[0] - best)
