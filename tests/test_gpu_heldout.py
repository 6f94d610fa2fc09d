"""The local-energy check of the Kagome 6x6x3 workload (108 sites, L = 4, F = 32, weight
scale 0.1, the benchmark's parameters): the incremental local energy on 1024 held-out
configurations -- uniform random S_z = 0 states from a seed the benchmark does not draw --
against the FP64 oracle (on the BF16-rounded W), in both tensor-core precisions.  The GPU
call has the benchmark's launch configuration: 16384 configurations, the held-out ones at
every 16th position among other random states.  Reports
the max and median per-sample relative error; the batch-mean energy must agree within
1e-4 relative and, for BF16X2, every sample within 1e-5.  The oracle runs over the host
cores in a spawn pool (started before any GPU call of this module)."""
import multiprocessing as mp
import os

import numpy as np
import pytest

from paper_2011_12453_gb300 import workloads as W

pytestmark = pytest.mark.gpu

F, L, N_HELD, SEED, N_LAUNCH = 32, 4, 1024, 20211, 16384
_POOL = {}


def _oracle_chunk(args):
    th, spins = args
    os.environ["OMP_NUM_THREADS"] = "1"
    from oracle import gcn, heisenberg
    from paper_2011_12453_gb300 import workloads as Wk

    g = Wk.kagome(6)
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    return heisenberg.local_energy(lambda x: gcn.logpsi_complex(th, F, L, Ah, x), g.edges, g.J, spins)


def _round_w(th):
    import torch

    out = th.copy()
    o = 3 * F
    out[o:o + 2 * F * F] = torch.tensor(out[o:o + 2 * F * F], dtype=torch.float32).to(torch.bfloat16).double().numpy()
    return out


@pytest.fixture(scope="module")
def oracle_energies():
    """The oracle's E_loc of the held-out set, started in a spawn pool before the GPU is used."""
    import torch

    g = W.kagome(6)
    theta = torch.tensor(W.random_theta(F, L, seed=0, scale=0.1), dtype=torch.float32)
    th = _round_w(theta.double().numpy())
    spins = W.random_spins(g.n_sites, N_HELD, seed=SEED)
    workers = max(1, min(16, os.cpu_count() or 1))
    chunks = np.array_split(np.arange(N_HELD), workers * 4)
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        parts = pool.map(_oracle_chunk, [(th, spins[c]) for c in chunks])
    return theta, spins, np.concatenate(parts)


@pytest.mark.parametrize("prec_name", ["bf16", "bf16x2"])
def test_heldout_local_energy_kagome108(oracle_energies, prec_name):
    import torch

    from paper_2011_12453_gb300 import build as B, gna

    theta_cpu, spins, want = oracle_energies
    B.build()
    torch.cuda.set_device(0)
    g = W.kagome(6)
    graph = gna.Graph.from_workload(g, L)
    model = gna.Model(F, L, gna.PREC_BF16 if prec_name == "bf16" else gna.PREC_BF16X2)
    theta = theta_cpu.cuda()
    batch = W.random_spins(g.n_sites, N_LAUNCH, seed=SEED + 1)
    pos = np.arange(N_HELD) * (N_LAUNCH // N_HELD)
    batch[pos] = spins
    gna.device_status(clear=True)  # the status word is sticky: start from a clean one
    E = gna.local_energy(graph, model, theta, torch.tensor(batch, device="cuda"), gna.ELOC_INCREMENTAL).cpu().numpy()
    assert gna.device_status(clear=True) == 0
    got = E[pos, 0] + 1j * E[pos, 1]
    rel = np.abs(got - want) / np.abs(want)
    mean_rel = abs(got.real.mean() - want.real.mean()) / abs(want.real.mean())
    print(f"\n{prec_name} held-out E_loc on {N_HELD} configurations: per-sample relative error max {rel.max():.2e} "
          f"median {np.median(rel):.2e}; batch-mean {mean_rel:.2e}")
    assert mean_rel <= 1e-4
    if prec_name == "bf16x2":
        assert rel.max() <= 1e-5
