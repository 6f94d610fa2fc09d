"""Sample-sharded ISGO on CPU (gloo, world size 2): paper_2011_12453_gb300.shard composes the
per-shard steps with the four collectives (max of the log-weight shift; sums of the weight
sums and energies; of the variance, 1/ESS and copies; of the gradient).  With the per-shard
steps taken from the FP64 oracle, the gradient and statistics of two shards of unequal
size (contiguous blocks of an odd number of samples, with counts) equal the
single-process ISGO gradient of all samples to 1e-12, on both ranks."""
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
F, L, NB = 16, 2, 37


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    from oracle import gcn
    from paper_2011_12453_gb300 import workloads as W

    g = W.kagome(2)
    th = W.random_theta(F, L, seed=3, scale=0.5)
    th0 = th - W.random_theta(F, L, seed=4, scale=0.05)
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    s = W.random_spins(g.n_sites, NB, seed=5)
    lp0 = gcn.logpsi(th0, F, L, Ah, s)
    counts = np.random.default_rng(6).integers(1, 4, size=NB).astype(np.float64)
    return g, th, Ah, s, lp0, counts


class OracleKernels:
    """The per-shard steps restated with the FP64 oracle (CPU tensors), with the contract of
    the library's gna_isgo_partials / gna_isgo_finish."""

    def __init__(self, g, th, Ah):
        self.g, self.th, self.Ah = g, th, Ah

    def forward(self, theta, spins):
        import torch
        from oracle import gcn

        return torch.tensor(gcn.logpsi(self.th, F, L, self.Ah, spins.numpy()))

    def local_energy(self, theta, spins):
        import torch
        from oracle import gcn, heisenberg

        E = heisenberg.local_energy(lambda x: gcn.logpsi_complex(self.th, F, L, self.Ah, x), self.g.edges, self.g.J,
                                    spins.numpy())
        return torch.tensor(np.stack([E.real, E.imag], axis=1))

    @staticmethod
    def _logw(lp, lp0, counts):
        lw = 2.0 * (lp[:, 0] - lp0[:, 0]).numpy()
        return lw + (np.log(counts.numpy()) if counts is not None else 0.0)

    def partials(self, lp, lp0, E, counts):
        import torch

        lw = self._logw(lp, lp0, counts)
        m = lw.max()
        w = np.exp(lw - m)
        return torch.tensor([m, w.sum(), (w * E[:, 0].numpy()).sum(), (w * E[:, 1].numpy()).sum()])

    def finish(self, lp, lp0, E, g4, counts):
        import torch

        lw = self._logw(lp, lp0, counts)
        g = g4.numpy()
        p = np.exp(lw - g[0]) / g[1]
        dr, di = E[:, 0].numpy() - g[2], E[:, 1].numpy() - g[3]
        c = counts.numpy() if counts is not None else np.ones(len(p))
        cot = torch.tensor(np.stack([2 * p * dr, 2 * p * di], axis=1))
        return cot, torch.tensor([(p * (dr * dr + di * di)).sum(), (p * p / c).sum(), c.sum()])

    def backward(self, theta, spins, cot):
        import torch
        from oracle import isgo

        return torch.tensor(isgo.backward(self.th, F, L, self.Ah, spins.numpy(), cot.numpy()))


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from paper_2011_12453_gb300 import shard

    dist.init_process_group("gloo", rank=rank, world_size=world)
    g, th, Ah, s, lp0, counts = _problem()
    lo, hi = shard.shard_range(NB, rank, world)
    grad, stats, copies = shard.isgo_grad(OracleKernels(g, th, Ah), None, torch.tensor(s[lo:hi]),
                                          torch.tensor(lp0[lo:hi]), shard.DistComm(),
                                          counts=torch.tensor(counts[lo:hi]))
    out.put((rank, hi - lo, grad.numpy(), stats.numpy(), float(copies)))
    dist.destroy_process_group()


def test_sharded_isgo_equals_single_process_gloo():
    import torch.multiprocessing as mp

    from oracle import isgo

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] + res[1][1] == NB and res[0][1] != res[1][1]
    g, th, Ah, s, lp0, counts = _problem()
    g_o, Ebar, var, ess, _, _ = isgo.isgo_gradient(th, F, L, Ah, g.edges, g.J, s, lp0[:, 0] + 1j * lp0[:, 1],
                                                   counts=counts)
    want = np.array([Ebar.real, Ebar.imag, var, ess])
    for _, _, grad, stats, copies in res:
        assert np.all(np.abs(grad - g_o) <= 1e-12 * np.maximum(np.abs(g_o), np.abs(g_o).max()))
        assert np.all(np.abs(stats - want) <= 1e-12 * np.maximum(np.abs(want), 1.0))
        assert copies == counts.sum()
    assert np.array_equal(res[0][2], res[1][2])
