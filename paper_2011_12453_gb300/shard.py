"""Sample-sharded ISGO step across processes (the scaling section of arXiv:2011.12453:
data-parallel workers each hold a block of the samples; the weight sums and the energy
are summed across workers, then the gradient).

Partitioning: each process holds a contiguous block of the chains (and so of the
samples); every per-sample step -- forward, local energy, weights, cotangents, backward --
runs on the process that holds the sample.  Four collectives per ISGO gradient, all on
small device tensors (no host synchronisation):

  1. max over shards of the largest log weight m (the common shift of the log-sum-exp);
  2. sum of each shard's (S, S Re E, S Im E) rescaled by exp(m_shard - m), giving the
     normalisation S and Ebar;
  3. sum of each shard's (sum p |E - Ebar|^2, sum p^2/c, sum c): variance, 1/ESS, copies;
  4. sum of each shard's part of the gradient (P float64 values).

The arithmetic of each shard runs in the library's kernels (gna_isgo_partials,
gna_isgo_finish, gna_backward); this module only composes them with the collectives.
"""
from __future__ import annotations

from . import gna


class DistComm:
    """Collectives of a torch.distributed process group (NCCL for CUDA tensors, gloo for
    CPU tensors), in place."""

    def __init__(self, group=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group

    def max_(self, t):
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return t

    def sum_(self, t):
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return t


class LibraryKernels:
    """The per-shard steps on the device, through the library's C ABI."""

    def __init__(self, graph: gna.Graph, model: gna.Model):
        self.graph, self.model = graph, model

    def forward(self, theta, spins):
        return gna.forward(self.graph, self.model, theta, spins)

    def local_energy(self, theta, spins):
        return gna.local_energy(self.graph, self.model, theta, spins, gna.ELOC_INCREMENTAL)

    def partials(self, lp, lp0, E, counts):
        return gna.isgo_partials(lp, lp0, E, counts)

    def finish(self, lp, lp0, E, global4, counts):
        return gna.isgo_finish(lp, lp0, E, global4, counts)

    def backward(self, theta, spins, cot):
        return gna.backward(self.graph, self.model, theta, spins, cot)


def combine_partials(part4, comm):
    """(m, S, S Re E, S Im E) of this shard -> the global (m, S, Re Ebar, Im Ebar), same device."""
    import torch

    m = part4[0:1].clone()
    comm.max_(m)
    f = torch.where(part4[0] > float("-inf"), torch.exp(part4[0] - m[0]), torch.zeros_like(part4[0]))
    sums = part4[1:4] * f
    comm.sum_(sums)
    return torch.stack([m[0], sums[0], sums[1] / sums[0], sums[2] / sums[0]])


def combine_stats(global4, part3, comm):
    """Global statistics (Re Ebar, Im Ebar, var, ess) and the number of copies."""
    import torch

    p3 = part3.clone()
    comm.sum_(p3)
    return torch.stack([global4[2], global4[3], p3[0], 1.0 / p3[1]]), p3[2]


def isgo_grad(kernels, theta, spins, logpsi0, comm, counts=None):
    """One ISGO gradient (Eq. isgo) over the samples of all shards: (grad [P], stats [4],
    copies), identical on every shard.  spins, logpsi0 and counts are this shard's block."""
    lp = kernels.forward(theta, spins)
    E = kernels.local_energy(theta, spins)
    g4 = combine_partials(kernels.partials(lp, logpsi0, E, counts), comm)
    cot, part3 = kernels.finish(lp, logpsi0, E, g4, counts)
    stats, copies = combine_stats(g4, part3, comm)
    grad = kernels.backward(theta, spins, cot)
    comm.sum_(grad)
    return grad, stats, copies


def shard_range(n: int, rank: int, world: int):
    """The contiguous block [lo, hi) of n items that `rank` of `world` holds (sizes differ by
    at most one)."""
    return n * rank // world, n * (rank + 1) // world
