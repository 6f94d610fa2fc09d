"""Host driver of the method's outer loops on top of the C ABI (no arithmetic of its own
beyond bookkeeping and statistics):

* ISGO iterations (scaling section and Eq. isgo of arXiv:2011.12453): sample with the
  current parameters, then reuse the samples for K gradient steps, each weighting the
  samples by |Psi|^2 / |Psi^0|^2 -- isgo_grad followed by the SGD update, all on the
  device; only the four statistics come back to the host.
* Training of the learned exchange proposal on the chains' own samples (per-bond
  Delta log Psi from the local-energy call as targets, Adam steps on the device).
* Integrated autocorrelation time of an observable series (Sokal's automatic window)
  and effective samples per second, to compare proposals.
"""
from __future__ import annotations

import time

import numpy as np

from . import gna


class Chains:
    """C Metropolis chains of one model on one graph, with a running step counter."""

    def __init__(self, graph: gna.Graph, model: gna.Model, theta, spins0, seed: int):
        import torch

        self.graph, self.model, self.theta = graph, model, theta
        self.spins = torch.as_tensor(spins0, device=theta.device).contiguous()
        self.seed = seed
        self.step = 0
        self.accepted = torch.zeros(self.spins.shape[0], dtype=torch.int32, device=theta.device)

    def sweep(self, n_sweeps: int, record_every: int = 0, proposal=None, eps: float = 0.1, trace: bool = False):
        out = gna.metropolis_sweep(self.graph, self.model, self.theta, self.spins, n_sweeps, record_every, self.seed,
                                   self.step, trace=trace, n_accepted=self.accepted, proposal=proposal, eps=eps)
        self.step += n_sweeps * self.graph.n_sites
        return out


def isgo_iteration(chains: Chains, K: int, lr: float, sweeps: int = 1, group: bool = False):
    """One ISGO iteration: `sweeps` sweeps then one recorded sample per chain, reused for K
    updates of theta; with group=True duplicated samples are first grouped into unique
    states with counts (scaling section).  log Psi^0 is the sampler's record, except for
    the tensor-core precisions, whose sampler computes in BF16 while the forward may not
    (BF16X2): there it is evaluated by the forward at the sampling parameters, the function
    that evaluates log Psi at the later parameters, so that the weights are 1 at theta^0.
    Returns the statistics [K][4] (Re E, Im E, var, ESS) on the host."""
    import torch

    samples, lp0, _, _ = chains.sweep(sweeps, record_every=sweeps)
    s = samples[-1].contiguous()
    l0 = lp0[-1].contiguous()
    counts = None
    if group:
        s, l0, counts = gna.dedup(s, l0)
        s, l0, counts = s.contiguous(), l0.contiguous(), counts.contiguous()
    if chains.model.prec in (gna.PREC_BF16, gna.PREC_BF16X2):
        l0 = gna.forward(chains.graph, chains.model, chains.theta, s)
    stats = torch.empty((K, 4), dtype=torch.float64, device=s.device)
    grad = torch.empty(chains.model.num_params, dtype=torch.float64, device=s.device)
    for k in range(K):
        gna.isgo_grad(chains.graph, chains.model, chains.theta, s, l0, counts=counts, grad=grad, stats=stats[k])
        gna.sgd_update(chains.model, chains.theta, grad, lr)
    return stats.cpu().numpy()


def train_proposal(graph: gna.Graph, model: gna.Model, theta, spins, params, steps: int, lr: float = 3e-3,
                   adam_state=None):
    """Adam steps of the proposal network on configurations `spins` (targets from the
    incremental local-energy call).  Returns (losses, adam_state)."""
    import torch

    _, dl = gna.local_energy(graph, model, theta, spins, gna.ELOC_INCREMENTAL, bonds=True)
    if adam_state is None:
        adam_state = [torch.zeros_like(params), torch.zeros_like(params), 0]
    m, v, t = adam_state
    losses = []
    for _ in range(steps):
        t += 1
        grad, loss = gna.proposal_grad(graph, spins, dl, params)
        gna.proposal_adam(params, m, v, grad, t, lr)
        losses.append(loss)
    adam_state[2] = t
    return [float(x.item()) for x in losses], adam_state


def tau_int(x: np.ndarray, c: float = 5.0) -> float:
    """Integrated autocorrelation time with Sokal's automatic window (smallest M >= c tau)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    d = x - x.mean()
    var = float((d * d).mean())
    if var == 0.0:
        return 1.0
    tau, acc = 1.0, 0.0
    for M in range(1, n):
        acc += float((d[: n - M] * d[M:]).sum() / n / var)
        tau = 1.0 + 2.0 * acc
        if M >= c * tau:
            break
    return float(tau)


def energy_series(chains: Chains, n_sweeps: int, proposal=None, eps: float = 0.1, energy_model=None):
    """Local energy of every chain after each of n_sweeps sweeps: (E [n_sweeps][C] float64,
    device seconds spent sampling).  energy_model: the model (precision) of the local
    energies, default the chains' own."""
    import torch

    graph, theta = chains.graph, chains.theta
    model = chains.model if energy_model is None else energy_model
    C = chains.spins.shape[0]
    series = np.empty((n_sweeps, C))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_sample = 0.0
    for k in range(n_sweeps):
        e0.record()
        chains.sweep(1, proposal=proposal, eps=eps)
        e1.record()
        E = gna.local_energy(graph, model, theta, chains.spins, gna.ELOC_INCREMENTAL)
        torch.cuda.synchronize()
        t_sample += e0.elapsed_time(e1) / 1000.0
        series[k] = E[:, 0].cpu().numpy()
    return series, t_sample


def ess_per_second(series: np.ndarray, seconds: float):
    """(mean tau_int over chains, total effective samples, effective samples per second)."""
    taus = np.array([tau_int(series[:, c]) for c in range(series.shape[1])])
    ess = float((series.shape[0] / np.maximum(taus, 1.0)).sum())
    return float(taus.mean()), ess, ess / seconds
