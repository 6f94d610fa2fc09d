"""The learned exchange proposal on the random-graph workload as specified: 32 Erdos-Renyi
graphs (sizes uniform in 32..96, mean degree 4, J uniform in [0.5, 1.5]), GCN L = 3, F = 32,
4096 chains per graph.  On each graph psi is first trained by ISGO (20 iterations of 2
sweeps and 5 reuse steps on the tensor-core path, BF16X2; the best state with ESS > C/2
kept; when no iteration keeps that ESS, psi stays at its initial parameters), the proposal network is trained on the chains' own samples (per-bond Delta log Psi
targets, Adam).  The chains are then equilibrated by sweeps of learned moves (the
trained wavefunctions are peaked, and plain exchange moves take long to reach their
high-probability states; 60 sweeps), and from that state, after 20 sweeps of warm-up each, 60 sweeps
of plain and of learned moves (both on the FP32 warp-per-chain sampler, the one that runs
learned moves) give the local-energy series of every chain: integrated autocorrelation
time (Sokal window), effective samples and effective samples per second of device sampling
time, and the mean energy with its standard error.

Asserted: both samplers give the same energy on every graph (within 5 combined standard
errors), the learned moves are accepted more often per step than the plain ones, and the
chains keep S_z.  Reported (printed, not asserted): tau_int and ESS/s of both samplers
over the 32 graphs -- the gain in effective samples per second is the question this
measurement answers, and the answer may be negative."""
import numpy as np
import pytest

from paper_2011_12453_gb300 import build as B, gna, workloads as W

pytestmark = pytest.mark.gpu

F, L, C = 32, 3, 4096
ISGO_ITERS, EQUIL, WARM, SERIES = 20, 60, 20, 60


@pytest.fixture(scope="module")
def torch():
    import torch as t

    B.build()
    t.cuda.set_device(0)
    return t


def test_learned_proposal_on_the_random_graph_set(torch):
    from paper_2011_12453_gb300 import vmc

    graphs = W.random_graph_set(32)
    rows = []
    for gi, g in enumerate(graphs):
        graph = gna.Graph.from_workload(g, L)
        model = gna.Model(F, L, gna.PREC_FP32)
        mx2 = gna.Model(F, L, gna.PREC_BF16X2)
        theta = torch.tensor(W.random_theta(F, L, gi, 0.3), dtype=torch.float32, device="cuda")
        n_up = g.n_sites // 2
        ch = vmc.Chains(graph, mx2, theta, W.random_spins(g.n_sites, C, 100 + gi, n_up=n_up), seed=5 + gi)
        ch.sweep(10)
        best = (np.inf, theta.clone(), ch.spins.clone())
        for _ in range(ISGO_ITERS):
            st = vmc.isgo_iteration(ch, K=5, lr=5e-4, sweeps=2)
            if np.isfinite(st[-1, 0]) and st[-1, 0] < best[0] and st[-1, 3] > 0.5 * C:
                best = (float(st[-1, 0]), theta.clone(), ch.spins.clone())
        theta.copy_(best[1])
        ch = vmc.Chains(graph, mx2, theta, best[2], seed=17 + gi)
        ch.sweep(10)
        prop = torch.tensor(W.random_proposal_params(1 + gi, 0.3), dtype=torch.float32, device="cuda")
        state = None
        for _ in range(4):
            ch.sweep(2)
            _, state = vmc.train_proposal(graph, mx2, theta, ch.spins, prop, 50, 3e-3, state)
        eq = vmc.Chains(graph, model, theta, ch.spins.clone(), seed=55 + gi)
        eq.sweep(EQUIL, proposal=prop)
        res = {}
        for name, p in (("plain", None), ("learned", prop)):
            c2 = vmc.Chains(graph, model, theta, eq.spins.clone(), seed=99 + gi)
            c2.sweep(WARM, proposal=p)
            a0 = c2.accepted.sum().item()
            series, secs = vmc.energy_series(c2, SERIES, proposal=p, energy_model=mx2)
            tau, ess, _ = vmc.ess_per_second(series, secs)
            means = series.mean(axis=0)
            x = c2.spins.cpu().numpy()
            assert np.all((x > 0).sum(1) == n_up)
            res[name] = dict(E=float(series.mean()), err=float(means.std() / np.sqrt(C)), tau=tau, ess=ess,
                             secs=secs, acc=(c2.accepted.sum().item() - a0) / (SERIES * C * g.n_sites))
        pl, le = res["plain"], res["learned"]
        assert abs(pl["E"] - le["E"]) < 5 * np.hypot(pl["err"], le["err"]), (gi, pl, le)
        rows.append((g.n_sites, best[0], pl, le))
    acc_p = np.mean([r[2]["acc"] for r in rows])
    acc_l = np.mean([r[3]["acc"] for r in rows])
    ess_p = sum(r[2]["ess"] for r in rows) / sum(r[2]["secs"] for r in rows)
    ess_l = sum(r[3]["ess"] for r in rows) / sum(r[3]["secs"] for r in rows)
    tau_p = np.mean([r[2]["tau"] for r in rows])
    tau_l = np.mean([r[3]["tau"] for r in rows])
    wins = sum(r[3]["ess"] / r[3]["secs"] > r[2]["ess"] / r[2]["secs"] for r in rows)
    print(f"\nrandom-graph set (32 graphs, {C} chains, {EQUIL} + {WARM} + {SERIES} sweeps): acceptance per step plain {acc_p:.4f} "
          f"learned {acc_l:.4f}; tau_int (sweeps) plain {tau_p:.2f} learned {tau_l:.2f}; ESS/s plain {ess_p:.0f} "
          f"learned {ess_l:.0f} (ratio {ess_l / ess_p:.3f}; learned ahead on {wins} of 32 graphs)")
    for n, e, pl, le in rows:
        print(f"  n={n:3d} E_train={e:9.3f} E plain {pl['E']:9.4f}+-{pl['err']:.4f} learned {le['E']:9.4f}+-"
              f"{le['err']:.4f} tau {pl['tau']:.2f}/{le['tau']:.2f} ESS/s {pl['ess'] / pl['secs']:.0f}/"
              f"{le['ess'] / le['secs']:.0f}")
    assert acc_l > acc_p
