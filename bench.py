"""Benchmark of the GNA-VMC hot path on one GB300 (or N replicas under torchrun).

Workload: Kagome 6x6x3 (108 sites, 216 bonds, periodic), Heisenberg J = 1, GCN with
L = 4 layers of width F = 32 (shared weights, tanh, two-unit complex readout),
theta ~ N(0, 0.1^2) (seed 0), 16384 Metropolis chains started from uniform random
S_z = 0 configurations (seed 1).  Synthetic, seeded data.

One step = one pass of the whole hot path over one batch:
  Metropolis pair-exchange sweep of every chain (one recorded sample per chain)
  -> log Psi forward -> incremental local energy -> ISGO weights and statistics
  -> backward VJP -> SGD update, all through the library's C ABI on the device.
value = samples through the step per second (whole job, all ranks).

Also reported: the incremental local energy alone and the plain FP32 full
re-evaluation comparator (samples/s), their energy agreement, the ISGO step time, the
roofline of the dominant kernel, the CPU oracle baseline, and an end-to-end figure with
host buffers.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--prec bf16|fp32]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2011_12453_gb300 import workloads as W  # noqa: E402

METRIC = "local-energy samples/s and ISGO step time vs plain FP32 GPU form at ≤1e-4 rel. energy"
WORKLOAD = dict(workload="kagome_6x6x3_heisenberg", n_sites=108, n_bonds=216, L=4, F=32, chains=16384,
                sweeps_per_step=1, theta_seed=0, spin_seed=1)
L2_FLUSH_BYTES = 512 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--prec", default=os.environ.get("GNA_BENCH_PREC", "auto"))
    p.add_argument("--chains", type=int, default=WORKLOAD["chains"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--only", default=None, choices=["eloc", "eloc_full", "metropolis", "backward", "forward"],
                   help="time one call of the path alone (for profiling); prints a short JSON line")
    return p.parse_args()


# ---------------------------------------------------------------------------------
# distributed plumbing (replicas: every rank runs its own chains; no data-path collective)
# ---------------------------------------------------------------------------------

def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(backend):
    import torch.distributed as dist

    ws, rank, _ = dist_info()
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend, rank=rank, world_size=ws)
    return ws, rank


def barrier():
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 9:
                for k, n in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


# ---------------------------------------------------------------------------------
# algorithmic work of the incremental local energy (FLOPs per sample)
# ---------------------------------------------------------------------------------

def incremental_flops(g, F, L, ball, deg_of, spins_np):
    """Per sample: one forward (the layer cache) + for each antiparallel bond e,
    sum_{l=1..L} sum_{v in ball_l(e)} (4 F^2 + 2 deg(v) F)."""
    N = g.n_sites
    fwd = L * sum(4 * F * F + 2 * deg_of[v] * F for v in range(N))
    per_bond = np.array([sum(ball[e][l] for l in range(1, L + 1)) for e in range(g.n_edges)], dtype=np.float64)
    # regular lattices: every row has the same degree; use the exact per-bond row-degree sums otherwise
    deg_mean = float(np.mean(deg_of))
    per_bond_flops = per_bond * (4 * F * F + 2 * deg_mean * F)
    anti = spins_np[:, g.edges[:, 0]] != spins_np[:, g.edges[:, 1]]
    return fwd + (anti * per_bond_flops[None, :]).sum(axis=1)


def full_flops(g, F, L, deg_of, spins_np):
    N = g.n_sites
    fwd = L * sum(4 * F * F + 2 * deg_of[v] * F for v in range(N))
    anti = (spins_np[:, g.edges[:, 0]] != spins_np[:, g.edges[:, 1]]).sum(axis=1)
    return fwd * (1 + anti)


# ---------------------------------------------------------------------------------
# CPU oracle baseline (bounded sample, spawn pool, single-threaded BLAS per worker)
# ---------------------------------------------------------------------------------

def _oracle_worker(args):
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    os.environ["MKL_NUM_THREADS"] = "1"
    F, L, n_per, seed = args
    from oracle import gcn, isgo

    g = W.kagome(6)
    th = W.random_theta(F, L, 0)
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    s = W.random_spins(g.n_sites, n_per, seed)
    t = time.perf_counter()
    lp0 = gcn.logpsi_complex(th, F, L, Ah, s)
    isgo.isgo_gradient(th, F, L, Ah, g.edges, g.J, s, lp0)
    return n_per, time.perf_counter() - t


def cpu_oracle_rate(n_per_worker=6, workers=None):
    import multiprocessing as mp

    workers = workers or min(16, os.cpu_count() or 1)
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env_keep:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        t0 = time.perf_counter()
        with ctx.Pool(workers) as pool:
            res = pool.map(_oracle_worker, [(WORKLOAD["F"], WORKLOAD["L"], n_per_worker, 100 + w) for w in range(workers)])
        wall = time.perf_counter() - t0
    finally:
        for k, v in env_keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    n = sum(r[0] for r in res)
    busy = max(r[1] for r in res)
    return {"value": n / busy, "unit": "samples/s", "cores": workers, "kind": "oracle",
            "sample": f"{n} Kagome-108 configurations ({n_per_worker} per worker, {workers} spawn workers, "
                      f"1 BLAS thread each): FP64 forward + full-re-evaluation local energy + ISGO weights + "
                      f"backward; rate = configurations / slowest worker's busy time",
            "wall_s": wall}


# ---------------------------------------------------------------------------------
# reference arm: the oracle as it stands
# ---------------------------------------------------------------------------------

def run_reference(a):
    ws, rank, _ = dist_info()
    if ws > 1 and rank != 0:
        return 0
    per_step = []
    workers = min(16, os.cpu_count() or 1)
    for k in range(a.warmup + a.steps):
        r = cpu_oracle_rate(n_per_worker=2, workers=workers)
        if k >= a.warmup:
            per_step.append(r)
    n = sum(2 * workers for _ in per_step)
    t = sum(2 * workers / r["value"] for r in per_step)
    value = n / t
    line = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1000.0 * t / len(per_step), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": dict(WORKLOAD, l2="n/a (CPU)"),
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": workers, "kind": "oracle",
                             "sample": per_step[0]["sample"]},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------

def run_ours(a):
    import torch

    from paper_2011_12453_gb300 import build as B, gna

    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    init_dist("nccl" if ws > 1 else "gloo")
    B.build()
    dev = torch.device("cuda", local)
    g = W.kagome(6)
    F, L, C = WORKLOAD["F"], WORKLOAD["L"], a.chains
    prec_name = a.prec
    graph = gna.Graph.from_workload(g, L)
    if prec_name == "auto":
        prec_name = "bf16"
        try:
            gna.workspace_size(graph, gna.Model(F, L, gna.PREC_BF16), gna.OP_ELOC_INCR, C)
        except gna.GnaError:
            prec_name = "fp32"
    prec = {"bf16": gna.PREC_BF16, "fp32": gna.PREC_FP32}[prec_name]
    model = gna.Model(F, L, prec)
    model32 = gna.Model(F, L, gna.PREC_FP32)
    theta = torch.tensor(W.random_theta(F, L, 0), dtype=torch.float32, device=dev)
    chains = torch.tensor(W.random_spins(g.n_sites, C, 1 + 1000 * rank), device=dev)
    P = model.num_params
    lp = torch.empty((C, 2), dtype=torch.float64, device=dev)
    E = torch.empty((C, 2), dtype=torch.float64, device=dev)
    grad = torch.empty(P, dtype=torch.float64, device=dev)
    acc = torch.zeros(C, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    lr = 1e-3
    seed = 12345 + rank
    state = {"step": 0}
    n_sites = g.n_sites

    def step(ev=None):
        # ev: list of 7 events recorded between the phases
        t = state["step"]
        if ev:
            ev[0].record(stream)
        samples, lp0, _, _ = gna.metropolis_sweep(graph, model, theta, chains, 1, 1, seed, t * n_sites, n_accepted=acc)
        s = samples[0]
        if ev:
            ev[1].record(stream)
        gna.forward(graph, model, theta, s, out=lp)
        if ev:
            ev[2].record(stream)
        gna.local_energy(graph, model, theta, s, gna.ELOC_INCREMENTAL, out=E)
        if ev:
            ev[3].record(stream)
        cot, stats = gna.isgo_weights(lp, lp0[0], E)
        if ev:
            ev[4].record(stream)
        gna.backward(graph, model, theta, s, cot, out=grad)
        gna.sgd_update(model, theta, grad, lr)
        if ev:
            ev[5].record(stream)
        state["step"] += 1
        return s, stats

    # burn-in + warm-up
    for _ in range(max(a.warmup, 3)):
        step()
    torch.cuda.synchronize()

    K = a.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(K)]
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    for k in range(K):
        flush.zero_()  # L2 flush between timed steps (outside the events)
        s, stats = step(evs[k])
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ph = np.array([[evs[k][i].elapsed_time(evs[k][i + 1]) for i in range(5)] for k in range(K)])  # ms
    step_ms = ph.sum(axis=1)
    t_total = max_over_ranks(float(step_ms.sum()) / 1000.0, dev)
    value = ws * C * K / t_total
    last_s = s.clone()

    # energy agreement on the last step's samples: this path vs the plain FP32 full re-evaluation
    E_ours = gna.local_energy(graph, model, theta, last_s, gna.ELOC_INCREMENTAL).cpu().numpy()
    E_full = gna.local_energy(graph, model32, theta, last_s, gna.ELOC_FULL).cpu().numpy()
    rel = abs(E_ours[:, 0].mean() - E_full[:, 0].mean()) / abs(E_full[:, 0].mean())
    per_sample = np.abs(E_ours[:, 0] - E_full[:, 0]) / np.abs(E_full[:, 0]).clip(1e-12)

    # comparator timing: FP32 full re-evaluation vs this path's incremental, same samples
    def time_call(fn, reps=3):
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    t_full = time_call(lambda: gna.local_energy(graph, model32, theta, last_s, gna.ELOC_FULL, out=E), reps=2)
    t_incr = float(np.median(ph[:, 2]))

    # end to end through the public API with host buffers: pinned chains in, statistics out
    host_chains = chains.cpu().pin_memory()
    host_stats = torch.empty(4, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for k in range(max(2, min(K, 5))):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        chains.copy_(host_chains, non_blocking=True)
        _, st = step()
        host_stats.copy_(st, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_value = ws * C / (max_over_ranks(float(np.mean(e2e_ms)) / 1000.0, dev))

    # roofline of the dominant kernel (the incremental local energy)
    spins_np = last_s.cpu().numpy()
    deg = np.bincount(g.edges.ravel(), minlength=g.n_sites)
    ball = gna.ball_sizes_host(g.n_sites, g.edges, L)
    fl_incr = float(incremental_flops(g, F, L, ball, deg, spins_np).sum())
    fl_full = float(full_flops(g, F, L, deg, spins_np).sum())
    peaks, peak_kind = measured_peaks()
    if prec == gna.PREC_BF16:
        peak = peaks["bf16_tflops_sustained"]
        bound = "tensor"
    else:
        # FP32 FMA pipe: 152 SMs x 128 lanes x 2 flop x max SM clock
        peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        bound = "alu"
    achieved = fl_incr / (t_incr / 1000.0) / 1e12
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": "gna_local_energy incremental (k_eloc_incr)",
            "peak_source": peak_kind if bound == "tensor" else "derived: 152 SM x 128 FP32 lanes x 2 x sm_max_mhz",
            "flops_per_launch": fl_incr}

    cpu = None
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        cpu = cpu_oracle_rate()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": ws, "steps": K, "warmup": a.warmup,
            "ms_per_step": float(step_ms.mean()), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": prec_name, "data": "synthetic",
            "config": dict(WORKLOAD, chains=C, l2="flushed between timed steps (512 MiB write)",
                           parallelism=f"replicas{ws}"),
            "isgo_step_ms": float(ph[:, 1:].sum(axis=1).mean()),
            "phases_ms": {n: float(ph[:, i].mean()) for i, n in
                          enumerate(["metropolis_sweep", "forward", "local_energy", "isgo_weights",
                                     "backward_sgd"])},
            "comparator": {"eloc_incremental_samples_per_s": C / (t_incr / 1000.0),
                           "eloc_fp32_full_samples_per_s": C / (t_full / 1000.0),
                           "speedup": t_full / t_incr,
                           "energy_rel_diff_mean": float(rel),
                           "energy_rel_diff_per_sample_max": float(per_sample.max()),
                           "fp32_full_tflops": fl_full / (t_full / 1000.0) / 1e12},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "samples/s", "h2d_bytes_per_step": int(C * g.n_sites),
                    "d2h_bytes_per_step": 32},
            "gpu_launches": int(K * 10),
            "clocks": clk,
            "acceptance": float(acc.sum().item()) / max(1, (state["step"]) * C * g.n_sites),
        }
        print(json.dumps(line))
    return 0


def run_only(a):
    """One operation of the step alone, W + K launches on the same workload."""
    import torch

    from paper_2011_12453_gb300 import build as B, gna

    B.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    g = W.kagome(6)
    F, L, C = WORKLOAD["F"], WORKLOAD["L"], a.chains
    prec = {"bf16": gna.PREC_BF16, "fp32": gna.PREC_FP32, "auto": gna.PREC_BF16}[a.prec]
    graph = gna.Graph.from_workload(g, L)
    model = gna.Model(F, L, prec)
    model32 = gna.Model(F, L, gna.PREC_FP32)
    theta = torch.tensor(W.random_theta(F, L, 0), dtype=torch.float32, device=dev)
    spins = torch.tensor(W.random_spins(g.n_sites, C, 1), device=dev)
    cot = torch.randn(C, 2, dtype=torch.float64, device=dev)
    out = torch.empty((C, 2), dtype=torch.float64, device=dev)

    def call(k):
        if a.only == "eloc":
            gna.local_energy(graph, model, theta, spins, gna.ELOC_INCREMENTAL, out=out)
        elif a.only == "eloc_full":
            gna.local_energy(graph, model32, theta, spins, gna.ELOC_FULL, out=out)
        elif a.only == "forward":
            gna.forward(graph, model, theta, spins, out=out)
        elif a.only == "backward":
            gna.backward(graph, model, theta, spins, cot)
        else:
            gna.metropolis_sweep(graph, model, theta, spins, 1, 0, 7, k * g.n_sites)

    for k in range(a.warmup):
        call(k)
    torch.cuda.synchronize()
    ts = []
    for k in range(a.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call(a.warmup + k)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    print(json.dumps({"only": a.only, "prec": a.prec, "chains": C, "ms": ts, "median_ms": float(np.median(ts)),
                      "samples_per_s": C / (float(np.median(ts)) / 1000.0)}))
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    if a.only:
        return run_only(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
