"""Benchmark of the GNA-VMC hot path on one GB300 (or N replicas under torchrun).

Workload: Kagome 6x6x3 (108 sites, 216 bonds, periodic), Heisenberg J = 1, GCN with
L = 4 layers of width F = 32 (shared weights, tanh, two-unit complex readout),
theta ~ N(0, 0.1^2) (seed 0), 16384 Metropolis chains started from uniform random
S_z = 0 configurations (seed 1).  Synthetic, seeded data.

One step = one pass of the whole hot path over one batch:
  Metropolis pair-exchange sweep of every chain (one recorded sample per chain)
  -> incremental local energy and log Psi (one call: on the tensor cores the local-energy
  kernel's own forward gives log Psi) -> ISGO weights and statistics
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
# One step = one ISGO iteration: `recorded_sweeps` Metropolis sweeps of every chain (one
# sample per chain per sweep) reused for `reuse` updates, each update = incremental local
# energy with log Psi + ISGO weights + backward + SGD.  The default is the Kagome 108-site workload.
WORKLOADS = {
    "kagome108": dict(workload="kagome_6x6x3_heisenberg", lattice="kagome", size=6, n_sites=108, n_bonds=216, L=4,
                      F=32, chains=16384, recorded_sweeps=1, reuse=1, proposal="plain", theta_seed=0, spin_seed=1,
                      comparator_samples=16384),
    "triangular144": dict(workload="triangular_12x12_heisenberg", lattice="triangular", size=12, n_sites=144,
                          n_bonds=432, L=4, F=48, chains=16384, recorded_sweeps=4, reuse=10, proposal="plain",
                          theta_seed=0, spin_seed=2, comparator_samples=4096),
    "kagome432": dict(workload="kagome_12x12x3_heisenberg", lattice="kagome", size=12, n_sites=432, n_bonds=864, L=6,
                      F=64, chains=16384, recorded_sweeps=16, reuse=10, proposal="learned", theta_seed=0, spin_seed=1,
                      comparator_samples=1024),
}
WORKLOAD = WORKLOADS["kagome108"]
L2_FLUSH_BYTES = 512 << 20


def make_graph(wl):
    return W.kagome(wl["size"]) if wl["lattice"] == "kagome" else W.triangular(wl["size"], wl["size"])


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--prec", default=os.environ.get("GNA_BENCH_PREC", "auto"),
                   help="bf16x2 (default: split-operand tensor-core GEMMs, the path that meets the energy, "
                        "variance and gradient accuracy targets), bf16 or fp32")
    p.add_argument("--backward-prec", default="same", choices=["same", "fp32"],
                   help="arithmetic of the step's backward: that of --prec (default) or FP32, whose ISGO "
                        "gradient stays accurate at nearly flat wavefunctions")
    p.add_argument("--workload", default="kagome108", choices=sorted(WORKLOADS))
    p.add_argument("--chains", type=int, default=None, help="override the workload's chain count")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--extra", default="triangular144,kagome432",
                   help="comma-separated workloads also timed after the headline one (ISGO step, local-energy "
                        "samples/s, roofline, energy agreement), or 'none'")
    p.add_argument("--extra-reuse", type=int, default=2,
                   help="reuse updates timed for the Kagome 432 workload (its 10-update iteration is reported "
                        "as the timed sweeps + 10 x the mean timed update)")
    p.add_argument("--only", default=None, choices=["eloc", "eloc_logpsi", "eloc_full", "metropolis", "backward", "forward"],
                   help="time one call of the path alone (for profiling); prints a short JSON line")
    a = p.parse_args()
    a.wl = dict(WORKLOADS[a.workload])
    if a.chains is not None:
        a.wl["chains"] = a.chains
    return a


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
    wl, n_per, seed = args
    from oracle import gcn, isgo

    g = make_graph(wl)
    F, L = wl["F"], wl["L"]
    th = W.random_theta(F, L, wl["theta_seed"])
    Ah = gcn.norm_adjacency(gcn.adjacency(g.n_sites, g.edges))
    s = W.random_spins(g.n_sites, n_per, seed)
    t = time.perf_counter()
    lp0 = gcn.logpsi_complex(th, F, L, Ah, s)
    isgo.isgo_gradient(th, F, L, Ah, g.edges, g.J, s, lp0)
    return n_per, time.perf_counter() - t


def cpu_oracle_rate(wl, n_per_worker=6, workers=None):
    """The FP64 oracle's forward + full-re-evaluation local energy + ISGO weights + backward
    on a bounded sample of the workload's configurations, one process per core."""
    import multiprocessing as mp

    workers = workers or min(16, os.cpu_count() or 1)
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env_keep:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        t0 = time.perf_counter()
        with ctx.Pool(workers) as pool:
            res = pool.map(_oracle_worker, [(wl, n_per_worker, 100 + w) for w in range(workers)])
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
            "sample": f"{n} {wl['workload']} configurations ({n_per_worker} per worker, {workers} spawn workers, "
                      f"1 BLAS thread each): FP64 forward + full-re-evaluation local energy + ISGO weights + "
                      f"backward; rate = configurations / slowest worker's busy time",
            "wall_s": wall}


def oracle_sample_size(wl):
    """Configurations per worker for about 10-30 s of oracle work."""
    return {"kagome108": 6, "triangular144": 2, "kagome432": 1}.get(wl.get("key", ""), 2)


# ---------------------------------------------------------------------------------
# reference arm: the oracle as it stands
# ---------------------------------------------------------------------------------

def run_reference(a):
    ws, rank, _ = dist_info()
    if ws > 1 and rank != 0:
        return 0
    wl = dict(a.wl, key=a.workload)
    per_step = []
    workers = min(16, os.cpu_count() or 1)
    n_per = 2 if a.workload == "kagome108" else 1
    for k in range(a.warmup + a.steps):
        r = cpu_oracle_rate(wl, n_per_worker=n_per, workers=workers)
        if k >= a.warmup:
            per_step.append(r)
    n = sum(n_per * workers for _ in per_step)
    t = sum(n_per * workers / r["value"] for r in per_step)
    value = n / t
    cfg = {k: v for k, v in a.wl.items() if k != "comparator_samples"}
    line = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1000.0 * t / len(per_step), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": dict(cfg, l2="n/a (CPU)"),
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": workers, "kind": "oracle",
                             "sample": per_step[0]["sample"]},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------

# DRAM bytes per sample of the dominant kernels from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum of one launch / the samples it processed), valid only for the source file
# that was profiled: keyed by (workload, kernel) with the SHA-256 of that source (carried
# forward only across changes to other kernels of the file).
PROFILED_TRAFFIC = {
    # ncu --set full of gna_local_energy_logpsi, 2048 configurations, one launch: 3,085,824 B read
    # + 1,172,992 B written
    ("kagome_6x6x3_heisenberg", "k_tc<1>"): {"bytes_per_unit": (3085824 + 1172992) / 2048,
                                             "sha256": "4f986c229ef99251b5f5cf6d28437d630522986576258425c1c822240624057c"},
    # the same for BF16 operands: 3,069,952 B read + 1,056,768 B written
    ("kagome_6x6x3_heisenberg", "k_tc<0>"): {"bytes_per_unit": (3069952 + 1056768) / 2048,
                                             "sha256": "4f986c229ef99251b5f5cf6d28437d630522986576258425c1c822240624057c"},
    # ncu --set full, 2048 chains, one sweep: 481,241,600 B read + 1,433,287,424 B written (the
    # sampler's code is unchanged since; the file changed in the local-energy kernel only)
    ("kagome_6x6x3_heisenberg", "k_tc_metro"): {"bytes_per_unit": (481241600 + 1433287424) / 2048,
                                                "sha256": "4f986c229ef99251b5f5cf6d28437d630522986576258425c1c822240624057c"},
}


def _source_sha(rel):
    import hashlib

    with open(os.path.join(ROOT, "paper_2011_12453_gb300", "csrc", rel), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def profiled_traffic(workload, kernel, source, units):
    rec = PROFILED_TRAFFIC.get((workload, kernel))
    if rec is None or rec["sha256"] != _source_sha(source):
        return None
    return rec["bytes_per_unit"] * units


def sweep_flops(g, F, L, ball, deg_of, spins_np, steps_per_chain):
    """Expected algorithmic FLOPs of `steps_per_chain` plain exchange proposals per chain: the
    bond is uniform over the edges, an antiparallel bond costs
    sum_{l=1..L} |ball_l(e)| (4F^2 + 2 deg F) (the difference propagation), a parallel one
    nothing; the antiparallel set is taken from the chains' recorded states (stationary
    chains), plus one forward per chain for the launch's layer cache."""
    N = g.n_sites
    fwd = L * sum(4 * F * F + 2 * deg_of[v] * F for v in range(N))
    deg_mean = float(np.mean(deg_of))
    per_bond = np.array([sum(ball[e][l] for l in range(1, L + 1)) for e in range(g.n_edges)], dtype=np.float64)
    per_bond *= 4 * F * F + 2 * deg_mean * F
    anti = spins_np[:, g.edges[:, 0]] != spins_np[:, g.edges[:, 1]]
    per_step = (anti * per_bond[None, :]).sum(axis=1) / g.n_edges
    return float((fwd + steps_per_chain * per_step).sum())

PRECS = {"bf16": 2, "bf16x2": 3, "fp32": 1}


def measure_workload(key, prec_name, dev, flush, K_timed, peaks, peak_kind):
    """One ISGO iteration of another workload, timed with CUDA events on the current stream:
    the recorded sweeps of all chains (plain moves on the tensor-core sampler), then
    min(K, K_timed) reuse updates over all S x C samples (incremental local energy with log Psi,
    ISGO weights, backward + SGD; L2 flushed before each).  Reports the mean update (the ISGO
    step), the iteration (sweeps + K updates; extrapolated from the timed updates when
    K_timed < K), local-energy samples/s with the roofline of k_tc, and the energy agreement
    with the plain FP32 full re-evaluation on a subset of the samples."""
    import torch

    from paper_2011_12453_gb300 import gna

    wl = dict(WORKLOADS[key])
    g = make_graph(wl)
    F, L, C = wl["F"], wl["L"], wl["chains"]
    S, K = wl["recorded_sweeps"], wl["reuse"]
    N = g.n_sites
    Bn = S * C
    graph = gna.Graph.from_workload(g, L)
    model = gna.Model(F, L, PRECS[prec_name])
    model32 = gna.Model(F, L, gna.PREC_FP32)
    theta = torch.tensor(W.random_theta(F, L, wl["theta_seed"]), dtype=torch.float32, device=dev)
    chains = torch.tensor(W.random_spins(N, C, wl["spin_seed"]), device=dev)
    lp0 = torch.empty((Bn, 2), dtype=torch.float64, device=dev)
    lp = torch.empty((Bn, 2), dtype=torch.float64, device=dev)
    E = torch.empty((Bn, 2), dtype=torch.float64, device=dev)
    grad = torch.empty(model.num_params, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def ev():
        return torch.cuda.Event(enable_timing=True)

    # warm-up (untimed): one sweep of every chain, one update on a slice with a copy of theta
    gna.metropolis_sweep(graph, model, theta, chains, 1, 0, 777, 0)
    sl = chains[:min(C, 1024)].contiguous()
    th_w = theta.clone()
    l_w = gna.forward(graph, model, th_w, sl)
    E_w = gna.local_energy(graph, model, th_w, sl, gna.ELOC_INCREMENTAL)
    c_w, _ = gna.isgo_weights(l_w, l_w, E_w)
    gna.sgd_update(model, th_w, gna.backward(graph, model, th_w, sl, c_w), 1e-3)
    torch.cuda.synchronize()
    flush.zero_()
    e0, e1 = ev(), ev()
    e0.record(stream)
    samples, _, _, _ = gna.metropolis_sweep(graph, model, theta, chains, S, 1, 12345, N, record_logpsi=False)
    e1.record(stream)
    torch.cuda.synchronize()
    t_sweeps = e0.elapsed_time(e1)
    s = samples.view(Bn, N)
    kt = min(K, K_timed)
    ph = np.zeros((kt, 3))
    for k in range(kt):
        flush.zero_()
        ms = [ev() for _ in range(4)]
        cur = lp0 if k == 0 else lp
        ms[0].record(stream)
        gna.local_energy_logpsi(graph, model, theta, s, out=E, out_logpsi=cur)
        ms[1].record(stream)
        cot, stats = gna.isgo_weights(cur, lp0, E)
        ms[2].record(stream)
        gna.backward(graph, model, theta, s, cot, out=grad)
        gna.sgd_update(model, theta, grad, 1e-4)
        ms[3].record(stream)
        torch.cuda.synchronize()
        ph[k] = [ms[i].elapsed_time(ms[i + 1]) for i in range(3)]
    upd = float(ph.sum(axis=1).mean())
    t_eloc = float(ph[:, 0].mean())  # the local energy with its forward's log Psi
    spins_np = s.cpu().numpy()
    deg = np.bincount(g.edges.ravel(), minlength=N)
    ball = gna.ball_sizes_host(N, g.edges, L)
    fl = float(incremental_flops(g, F, L, ball, deg, spins_np).sum())
    achieved = fl / (t_eloc / 1000.0) / 1e12
    nc = min(Bn, wl["comparator_samples"])
    sub = s[:nc].contiguous()
    E_ours = E[:nc].cpu().numpy()
    E_full = gna.local_energy(graph, model32, theta, sub, gna.ELOC_FULL).cpu().numpy()
    rel = abs(E_ours[:, 0].mean() - E_full[:, 0].mean()) / abs(E_full[:, 0].mean())
    per_sample = np.abs(E_ours[:, 0] - E_full[:, 0]) / np.abs(E_full[:, 0]).clip(1e-12)
    return {"workload": wl["workload"], "dtype": prec_name, "n_sites": N, "L": L, "F": F, "chains": C,
            "recorded_sweeps": S, "samples": Bn, "reuse": K, "reuse_timed": kt, "proposal": "plain",
            "sweeps_ms": t_sweeps, "isgo_step_ms": upd,
            "isgo_iteration_ms": t_sweeps + K * upd, "isgo_iteration_extrapolated": kt < K,
            "phases_ms_per_update": {"local_energy_logpsi": t_eloc, "isgo_weights": float(ph[:, 1].mean()),
                                     "backward_sgd": float(ph[:, 2].mean())},
            "eloc_samples_per_s": Bn / (t_eloc / 1000.0),
            "sample_updates_per_s": Bn / (upd / 1000.0),
            "roofline": {"bound": "tensor", "kernel": "k_tc (gna_local_energy_logpsi, %s)" % prec_name,
                         "achieved": achieved, "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s",
                         "frac": achieved / peaks["bf16_tflops_sustained"],
                         "peak_source": peak_kind + " bf16_tflops_sustained", "flops_per_launch": fl,
                         "traffic": None},
            "energy_vs_fp32_full": {"samples": nc, "rel_diff_mean": float(rel),
                                    "rel_diff_per_sample_max": float(per_sample.max())}}


def run_ours(a):
    import torch

    from paper_2011_12453_gb300 import build as B, gna, vmc

    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    init_dist("nccl" if ws > 1 else "gloo")
    B.build()
    dev = torch.device("cuda", local)
    wl = a.wl
    g = make_graph(wl)
    F, L, C = wl["F"], wl["L"], wl["chains"]
    S, K = wl["recorded_sweeps"], wl["reuse"]
    N = g.n_sites
    Bn = S * C
    prec_name = a.prec
    graph = gna.Graph.from_workload(g, L)
    if prec_name == "auto":
        prec_name = "bf16x2"
        try:
            gna.workspace_size(graph, gna.Model(F, L, gna.PREC_BF16X2), gna.OP_ELOC_INCR, Bn)
        except gna.GnaError:
            prec_name = "fp32"
    prec = {"bf16": gna.PREC_BF16, "bf16x2": gna.PREC_BF16X2, "fp32": gna.PREC_FP32}[prec_name]
    model = gna.Model(F, L, prec)
    model32 = gna.Model(F, L, gna.PREC_FP32)
    model_bwd = model32 if a.backward_prec == "fp32" else model
    theta = torch.tensor(W.random_theta(F, L, wl["theta_seed"]), dtype=torch.float32, device=dev)
    chains = torch.tensor(W.random_spins(N, C, wl["spin_seed"] + 1000 * rank), device=dev)
    P = model.num_params
    lp = torch.empty((Bn, 2), dtype=torch.float64, device=dev)
    lp0 = torch.empty((Bn, 2), dtype=torch.float64, device=dev)
    E = torch.empty((Bn, 2), dtype=torch.float64, device=dev)
    grad = torch.empty(P, dtype=torch.float64, device=dev)
    acc = torch.zeros(C, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    lr = 1e-3
    seed = 12345 + rank
    state = {"step": 0}
    prop = None
    if wl["proposal"] == "learned":
        prop = torch.tensor(W.random_proposal_params(1, 0.3), dtype=torch.float32, device=dev)

    def step(marks=None):
        def mark(name):
            if marks is not None:
                e = torch.cuda.Event(enable_timing=True)
                e.record(stream)
                marks.append((name, e))

        mark("start")
        samples, _, _, _ = gna.metropolis_sweep(graph, model, theta, chains, S, 1, seed, state["step"] * S * N,
                                                n_accepted=acc, proposal=prop, eps=0.1, record_logpsi=False)
        s = samples.view(Bn, N)
        mark("metropolis_sweep")
        stats = None
        for k in range(K):
            # log Psi^0: the first update's log Psi at the sampling parameters (weights exactly 1)
            cur = lp0 if k == 0 else lp
            gna.local_energy_logpsi(graph, model, theta, s, out=E, out_logpsi=cur)
            mark("local_energy_logpsi")
            cot, stats = gna.isgo_weights(cur, lp0, E)
            mark("isgo_weights")
            gna.backward(graph, model_bwd, theta, s, cot, out=grad)
            gna.sgd_update(model, theta, grad, lr)
            mark("backward_sgd")
        state["step"] += 1
        return s, stats

    # burn-in + warm-up (the learned proposal is trained on the burnt-in chains first)
    if prop is not None:
        gna.metropolis_sweep(graph, model, theta, chains, 2, 0, seed + 7, 0, records=False)
        vmc.train_proposal(graph, model, theta, chains, prop, 50, 3e-3)
    for _ in range(max(a.warmup, 3)):
        step()
    torch.cuda.synchronize()

    Ksteps = a.steps
    marks = [[] for _ in range(Ksteps)]
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    for k in range(Ksteps):
        flush.zero_()  # L2 flush between timed steps (outside the events)
        s, stats = step(marks[k])
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    names = ["metropolis_sweep", "local_energy_logpsi", "isgo_weights", "backward_sgd"]
    ph = np.zeros((Ksteps, len(names)))  # ms per step, summed over the reuse updates
    for k in range(Ksteps):
        for (_, e0), (nm, e1) in zip(marks[k][:-1], marks[k][1:]):
            ph[k, names.index(nm)] += e0.elapsed_time(e1)
    step_ms = ph.sum(axis=1)
    t_total = max_over_ranks(float(step_ms.sum()) / 1000.0, dev)
    value = ws * Bn * K * Ksteps / t_total
    last_s = s.clone()

    # energy agreement and comparator timing on a bounded subset of the last step's samples:
    # this path's incremental local energy vs the plain FP32 full re-evaluation
    nc = min(Bn, wl["comparator_samples"])
    sub = last_s[:nc].contiguous()
    E_ours = gna.local_energy(graph, model, theta, sub, gna.ELOC_INCREMENTAL).cpu().numpy()
    E_full = gna.local_energy(graph, model32, theta, sub, gna.ELOC_FULL).cpu().numpy()
    rel = abs(E_ours[:, 0].mean() - E_full[:, 0].mean()) / abs(E_full[:, 0].mean())
    per_sample = np.abs(E_ours[:, 0] - E_full[:, 0]) / np.abs(E_full[:, 0]).clip(1e-12)
    Esub = torch.empty((nc, 2), dtype=torch.float64, device=dev)

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

    t_full = time_call(lambda: gna.local_energy(graph, model32, theta, sub, gna.ELOC_FULL, out=Esub), reps=2)
    t_incr_sub = time_call(lambda: gna.local_energy(graph, model, theta, sub, gna.ELOC_INCREMENTAL, out=Esub))
    t_incr = float(np.median(ph[:, 1])) / K  # one local-energy launch (with its forward) over all Bn samples

    # end to end through the public API with host buffers: pinned chains in, statistics out
    host_chains = chains.cpu().pin_memory()
    host_stats = torch.empty(4, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for k in range(max(2, min(Ksteps, 5)) if K == 1 else 1):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        chains.copy_(host_chains, non_blocking=True)
        _, st = step()
        host_stats.copy_(st, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_value = ws * Bn * K / (max_over_ranks(float(np.mean(e2e_ms)) / 1000.0, dev))

    # roofline of the dominant kernel of the step (the sampler or the incremental local energy)
    spins_np = last_s.cpu().numpy()
    deg = np.bincount(g.edges.ravel(), minlength=N)
    ball = gna.ball_sizes_host(N, g.edges, L)
    fl_incr = float(incremental_flops(g, F, L, ball, deg, spins_np).sum())
    fl_full_sub = float(full_flops(g, F, L, deg, spins_np[:nc]).sum())
    fl_sweep = sweep_flops(g, F, L, ball, deg, spins_np[(S - 1) * C:], S * N)
    peaks, peak_kind = measured_peaks()
    alu_peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    t_sweep = float(np.median(ph[:, 0]))
    if t_sweep >= K * t_incr:
        if prec in (gna.PREC_BF16, gna.PREC_BF16X2) and prop is None:
            roof = {"bound": "tensor", "achieved": fl_sweep / (t_sweep / 1000.0) / 1e12,
                    "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s",
                    "kernel": "k_tc_metro (gna_metropolis_sweep, %d sweeps, BF16 tcgen05)" % S,
                    "peak_source": peak_kind + " bf16_tflops_sustained", "flops_per_launch": fl_sweep,
                    "traffic": profiled_traffic(wl["workload"], "k_tc_metro", "tc.cu", C * S)}
        else:
            roof = {"bound": "alu", "achieved": fl_sweep / (t_sweep / 1000.0) / 1e12, "peak": alu_peak,
                    "unit": "TFLOP/s", "kernel": "k_metro_warp (gna_metropolis_sweep, %d sweeps)" % S,
                    "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x sm_max_mhz (FP32 difference propagation)",
                    "flops_per_launch": fl_sweep, "traffic": None}
    elif prec in (gna.PREC_BF16, gna.PREC_BF16X2):
        roof = {"bound": "tensor", "achieved": fl_incr / (t_incr / 1000.0) / 1e12,
                "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s",
                "kernel": ("k_tc<1> (gna_local_energy_logpsi, split BF16 operands, tcgen05)"
                           if prec == gna.PREC_BF16X2 else "k_tc<0> (gna_local_energy_logpsi, BF16 tcgen05)"),
                "peak_source": peak_kind + " bf16_tflops_sustained", "flops_per_launch": fl_incr,
                "traffic": profiled_traffic(wl["workload"], "k_tc<1>" if prec == gna.PREC_BF16X2 else "k_tc<0>",
                                            "tc.cu", Bn)}
    else:
        roof = {"bound": "alu", "achieved": fl_incr / (t_incr / 1000.0) / 1e12, "peak": alu_peak,
                "unit": "TFLOP/s", "kernel": "k_eloc_incr (gna_local_energy incremental, FP32)",
                "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x sm_max_mhz", "flops_per_launch": fl_incr,
                "traffic": None}
    roof["frac"] = roof["achieved"] / roof["peak"]
    other = {"local_energy_tflops": fl_incr / (t_incr / 1000.0) / 1e12,
             "sweep_tflops": fl_sweep / (t_sweep / 1000.0) / 1e12}

    # the single-BF16 (fast) local energy on the same samples: time, roofline, energy agreement
    fast = None
    if prec == gna.PREC_BF16X2:
        model16 = gna.Model(F, L, gna.PREC_BF16)
        t16 = time_call(lambda: gna.local_energy(graph, model16, theta, sub, gna.ELOC_INCREMENTAL, out=Esub))
        E16 = gna.local_energy(graph, model16, theta, sub, gna.ELOC_INCREMENTAL).cpu().numpy()
        fl_sub = float(incremental_flops(g, F, L, ball, deg, spins_np[:nc]).sum())
        fast = {"dtype": "bf16", "eloc_samples_per_s": nc / (t16 / 1000.0),
                "tflops": fl_sub / (t16 / 1000.0) / 1e12,
                "frac": fl_sub / (t16 / 1000.0) / 1e12 / peaks["bf16_tflops_sustained"],
                "energy_rel_diff_mean_vs_fp32_full": float(abs(E16[:, 0].mean() - E_full[:, 0].mean()) /
                                                           abs(E_full[:, 0].mean())),
                "energy_rel_diff_per_sample_max_vs_fp32_full": float((np.abs(E16[:, 0] - E_full[:, 0]) /
                                                                      np.abs(E_full[:, 0]).clip(1e-12)).max())}
    extras = {}
    if rank == 0 and a.extra != "none":
        for key in [k for k in a.extra.split(",") if k and k != a.workload]:
            extras[key] = measure_workload(key, prec_name, dev, flush, 10 if key != "kagome432" else a.extra_reuse,
                                           peaks, peak_kind)

    cpu = None
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        cpu = cpu_oracle_rate(dict(wl, key=a.workload), n_per_worker=oracle_sample_size(dict(wl, key=a.workload)))
    if rank == 0:
        cfg = {k: v for k, v in wl.items() if k != "comparator_samples"}
        line = {
            "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": ws, "steps": Ksteps,
            "warmup": a.warmup, "ms_per_step": float(step_ms.mean()), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": prec_name, "data": "synthetic",
            "config": dict(cfg, samples_per_step=Bn, l2="flushed between timed steps (512 MiB write)",
                           parallelism=f"replicas{ws}",
                           backward=prec_name if a.backward_prec == "same" else a.backward_prec),
            "isgo_step_ms": float(ph[:, 1:].sum(axis=1).mean()) / K,
            "phases_ms": {n: float(ph[:, i].mean()) for i, n in enumerate(names)},
            "comparator": {"samples": nc,
                           "eloc_incremental_samples_per_s": nc / (t_incr_sub / 1000.0),
                           "eloc_fp32_full_samples_per_s": nc / (t_full / 1000.0),
                           "speedup": t_full / t_incr_sub,
                           "energy_rel_diff_mean": float(rel),
                           "energy_rel_diff_per_sample_max": float(per_sample.max()),
                           "fp32_full_tflops": fl_full_sub / (t_full / 1000.0) / 1e12},
            "roofline": roof,
            "other_kernels": other,
            "bf16_fast_local_energy": fast,
            "extra_workloads": extras,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "samples/s", "h2d_bytes_per_step": int(C * N),
                    "d2h_bytes_per_step": 32},
            # per step: the sweep, then per update the local energy with log Psi (one launch on the
            # tensor cores, forward + local energy otherwise), 4 weight kernels, backward + its
            # reduction, SGD
            "gpu_launches": int(Ksteps * (1 + (8 if prec in (gna.PREC_BF16, gna.PREC_BF16X2) else 9) * K)),
            "clocks": clk,
            "acceptance": float(acc.sum().item()) / max(1, state["step"] * S * C * N),
        }
        print(json.dumps(line))
    return 0


def run_only(a):
    """One operation of the step alone, W + K launches on the workload's chains."""
    import torch

    from paper_2011_12453_gb300 import build as B, gna

    B.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    wl = a.wl
    g = make_graph(wl)
    F, L, C = wl["F"], wl["L"], wl["chains"]
    prec = {"bf16": gna.PREC_BF16, "bf16x2": gna.PREC_BF16X2, "fp32": gna.PREC_FP32, "auto": gna.PREC_BF16}[a.prec]
    graph = gna.Graph.from_workload(g, L)
    model = gna.Model(F, L, prec)
    model32 = gna.Model(F, L, gna.PREC_FP32)
    theta = torch.tensor(W.random_theta(F, L, wl["theta_seed"]), dtype=torch.float32, device=dev)
    spins = torch.tensor(W.random_spins(g.n_sites, C, wl["spin_seed"]), device=dev)
    cot = torch.randn(C, 2, dtype=torch.float64, device=dev)
    out = torch.empty((C, 2), dtype=torch.float64, device=dev)
    lp_out = torch.empty((C, 2), dtype=torch.float64, device=dev)

    def call(k):
        if a.only == "eloc":
            gna.local_energy(graph, model, theta, spins, gna.ELOC_INCREMENTAL, out=out)
        elif a.only == "eloc_logpsi":
            gna.local_energy_logpsi(graph, model, theta, spins, out=out, out_logpsi=lp_out)
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
    print(json.dumps({"only": a.only, "workload": wl["workload"], "prec": a.prec, "chains": C, "ms": ts,
                      "median_ms": float(np.median(ts)), "samples_per_s": C / (float(np.median(ts)) / 1000.0)}))
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
