"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module holds no arithmetic of the method: it only builds the inputs that the
method consumes -- lattice edge lists with couplings, random parameter vectors and
random spin configurations -- from explicit seeds.  Nothing here imports the CUDA
binding or the oracle, so both sides can use it without touching each other.

Geometries follow the Numerical Experiments section of arXiv:2011.12453: Kagome
L x L x 3 and triangular lattices with periodic boundaries on both primitive
directions (a torus), and randomly connected graphs.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Graph:
    """An undirected simple graph with per-bond Heisenberg couplings."""

    n_sites: int
    edges: np.ndarray  # int32 [E][2], i < j not required, no duplicates, no self-loops
    J: np.ndarray  # float64 [E]
    name: str = ""
    seed: int | None = None  # final seed for random graphs (after resampling)

    @property
    def n_edges(self) -> int:
        return int(self.edges.shape[0])


def _check_simple(n: int, edges: np.ndarray) -> None:
    seen = set()
    for a, b in edges.tolist():
        if a == b:
            raise ValueError(f"self-loop at {a}")
        if not (0 <= a < n and 0 <= b < n):
            raise ValueError(f"edge ({a},{b}) out of range for n={n}")
        key = (min(a, b), max(a, b))
        if key in seen:
            raise ValueError(f"duplicate edge {key}")
        seen.add(key)


def kagome(Lx: int, Ly: int | None = None, J: float = 1.0) -> Graph:
    """Kagome lattice Lx x Ly x 3 on a torus.

    Cell (x, y) holds sites 0, 1, 2 with index 3*(x*Ly + y) + s.  Up triangle: the
    three in-cell bonds (0,1), (0,2), (1,2).  Down triangle: (x,y,1)-(x+1,y,0),
    (x,y,1)-(x+1,y-1,2) and (x+1,y,0)-(x+1,y-1,2), coordinates taken mod L.
    Every site has coordination 4 and there are 2N bonds.
    """
    Ly = Lx if Ly is None else Ly
    if Lx < 2 or Ly < 2:
        raise ValueError("Kagome torus needs Lx, Ly >= 2 to stay a simple graph")

    def idx(x: int, y: int, s: int) -> int:
        return 3 * ((x % Lx) * Ly + (y % Ly)) + s

    edges = []
    for x in range(Lx):
        for y in range(Ly):
            edges += [(idx(x, y, 0), idx(x, y, 1)), (idx(x, y, 0), idx(x, y, 2)),
                      (idx(x, y, 1), idx(x, y, 2))]
            edges += [(idx(x, y, 1), idx(x + 1, y, 0)), (idx(x, y, 1), idx(x + 1, y - 1, 2)),
                      (idx(x + 1, y, 0), idx(x + 1, y - 1, 2))]
    e = np.asarray(edges, dtype=np.int32)
    n = 3 * Lx * Ly
    _check_simple(n, e)
    return Graph(n, e, np.full(len(e), J, dtype=np.float64), f"kagome_{Lx}x{Ly}x3")


def triangular(Lx: int, Ly: int, J: float = 1.0) -> Graph:
    """Triangular lattice Lx x Ly on a torus: bonds along (1,0), (0,1) and (1,-1)."""
    if Lx < 3 or Ly < 3:
        raise ValueError("triangular torus needs Lx, Ly >= 3 to stay a simple graph")

    def idx(x: int, y: int) -> int:
        return (x % Lx) * Ly + (y % Ly)

    edges = []
    for x in range(Lx):
        for y in range(Ly):
            edges += [(idx(x, y), idx(x + 1, y)), (idx(x, y), idx(x, y + 1)),
                      (idx(x, y), idx(x + 1, y - 1))]
    e = np.asarray(edges, dtype=np.int32)
    _check_simple(Lx * Ly, e)
    return Graph(Lx * Ly, e, np.full(len(e), J, dtype=np.float64), f"triangular_{Lx}x{Ly}")


def _connected(n: int, edges: np.ndarray) -> bool:
    adj = [[] for _ in range(n)]
    for a, b in edges.tolist():
        adj[a].append(b)
        adj[b].append(a)
    seen = {0}
    stack = [0]
    while stack:
        v = stack.pop()
        for u in adj[v]:
            if u not in seen:
                seen.add(u)
                stack.append(u)
    return len(seen) == n


def erdos_renyi(n: int, p: float, seed: int, J_range: tuple[float, float] | None = None,
                max_tries: int = 1000) -> Graph:
    """Random graph G(n, p), resampled with seed+1, seed+2, ... until connected.

    J is 1 on every bond, or uniform in J_range when given (drawn from the same seed).
    """
    for t in range(max_tries):
        s = seed + t
        rng = np.random.default_rng(s)
        iu, ju = np.triu_indices(n, 1)
        keep = rng.random(iu.shape[0]) < p
        e = np.stack([iu[keep], ju[keep]], axis=1).astype(np.int32)
        if e.shape[0] == 0 or not _connected(n, e):
            continue
        if J_range is None:
            J = np.ones(e.shape[0])
        else:
            J = rng.uniform(J_range[0], J_range[1], e.shape[0])
        return Graph(n, e, J.astype(np.float64), f"er_{n}_p{p:.3f}", seed=s)
    raise RuntimeError("no connected sample found")


def random_graph_set(count: int = 32, seed: int = 1000, n_range: tuple[int, int] = (32, 96),
                     mean_degree: float = 4.0) -> list[Graph]:
    """`count` Erdos-Renyi graphs: sizes uniform in n_range (inclusive, drawn from `seed`),
    edge probability mean_degree/(n - 1), couplings J uniform in [0.5, 1.5]; graph g is
    erdos_renyi with seed `seed` + 1000 * (g + 1) (resampled until connected)."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(n_range[0], n_range[1] + 1, size=count)
    return [erdos_renyi(int(n), mean_degree / (int(n) - 1), seed + 1000 * (g + 1), J_range=(0.5, 1.5))
            for g, n in enumerate(sizes)]


def two_site() -> Graph:
    """Two sites joined by one bond (the singlet/triplet test system)."""
    return Graph(2, np.array([[0, 1]], dtype=np.int32), np.ones(1), "two_site")


def ring(n: int, J: float = 1.0) -> Graph:
    e = np.array([(i, (i + 1) % n) for i in range(n)], dtype=np.int32)
    _check_simple(n, e)
    return Graph(n, e, np.full(n, J), f"ring_{n}")


def complete(n: int, J: float = 1.0) -> Graph:
    iu, ju = np.triu_indices(n, 1)
    e = np.stack([iu, ju], axis=1).astype(np.int32)
    return Graph(n, e, np.full(e.shape[0], J), f"complete_{n}")


def complete_bipartite(a: int, b: int, J: float = 1.0) -> Graph:
    e = np.array([(i, a + k) for i in range(a) for k in range(b)], dtype=np.int32)
    return Graph(a + b, e, np.full(e.shape[0], J), f"K{a},{b}")


def num_params(F: int, L: int, shared: bool = True) -> int:
    """Length of the flat parameter vector (embedding, GCN layer(s), two-unit readout)."""
    n_layers = 1 if shared else L
    return 2 * F + F + n_layers * (2 * F * F + F) + (F + 2) * 2 + 2


def random_theta(F: int, L: int, seed: int, scale: float = 0.1, shared: bool = True) -> np.ndarray:
    """theta ~ N(0, scale^2), float64."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, num_params(F, L, shared)).astype(np.float64)


def random_spins(n_sites: int, batch: int, seed: int, n_up: int | None = None) -> np.ndarray:
    """int8 [batch][n_sites] of +-1 with exactly n_up up spins per row (default floor(N/2))."""
    n_up = n_sites // 2 if n_up is None else n_up
    rng = np.random.default_rng(seed)
    base = np.concatenate([np.ones(n_up, np.int8), -np.ones(n_sites - n_up, np.int8)])
    out = np.tile(base, (batch, 1))
    return rng.permuted(out, axis=1).astype(np.int8)


def all_sector_states(n_sites: int, n_up: int | None = None) -> np.ndarray:
    """Every configuration with n_up up spins, int8 [M][n_sites], in increasing bit order.

    Bit v of the integer code is 1 when site v is up.  Used to enumerate small systems.
    """
    n_up = n_sites // 2 if n_up is None else n_up
    codes = [c for c in range(1 << n_sites) if bin(c).count("1") == n_up]
    out = np.empty((len(codes), n_sites), dtype=np.int8)
    for k, c in enumerate(codes):
        for v in range(n_sites):
            out[k, v] = 1 if (c >> v) & 1 else -1
    return out


PROPOSAL_D_IN, PROPOSAL_HIDDEN = 9, 64


def proposal_num_params() -> int:
    """Length of the learned-proposal network's flat parameter vector (9 -> 64 -> 64 -> 1)."""
    d, h = PROPOSAL_D_IN, PROPOSAL_HIDDEN
    return d * h + h + h * h + h + h + 1


def random_proposal_params(seed: int, scale: float = 0.3) -> np.ndarray:
    """Random initial parameters [W1, b1, W2, b2, w3, b3] of the proposal network (float64)."""
    d, h = PROPOSAL_D_IN, PROPOSAL_HIDDEN
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, scale, (d, h))
    W2 = rng.normal(0, 3 * scale / np.sqrt(h), (h, h))
    w3 = rng.normal(0, 3 * scale / np.sqrt(h), h)
    return np.concatenate([W1.ravel(), np.zeros(h), W2.ravel(), np.zeros(h), w3, np.zeros(1)])
