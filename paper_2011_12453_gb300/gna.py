"""Thin ctypes binding over libgna.so (include/gna.h): argument marshalling only.

Every compute step runs in the library's CUDA kernels; PyTorch supplies device memory
and the current stream.  The binding raises GnaError when the library is missing or a
call returns an error status -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libgna.so")

GNA_OK = 0
GNA_ERR_INVALID_ARG = -1
GNA_ERR_CUDA = -2
GNA_ERR_TIMEOUT = -3
GNA_ERR_NONFINITE = -4
GNA_ERR_WORKSPACE = -5
GNA_ERR_UNSUPPORTED = -6
GNA_WARN_DEGENERATE_WEIGHTS = 1

PREC_FP64, PREC_FP32, PREC_BF16, PREC_BF16X2 = 0, 1, 2, 3
ACT_TANH, ACT_RELU_LN = 0, 1
ELOC_FULL, ELOC_INCREMENTAL = 0, 1
OP_FORWARD, OP_ELOC_FULL, OP_ELOC_INCR, OP_METROPOLIS, OP_BACKWARD, OP_ISGO_WEIGHTS, OP_ISGO_GRAD, \
    OP_METROPOLIS_LEARNED, OP_ELOC_LOGPSI = range(9)

EXPORTED = [
    "gna_version", "gna_status_string", "gna_graph_create", "gna_graph_create_xxz", "gna_graph_destroy", "gna_graph_info",
    "gna_ball_sizes_host", "gna_model_desc_init", "gna_num_params", "gna_workspace_size", "gna_forward",
    "gna_local_energy", "gna_local_energy_logpsi", "gna_metropolis_sweep", "gna_backward", "gna_backward_static",
    "gna_isgo_weights_workspace", "gna_isgo_weights", "isgo_grad",
    "gna_sgd_update", "gna_philox4x64_10", "gna_device_status", "gna_proposal_num_params",
    "gna_proposal_workspace_size", "gna_proposal_logits", "gna_proposal_grad", "gna_proposal_adam",
    "gna_dedup_workspace_size", "gna_dedup", "gna_debug_wait_limit",
    "gna_isgo_partials", "gna_isgo_finish",
]


class GnaError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: status {status} ({status_string(status)})")


class ModelDesc(ctypes.Structure):
    _fields_ = [("F", ctypes.c_int32), ("L", ctypes.c_int32), ("act", ctypes.c_int32),
                ("prec", ctypes.c_int32), ("shared_weights", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()

vp = ctypes.c_void_p
i32 = ctypes.c_int32
i64 = ctypes.c_int64
u64 = ctypes.c_uint64
sz = ctypes.c_size_t
dbl = ctypes.c_double


def lib():
    """Loads libgna.so (built by paper_2011_12453_gb300.build); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise GnaError(GNA_ERR_UNSUPPORTED, f"libgna.so not built ({_LIB_PATH}); run paper_2011_12453_gb300.build")
        L = ctypes.CDLL(_LIB_PATH)
        sig = {
            "gna_version": (i32, []),
            "gna_status_string": (ctypes.c_char_p, [i32]),
            "gna_graph_create": (i32, [i32, i32, vp, vp, i32, ctypes.POINTER(vp)]),
            "gna_graph_create_xxz": (i32, [i32, i32, vp, vp, vp, vp, vp, i32, ctypes.POINTER(vp)]),
            "gna_graph_destroy": (i32, [vp]),
            "gna_graph_info": (i32, [vp, vp, vp, vp]),
            "gna_ball_sizes_host": (i32, [i32, i32, vp, i32, vp]),
            "gna_model_desc_init": (i32, [ctypes.POINTER(ModelDesc), i32, i32, i32, i32, i32]),
            "gna_num_params": (i64, [ctypes.POINTER(ModelDesc)]),
            "gna_workspace_size": (i32, [vp, ctypes.POINTER(ModelDesc), i32, i64, ctypes.POINTER(sz)]),
            "gna_forward": (i32, [vp, ctypes.POINTER(ModelDesc), vp, vp, i64, vp, vp, sz, vp]),
            "gna_local_energy": (i32, [vp, ctypes.POINTER(ModelDesc), vp, vp, i64, i32, vp, vp, vp, sz, vp]),
            "gna_local_energy_logpsi": (i32, [vp, ctypes.POINTER(ModelDesc), vp, vp, i64, vp, vp, vp, sz, vp]),
            "gna_metropolis_sweep": (i32, [vp, ctypes.POINTER(ModelDesc), vp, vp, i64, i32, i32, u64, u64,
                                           vp, dbl, vp, vp, vp, vp, vp, sz, vp]),
            "gna_proposal_num_params": (i32, []),
            "gna_proposal_workspace_size": (i32, [vp, i64, ctypes.POINTER(sz)]),
            "gna_proposal_logits": (i32, [vp, vp, i64, vp, vp, vp]),
            "gna_proposal_grad": (i32, [vp, vp, vp, i64, vp, vp, vp, vp, sz, vp]),
            "gna_proposal_adam": (i32, [vp, vp, vp, vp, i32, dbl, vp]),
            "gna_backward": (i32, [vp, ctypes.POINTER(ModelDesc), vp, vp, i64, vp, vp, vp, sz, vp]),
            "gna_backward_static": (i32, [vp, ctypes.POINTER(ModelDesc), vp, vp, i64, vp, vp, vp]),
            "gna_isgo_weights_workspace": (i32, [i64, ctypes.POINTER(sz)]),
            "gna_isgo_weights": (i32, [vp, vp, vp, vp, i64, vp, vp, vp, sz, vp]),
            "isgo_grad": (i32, [vp, ctypes.POINTER(ModelDesc), vp, vp, vp, vp, i64, vp, vp, vp, sz, vp]),
            "gna_sgd_update": (i32, [ctypes.POINTER(ModelDesc), vp, vp, dbl, vp]),
            "gna_philox4x64_10": (i32, [vp, vp, i64, vp, vp]),
            "gna_device_status": (i32, [ctypes.POINTER(i32), i32]),
            "gna_dedup_workspace_size": (i32, [i64, i32, ctypes.POINTER(sz)]),
            "gna_dedup": (i32, [i32, vp, vp, i64, vp, vp, vp, vp, vp, sz, vp]),
            "gna_debug_wait_limit": (i32, [ctypes.c_uint32]),
            "gna_isgo_partials": (i32, [vp, vp, vp, vp, i64, vp, vp, sz, vp]),
            "gna_isgo_finish": (i32, [vp, vp, vp, vp, i64, vp, vp, vp, vp, sz, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return _lib


def status_string(st: int) -> str:
    try:
        return lib().gna_status_string(int(st)).decode()
    except Exception:
        return "?"


def _check(st: int, what: str) -> int:
    if st < 0:
        raise GnaError(st, what)
    return st


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _stream():
    import torch

    return torch.cuda.current_stream().cuda_stream


# ---------------------------------------------------------------------------------
# graph and model
# ---------------------------------------------------------------------------------

def ball_sizes_host(n_sites: int, edges: np.ndarray, n_layers: int) -> np.ndarray:
    """|ball_l(e)| for l = 0..n_layers of every bond (host only, no CUDA call)."""
    e = np.ascontiguousarray(edges, dtype=np.int32)
    out = np.zeros((e.shape[0], n_layers + 1), dtype=np.int32)
    _check(lib().gna_ball_sizes_host(n_sites, e.shape[0], e.ctypes.data if e.size else None, n_layers,
                                     out.ctypes.data if out.size else None), "gna_ball_sizes_host")
    return out


class Graph:
    """Device-resident graph handle: Heisenberg bonds J (gna_graph_create), or XXZ bonds
    xxz = (Jz, Jxy, hz, c) (gna_graph_create_xxz; J is then ignored)."""

    def __init__(self, n_sites: int, edges: np.ndarray, J: np.ndarray, max_layers: int, xxz=None):
        e = np.ascontiguousarray(edges, dtype=np.int32)
        h = vp()
        self._h = None
        if xxz is None:
            j = np.ascontiguousarray(J, dtype=np.float64)
            _check(lib().gna_graph_create(n_sites, e.shape[0], e.ctypes.data if e.size else None,
                                          j.ctypes.data if j.size else None, max_layers, ctypes.byref(h)),
                   "gna_graph_create")
        else:
            a = [np.ascontiguousarray(np.broadcast_to(np.asarray(x, dtype=np.float64), (e.shape[0],)))
                 for x in xxz]
            j = a[1]
            _check(lib().gna_graph_create_xxz(n_sites, e.shape[0], e.ctypes.data if e.size else None,
                                              *[x.ctypes.data if x.size else None for x in a],
                                              max_layers, ctypes.byref(h)),
                   "gna_graph_create_xxz")
        self._h = h
        self.n_sites = n_sites
        self.n_edges = int(e.shape[0])
        self.max_layers = max_layers
        self.edges = e
        self.J = j

    @classmethod
    def from_workload(cls, g, max_layers: int) -> "Graph":
        return cls(g.n_sites, g.edges, g.J, max_layers)

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            try:
                _lib.gna_graph_destroy(self._h)
            except Exception:
                pass
            self._h = None


class Model:
    def __init__(self, F: int, L: int, prec: int = PREC_FP64, shared: bool = True, act: int = ACT_TANH):
        self.desc = ModelDesc()
        _check(lib().gna_model_desc_init(ctypes.byref(self.desc), F, L, act, prec, int(shared)),
               "gna_model_desc_init")
        self.F, self.L, self.prec, self.shared, self.act = F, L, prec, bool(shared), act

    @property
    def num_params(self) -> int:
        return int(lib().gna_num_params(ctypes.byref(self.desc)))

    def theta_dtype(self):
        import torch

        return torch.float64 if self.prec == PREC_FP64 else torch.float32


def workspace_size(graph: Graph, model: Model, op: int, B: int) -> int:
    out = sz(0)
    _check(lib().gna_workspace_size(graph.handle, ctypes.byref(model.desc), op, B, ctypes.byref(out)),
           "gna_workspace_size")
    return int(out.value)


_ws_cache: dict = {}


def workspace(nbytes: int, device=None):
    """A reusable uint8 device buffer of at least nbytes (grown on demand, per device)."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    buf = _ws_cache.get(dev)
    if buf is None or buf.numel() < nbytes:
        buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev)
        _ws_cache[dev] = buf
    return buf


def _ws_for(graph, model, op, B):
    n = workspace_size(graph, model, op, B)
    w = workspace(n)
    return w.data_ptr(), w.numel()


# ---------------------------------------------------------------------------------
# compute
# ---------------------------------------------------------------------------------

def _check_theta(model: Model, theta):
    import torch

    if theta.dtype != model.theta_dtype() or not theta.is_cuda or not theta.is_contiguous():
        raise GnaError(GNA_ERR_INVALID_ARG, f"theta must be a contiguous CUDA {model.theta_dtype()} tensor")
    if theta.numel() != model.num_params:
        raise GnaError(GNA_ERR_INVALID_ARG, f"theta has {theta.numel()} entries, expected {model.num_params}")
    return torch


def _check_spins(graph: Graph, spins):
    import torch

    if spins.dtype != torch.int8 or not spins.is_cuda or not spins.is_contiguous() or spins.dim() != 2 \
            or spins.shape[1] != graph.n_sites:
        raise GnaError(GNA_ERR_INVALID_ARG, "spins must be a contiguous CUDA int8 [B][n_sites] tensor")


def forward(graph: Graph, model: Model, theta, spins, out=None):
    """log Psi(s) of each row of spins: float64 [B][2] (Re, Im)."""
    torch = _check_theta(model, theta)
    _check_spins(graph, spins)
    B = spins.shape[0]
    lp = out if out is not None else torch.empty((B, 2), dtype=torch.float64, device=spins.device)
    w, wn = _ws_for(graph, model, OP_FORWARD, B)
    _check(lib().gna_forward(graph.handle, ctypes.byref(model.desc), theta.data_ptr(), spins.data_ptr(), B,
                             lp.data_ptr(), w, wn, _stream()), "gna_forward")
    return lp


def local_energy(graph: Graph, model: Model, theta, spins, mode: int = ELOC_INCREMENTAL, bonds: bool = False,
                 out=None):
    """E_loc of each row of spins: float64 [B][2]; with bonds=True also float32 [B][E] Re Delta."""
    torch = _check_theta(model, theta)
    _check_spins(graph, spins)
    B = spins.shape[0]
    E = out if out is not None else torch.empty((B, 2), dtype=torch.float64, device=spins.device)
    dl = torch.empty((B, graph.n_edges), dtype=torch.float32, device=spins.device) if bonds else None
    op = OP_ELOC_FULL if mode == ELOC_FULL else OP_ELOC_INCR
    w, wn = _ws_for(graph, model, op, B)
    _check(lib().gna_local_energy(graph.handle, ctypes.byref(model.desc), theta.data_ptr(), spins.data_ptr(), B,
                                  mode, E.data_ptr(), _ptr(dl), w, wn, _stream()), "gna_local_energy")
    return (E, dl) if bonds else E


def local_energy_logpsi(graph: Graph, model: Model, theta, spins, out=None, out_logpsi=None):
    """Incremental E_loc and log Psi of each row of spins in one call: (float64 [B][2],
    float64 [B][2]), equal to local_energy(..., ELOC_INCREMENTAL) and forward(...)."""
    torch = _check_theta(model, theta)
    _check_spins(graph, spins)
    B = spins.shape[0]
    E = out if out is not None else torch.empty((B, 2), dtype=torch.float64, device=spins.device)
    lp = out_logpsi if out_logpsi is not None else torch.empty((B, 2), dtype=torch.float64, device=spins.device)
    w, wn = _ws_for(graph, model, OP_ELOC_LOGPSI, B)
    _check(lib().gna_local_energy_logpsi(graph.handle, ctypes.byref(model.desc), theta.data_ptr(), spins.data_ptr(),
                                         B, E.data_ptr(), lp.data_ptr(), w, wn, _stream()), "gna_local_energy_logpsi")
    return E, lp


def metropolis_sweep(graph: Graph, model: Model, theta, chain_spins, n_sweeps: int, record_every: int, seed: int,
                     step0: int, trace: bool = False, n_accepted=None, records: bool = True, proposal=None,
                     eps: float = 0.1, record_logpsi: bool = True):
    """Advance the chains in place; returns (samples [R][C][N] int8, logpsi [R][C][2], n_accepted [C], trace).

    proposal: float32 CUDA tensor of the proposal network's parameters (learned moves
    mixed with plain ones with probability eps) or None (plain moves).  trace rows are
    (bond or -1, accepted, value, kind).  record_logpsi=False records the samples only
    (logpsi is then None)."""
    torch = _check_theta(model, theta)
    _check_spins(graph, chain_spins)
    C = chain_spins.shape[0]
    R = n_sweeps // record_every if (record_every > 0 and records) else 0
    dev = chain_spins.device
    samples = torch.empty((R, C, graph.n_sites), dtype=torch.int8, device=dev) if R else None
    lpo = torch.empty((R, C, 2), dtype=torch.float64, device=dev) if R and record_logpsi else None
    acc = n_accepted if n_accepted is not None else torch.zeros(C, dtype=torch.int32, device=dev)
    tr = torch.empty((C, n_sweeps * graph.n_sites, 4), dtype=torch.float64, device=dev) if trace else None
    op = OP_METROPOLIS_LEARNED if proposal is not None else OP_METROPOLIS
    w, wn = _ws_for(graph, model, op, C)
    _check(lib().gna_metropolis_sweep(graph.handle, ctypes.byref(model.desc), theta.data_ptr(),
                                      chain_spins.data_ptr(), C, n_sweeps, record_every if R else 0, seed, step0,
                                      _ptr(proposal), float(eps), _ptr(samples), _ptr(lpo), acc.data_ptr(), _ptr(tr),
                                      w, wn, _stream()),
           "gna_metropolis_sweep")
    return samples, lpo, acc, tr


# ---------------------------------------------------------------------------------
# learned proposal
# ---------------------------------------------------------------------------------

def proposal_num_params() -> int:
    return int(lib().gna_proposal_num_params())


def proposal_logits(graph: Graph, spins, params):
    """float32 [B][E][2] logits (NaN on parallel bonds)."""
    import torch

    _check_spins(graph, spins)
    B = spins.shape[0]
    out = torch.empty((B, graph.n_edges, 2), dtype=torch.float32, device=spins.device)
    _check(lib().gna_proposal_logits(graph.handle, spins.data_ptr(), B, params.data_ptr(), out.data_ptr(), _stream()),
           "gna_proposal_logits")
    return out


def proposal_grad(graph: Graph, spins, dlogpsi_bonds, params):
    """(grad float64 [P], loss float64 [1]) of the proposal network's training loss."""
    import torch

    _check_spins(graph, spins)
    B = spins.shape[0]
    grad = torch.empty(proposal_num_params(), dtype=torch.float64, device=spins.device)
    loss = torch.empty(1, dtype=torch.float64, device=spins.device)
    n = sz(0)
    _check(lib().gna_proposal_workspace_size(graph.handle, B, ctypes.byref(n)), "gna_proposal_workspace_size")
    w = workspace(int(n.value))
    _check(lib().gna_proposal_grad(graph.handle, spins.data_ptr(), dlogpsi_bonds.contiguous().data_ptr(), B,
                                   params.data_ptr(), grad.data_ptr(), loss.data_ptr(), w.data_ptr(), w.numel(),
                                   _stream()), "gna_proposal_grad")
    return grad, loss


def proposal_adam(params, m, v, grad, t: int, lr: float):
    _check(lib().gna_proposal_adam(params.data_ptr(), m.data_ptr(), v.data_ptr(), grad.data_ptr(), int(t), float(lr),
                                   _stream()), "gna_proposal_adam")
    return params


def backward(graph: Graph, model: Model, theta, spins, cot, out=None):
    """sum_x cot[x] . d log Psi_x / d theta: float64 [P]."""
    torch = _check_theta(model, theta)
    _check_spins(graph, spins)
    B = spins.shape[0]
    g = out if out is not None else torch.empty(model.num_params, dtype=torch.float64, device=theta.device)
    cot = cot.contiguous()
    w, wn = _ws_for(graph, model, OP_BACKWARD, B)
    _check(lib().gna_backward(graph.handle, ctypes.byref(model.desc), theta.data_ptr(), spins.data_ptr(), B,
                              cot.data_ptr(), g.data_ptr(), w, wn, _stream()), "gna_backward")
    return g


def backward_static(graph: Graph, model: Model, theta, spins, cot, out=None):
    """As backward(), through gna_backward_static: no workspace, no device allocation by
    the library (its scratch is a fixed array inside libgna.so shared by all calls)."""
    torch = _check_theta(model, theta)
    _check_spins(graph, spins)
    B = spins.shape[0]
    g = out if out is not None else torch.empty(model.num_params, dtype=torch.float64, device=theta.device)
    cot = cot.contiguous()
    _check(lib().gna_backward_static(graph.handle, ctypes.byref(model.desc), theta.data_ptr(), spins.data_ptr(), B,
                                     cot.data_ptr(), g.data_ptr(), _stream()), "gna_backward_static")
    return g


def isgo_weights(logpsi, logpsi0, eloc, counts=None):
    """(cot [B][2], stats [4] = (Re Ebar, Im Ebar, var, ess)) on the device."""
    import torch

    B = logpsi.shape[0]
    cot = torch.empty((B, 2), dtype=torch.float64, device=logpsi.device)
    stats = torch.empty(4, dtype=torch.float64, device=logpsi.device)
    need = sz(0)
    _check(lib().gna_isgo_weights_workspace(B, ctypes.byref(need)), "gna_isgo_weights_workspace")
    w = workspace(int(need.value))
    _check(lib().gna_isgo_weights(logpsi.data_ptr(), logpsi0.data_ptr(), eloc.data_ptr(), _ptr(counts), B,
                                  cot.data_ptr(), stats.data_ptr(), w.data_ptr(), w.numel(), _stream()),
           "gna_isgo_weights")
    return cot, stats


def isgo_partials(logpsi, logpsi0, eloc, counts=None):
    """This shard's (m, S, S Re Ebar, S Im Ebar): float64 [4] on the device."""
    import torch

    B = logpsi.shape[0]
    part = torch.empty(4, dtype=torch.float64, device=logpsi.device)
    need = sz(0)
    _check(lib().gna_isgo_weights_workspace(B, ctypes.byref(need)), "gna_isgo_weights_workspace")
    w = workspace(int(need.value))
    _check(lib().gna_isgo_partials(logpsi.data_ptr(), logpsi0.data_ptr(), eloc.data_ptr(), _ptr(counts), B,
                                   part.data_ptr(), w.data_ptr(), w.numel(), _stream()), "gna_isgo_partials")
    return part


def isgo_finish(logpsi, logpsi0, eloc, global4, counts=None):
    """(cot [B][2], (sum p |E - Ebar|^2, sum p^2/c, sum c) [3]) of this shard on the device."""
    import torch

    B = logpsi.shape[0]
    cot = torch.empty((B, 2), dtype=torch.float64, device=logpsi.device)
    part = torch.empty(3, dtype=torch.float64, device=logpsi.device)
    need = sz(0)
    _check(lib().gna_isgo_weights_workspace(B, ctypes.byref(need)), "gna_isgo_weights_workspace")
    w = workspace(int(need.value))
    _check(lib().gna_isgo_finish(logpsi.data_ptr(), logpsi0.data_ptr(), eloc.data_ptr(), _ptr(counts), B,
                                 global4.data_ptr(), cot.data_ptr(), part.data_ptr(), w.data_ptr(), w.numel(),
                                 _stream()), "gna_isgo_finish")
    return cot, part


def isgo_grad(graph: Graph, model: Model, theta, spins, logpsi0, counts=None, grad=None, stats=None):
    """One ISGO gradient on the device: (grad float64 [P], stats float64 [4])."""
    torch = _check_theta(model, theta)
    _check_spins(graph, spins)
    B = spins.shape[0]
    g = grad if grad is not None else torch.empty(model.num_params, dtype=torch.float64, device=theta.device)
    s = stats if stats is not None else torch.empty(4, dtype=torch.float64, device=theta.device)
    w, wn = _ws_for(graph, model, OP_ISGO_GRAD, B)
    _check(lib().isgo_grad(graph.handle, ctypes.byref(model.desc), theta.data_ptr(), spins.data_ptr(),
                           logpsi0.data_ptr(), _ptr(counts), B, g.data_ptr(), s.data_ptr(), w, wn, _stream()),
           "isgo_grad")
    return g, s


def sgd_update(model: Model, theta, grad, lr: float):
    _check_theta(model, theta)
    _check(lib().gna_sgd_update(ctypes.byref(model.desc), theta.data_ptr(), grad.data_ptr(), float(lr), _stream()),
           "gna_sgd_update")
    return theta


def dedup(spins, logpsi=None):
    """Group duplicated samples: (unique spins [U][N], their log Psi^0 [U][2] or None,
    counts float64 [U]) in order of first occurrence.  Reads U back to the host."""
    import torch

    B, N = spins.shape
    dev = spins.device
    us = torch.empty_like(spins)
    ul = torch.empty((B, 2), dtype=torch.float64, device=dev) if logpsi is not None else None
    uc = torch.empty(B, dtype=torch.float64, device=dev)
    n = torch.zeros(1, dtype=torch.int64, device=dev)
    need = sz(0)
    _check(lib().gna_dedup_workspace_size(B, N, ctypes.byref(need)), "gna_dedup_workspace_size")
    w = workspace(int(need.value))
    _check(lib().gna_dedup(N, spins.data_ptr(), _ptr(logpsi), B, us.data_ptr(), _ptr(ul), uc.data_ptr(),
                           n.data_ptr(), w.data_ptr() if w.numel() else None, w.numel(), _stream()), "gna_dedup")
    U = int(n.item())
    return us[:U], (ul[:U] if ul is not None else None), uc[:U]


def philox(keys, counters):
    """Philox4x64-10 blocks: keys uint64-as-int64 [n][2], counters [n][4] -> [n][4] (CUDA tensors)."""
    import torch

    n = keys.shape[0]
    out = torch.empty((n, 4), dtype=torch.int64, device=keys.device)
    _check(lib().gna_philox4x64_10(keys.data_ptr(), counters.data_ptr(), n, out.data_ptr(), _stream()),
           "gna_philox4x64_10")
    return out


def device_status(clear: bool = True, with_status: bool = False):
    """Bit mask of the conditions kernels recorded (1 wait timed out, 2 non-finite, 4
    degenerate importance weights); with_status=True also returns the call's status (the
    most severe condition as a gna_status code)."""
    f = i32(0)
    st = lib().gna_device_status(ctypes.byref(f), int(clear))
    if st == GNA_ERR_CUDA:
        _check(st, "gna_device_status")
    return (int(f.value), int(st)) if with_status else int(f.value)


def debug_wait_limit(iterations: int | None) -> None:
    """Test hook: iteration limit of the tensor-core kernels' MMA waits (None: the default)."""
    _check(lib().gna_debug_wait_limit(ctypes.c_uint32(0xFFFFFFFF if iterations is None else iterations)),
           "gna_debug_wait_limit")


# ---------------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------------

def _autograd_class():
    import torch

    class GCNLogPsi(torch.autograd.Function):
        """log Psi(theta; s) with the library's hand-written backward as its derivative."""

        @staticmethod
        def forward(ctx, theta, spins, graph, model):
            ctx.save_for_backward(theta, spins)
            ctx.graph, ctx.model = graph, model
            return forward(graph, model, theta.detach().contiguous(), spins)

        @staticmethod
        def backward(ctx, gout):
            theta, spins = ctx.saved_tensors
            g = backward(ctx.graph, ctx.model, theta.detach().contiguous(), spins,
                         gout.to(torch.float64).contiguous())
            return g.to(theta.dtype), None, None, None

    return GCNLogPsi


_GCN = None


def gcn_logpsi(theta, spins, graph: Graph, model: Model):
    """Differentiable log Psi: float64 [B][2]; backward runs gna_backward."""
    global _GCN
    if _GCN is None:
        _GCN = _autograd_class()
    return _GCN.apply(theta, spins, graph, model)
