"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every symbol
include/gna.h declares, and its host logic (argument validation, parameter count, bond
neighbourhood sizes) agrees with independent Python code."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2011_12453_gb300 import build as B, gna, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def _header_symbols():
    text = open(os.path.join(ROOT, "include", "gna.h")).read()
    return sorted(set(re.findall(r"^GNA_API [^()]*?\b(\w+)\(", text, flags=re.M)))


def test_exports_every_declared_symbol():
    syms = _header_symbols()
    assert len(syms) >= 18
    L = ctypes.CDLL(B.LIB)
    for s in syms:
        assert hasattr(L, s), s
    assert sorted(gna.EXPORTED) == syms


def test_version_and_status_strings():
    assert gna.lib().gna_version() == 1
    assert gna.status_string(gna.GNA_ERR_WORKSPACE) == "workspace too small"


@pytest.mark.parametrize("F,L,shared", [(16, 2, True), (32, 4, True), (48, 4, False), (64, 6, True), (5, 0, False)])
def test_num_params_matches_layout(F, L, shared):
    m = gna.Model(F, L, gna.PREC_FP64, shared)
    assert m.num_params == W.num_params(F, L, shared)


@pytest.mark.parametrize("args", [(0, 2, 0, 0, 1), (65, 2, 0, 0, 1), (16, 9, 0, 0, 1), (16, 2, 2, 0, 1),
                                  (16, 2, 0, 4, 1), (16, 2, 0, 0, 2), (24, 2, 0, 2, 1), (24, 2, 0, 3, 1)])
def test_model_desc_rejects(args):
    d = gna.ModelDesc()
    assert gna.lib().gna_model_desc_init(ctypes.byref(d), *args) == gna.GNA_ERR_INVALID_ARG


def test_model_desc_accepts_relu_ln():
    d = gna.ModelDesc()
    for prec in (0, 1, 2, 3):
        assert gna.lib().gna_model_desc_init(ctypes.byref(d), 16, 3, gna.ACT_RELU_LN, prec, 1) == gna.GNA_OK
        assert d.act == gna.ACT_RELU_LN


def _bfs_balls(n, edges, L):
    nb = [set() for _ in range(n)]
    for a, b in edges.tolist():
        nb[a].add(b)
        nb[b].add(a)
    out = []
    for a, b in edges.tolist():
        ball = {a, b}
        sizes = [2]
        for _ in range(L):
            ball = ball | set().union(*[nb[v] for v in ball])
            sizes.append(len(ball))
        out.append(sizes)
    return np.array(out)


@pytest.mark.parametrize("name", ["kagome6", "tri", "er"])
def test_ball_sizes_match_bfs(name):
    g = {"kagome6": W.kagome(6), "tri": W.triangular(6, 5), "er": W.erdos_renyi(40, 0.1, seed=3)}[name]
    L = 5
    np.testing.assert_array_equal(gna.ball_sizes_host(g.n_sites, g.edges, L), _bfs_balls(g.n_sites, g.edges, L))


def test_ball_sizes_of_the_benchmark_lattices():
    # |ball_l| of one bond: Kagome 2, 7, 17, 32, 52, 75, 105 (12x12x3); triangular 2, 10, 24, 44, 70
    k = gna.ball_sizes_host(432, W.kagome(12).edges, 6)
    assert (k == [2, 7, 17, 32, 52, 75, 105]).all()
    t = gna.ball_sizes_host(144, W.triangular(12, 12).edges, 4)
    assert (t == [2, 10, 24, 44, 70]).all()


@pytest.mark.parametrize("n,edges", [
    (3, [[0, 0]]),            # self-loop
    (3, [[0, 1], [1, 0]]),    # duplicate in the other orientation
    (3, [[0, 3]]),            # out of range
    (3, [[-1, 1]]),
    (0, []),                  # no site
    (5000, []),               # too many sites
])
def test_graph_validation_rejects(n, edges):
    e = np.array(edges, dtype=np.int32).reshape(-1, 2)
    with pytest.raises(gna.GnaError) as ei:
        gna.ball_sizes_host(n, e, 2)
    assert ei.value.status == gna.GNA_ERR_INVALID_ARG
    # graph creation validates on the host before any device call
    J = np.ones(e.shape[0])
    h = gna.vp()
    st = gna.lib().gna_graph_create(n, e.shape[0], e.ctypes.data if e.size else None,
                                    J.ctypes.data if J.size else None, 2, ctypes.byref(h))
    assert st == gna.GNA_ERR_INVALID_ARG and not h.value


def test_nonfinite_coupling_rejected():
    e = np.array([[0, 1]], dtype=np.int32)
    J = np.array([np.nan])
    h = gna.vp()
    assert gna.lib().gna_graph_create(2, 1, e.ctypes.data, J.ctypes.data, 1, ctypes.byref(h)) == gna.GNA_ERR_INVALID_ARG


def test_isgo_workspace_query():
    n = gna.sz(0)
    assert gna.lib().gna_isgo_weights_workspace(1000, ctypes.byref(n)) == 0 and n.value > 0
    assert gna.lib().gna_isgo_weights_workspace(0, ctypes.byref(n)) == gna.GNA_ERR_INVALID_ARG


def test_xxz_graph_validation():
    e = np.array([[0, 1], [1, 2]], dtype=np.int32)
    ok = np.ones(2)
    bad = np.array([1.0, np.inf])
    h = gna.vp()
    lib = gna.lib()
    # any missing coefficient array, or a non-finite one, is rejected on the host
    for arrs in [(None, ok, ok, ok), (ok, None, ok, ok), (ok, ok, None, ok), (ok, ok, ok, None),
                 (bad, ok, ok, ok), (ok, bad, ok, ok), (ok, ok, bad, ok), (ok, ok, ok, bad)]:
        ptrs = [a.ctypes.data if a is not None else None for a in arrs]
        assert lib.gna_graph_create_xxz(3, 2, e.ctypes.data, *ptrs, 1, ctypes.byref(h)) == gna.GNA_ERR_INVALID_ARG
        assert not h.value


def test_compute_calls_reject_a_missing_graph():
    # argument checks that run before any device work: a null graph handle is refused by every
    # compute entry point with GNA_ERR_INVALID_ARG (no GPU needed)
    lib = gna.lib()
    d = gna.ModelDesc()
    assert lib.gna_model_desc_init(ctypes.byref(d), 16, 2, 0, gna.PREC_BF16X2, 1) == gna.GNA_OK
    p = ctypes.c_void_p(1)  # never dereferenced: the graph check comes first
    assert lib.gna_forward(None, ctypes.byref(d), p, p, 4, p, p, 0, None) == gna.GNA_ERR_INVALID_ARG
    assert lib.gna_local_energy(None, ctypes.byref(d), p, p, 4, 1, p, None, p, 0, None) == gna.GNA_ERR_INVALID_ARG
    assert lib.gna_local_energy_logpsi(None, ctypes.byref(d), p, p, 4, p, p, p, 0, None) == gna.GNA_ERR_INVALID_ARG
    n = ctypes.c_size_t(0)
    assert lib.gna_workspace_size(None, ctypes.byref(d), gna.OP_ELOC_LOGPSI, 4, ctypes.byref(n)) == \
        gna.GNA_ERR_INVALID_ARG
