"""Vertex insertion and deletion (pr_graph_resize) against the oracle.

Growing adds isolated vertices (self-loop only) at the end of the id range and
carries the ranks over by the closed form r * n / n_new (1 / n_new on the new
vertices); shrinking removes isolated vertices at the end.  Edge sets must be
bit-exact, carried ranks bit-identical to the oracle's rule, and the DF-P / ND
updates of a batch that connects the new vertices within 1e-9 with the same
iterations and frontier as the oracle's.
"""
import numpy as np
import pytest

import oracle
import synth
from cases import assert_same_run

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def lib():
    import paper_2401_15870_gb300 as pr
    pr.load()
    return pr


def same_graph(G, O):
    for mine, ref in ((G.out_csr(), O.out_csr()), (G.in_csr(), O.in_csr())):
        assert np.array_equal(mine[0], ref[0]) and np.array_equal(mine[1], ref[1])


@pytest.mark.parametrize("keep_order", [False, True])
def test_grow_then_batch_then_update(lib, keep_order):
    scale = 12
    n = 1 << scale
    src, dst = synth.rmat(scale, 16 * n, 501)
    G = lib.Graph.from_edges(n, src, dst, keep_order=keep_order)
    O = oracle.Graph(n, src, dst)
    r0, _ = O.update("static")
    G.set_ranks(r0)
    n_new = n + 777
    G.resize(n_new)
    O.resize(n_new)
    assert G.n == n_new and G.m == O.m
    same_graph(G, O)
    carried = oracle.resize_ranks(r0, n_new)
    assert np.array_equal(G.ranks(), carried)
    # nothing to do until a batch arrives
    st = G.update("dfp")
    assert st.vertices_processed == 0 and np.array_equal(G.ranks(), carried)
    # a batch that connects the new vertices to the old ones and to each other
    rng = np.random.default_rng(5)
    new = np.arange(n, n_new, dtype=np.int32)
    old = rng.integers(0, n, new.size).astype(np.int32)
    ins_s = np.concatenate([new, old, new[:100]]).astype(np.int32)
    ins_d = np.concatenate([old, new, new[100:200]]).astype(np.int32)
    cs, cd = synth.unique_edges(src, dst)
    ds, dd, _, _ = synth.batch(n, cs, cd, 200, 77)
    G.apply_batch(ds, dd, ins_s, ins_d)
    O.apply_batch(ds, dd, ins_s, ins_d)
    same_graph(G, O)
    for method in ("dfp", "df", "nd"):
        G.set_ranks(carried)
        st = G.update(method)
        ref, ost = O.update(method, r_prev=carried)
        assert np.max(np.abs(G.ranks() - ref)) < TOL, method
        assert_same_run(st, ost, method)


def test_shrink_after_deleting_edges(lib):
    scale = 11
    n = 1 << scale
    src, dst = synth.rmat(scale, 8 * n, 502)
    G = lib.Graph.from_edges(n, src, dst)
    O = oracle.Graph(n, src, dst)
    r0, _ = O.update("static")
    G.set_ranks(r0)
    n_new = n - 100
    # refused while the tail has edges; nothing changes
    with pytest.raises(lib.PRError) as e:
        G.resize(n_new)
    assert e.value.status == 1
    same_graph(G, O)
    assert np.array_equal(G.ranks(), r0)
    # delete every edge with an end in the tail, update, then remove the tail
    off, adj = O.out_csr()
    us = np.repeat(np.arange(n), np.diff(off))
    cut = (us != adj) & ((us >= n_new) | (adj >= n_new))
    G.apply_batch(us[cut].astype(np.int32), adj[cut].astype(np.int32))
    O.apply_batch(us[cut].astype(np.int32), adj[cut].astype(np.int32))
    G.set_ranks(r0)
    G.update("dfp")
    r1, _ = O.update("dfp", r_prev=r0)
    assert np.max(np.abs(G.ranks() - r1)) < TOL
    G.set_ranks(r1)
    G.resize(n_new)
    O.resize(n_new)
    same_graph(G, O)
    assert np.array_equal(G.ranks(), oracle.resize_ranks(r1, n_new))
    # the smaller graph takes batches and updates as before
    off, adj = O.out_csr()
    us = np.repeat(np.arange(n_new), np.diff(off)).astype(np.int32)
    b = synth.batch(n_new, *synth.unique_edges(us, adj), 150, 9)
    carried = oracle.resize_ranks(r1, n_new)
    G.apply_batch(*b)
    O.apply_batch(*b)
    G.set_ranks(carried)
    st = G.update("dfp")
    ref, ost = O.update("dfp", r_prev=carried)
    assert np.max(np.abs(G.ranks() - ref)) < TOL
    assert_same_run(st, ost)


def test_resize_argument_errors(lib):
    G = lib.Graph.from_edges(8, [0, 1], [1, 2])
    for bad in (0, -3):
        with pytest.raises(lib.PRError) as e:
            G.resize(bad)
        assert e.value.status == 1
    G.resize(8)                          # same size: nothing to do
    assert G.n == 8
