"""Temporal-stream parity (the real-dynamic-graph workload of Sec. 5.1.4 /
Sec. 5.2.1 at reduced size): a copying / preferential-attachment stream with
repeats and a heavy-tailed out-degree over 2^18 vertices and 24 edges per
vertex; the first 90% in timestamp order is the base graph, then ten
consecutive insertion-only batches of 1e-3 |E_T| follow, each with a DF-P
update.  Insertions land on the same hub rows again and again and repeat
earlier edges, so the batch edit takes its slack, repack and
ineffective-change paths.

Both sides start from the oracle's Static ranks of the base graph (the
previous snapshot's ranks are an input of Alg. 1).  Per batch:
  * the GPU's DF-P from the oracle's previous ranks equals the oracle's DF-P
    within 1e-9, with the same iterations, vertices ever affected and vertex
    updates (unless the oracle reports a near-tie that explains a difference);
  * the GPU's own chain (each update from its own previous DF-P ranks) stays
    within 1e-9 of the oracle's chain;
  * the edge sets and the effective change are bit-exact.
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


def test_temporal_stream_chained_dfp_matches_oracle(lib):
    n = 1 << 18
    m_t = 24 * n
    src, dst = synth.temporal(n, m_t, 3003)
    base = int(0.9 * m_t)
    bsize = m_t // 1000
    G = lib.Graph.from_edges(n, src[:base], dst[:base])
    O = oracle.Graph(n, src[:base], dst[:base])
    r_cpu, _ = O.update("static")
    r_gpu = r_cpu.copy()
    pos = base
    for step in range(10):
        s, d = src[pos:pos + bsize], dst[pos:pos + bsize]
        pos += bsize
        G.apply_batch(ins_src=s, ins_dst=d)
        O.apply_batch(ins_src=s, ins_dst=d)
        gd, gp = G.effective_delta()
        od, op = O.effective_delta()
        assert gd.size == 0 and np.array_equal(gp, op), step
        assert G.m == O.m, step
        ref, ost = O.update("dfp", r_prev=r_cpu)
        # the same previous ranks on both sides
        G.set_ranks(r_cpu)
        st = G.update("dfp")
        assert np.max(np.abs(G.ranks() - ref)) < TOL, step
        assert_same_run(st, ost, step)
        # the GPU's own chain
        G.set_ranks(r_gpu)
        G.update("dfp")
        r_gpu = G.ranks()
        r_cpu = ref
        assert np.max(np.abs(r_gpu - r_cpu)) < TOL, step
    # the graphs are still the same edge set
    go, gi = G.out_csr(), O.out_csr()
    assert np.array_equal(go[0], gi[0]) and np.array_equal(go[1], gi[1])
