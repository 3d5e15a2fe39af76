"""Groups: one update of many graphs in one launch sequence with the iteration
loop on the device.  Every graph's ranks must match the oracle within 1e-9
and be bit-identical, with identical statistics, to pr_update on the graph
alone from the same previous ranks (same arithmetic; the group only changes
how the work is scheduled)."""
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


def make_case(pr, scale, ef, bsize, seed, n=None):
    """GPU graph + oracle graph, static ranks of the base graph, one batch applied."""
    n = n or (1 << scale)
    src, dst = synth.rmat(max(scale, 1), ef * n, seed)
    src, dst = src % n, dst % n
    G = pr.Graph.from_edges(n, src, dst)
    O = oracle.Graph(n, src, dst)
    r0, _ = O.update("static")
    if bsize:
        cs, cd = synth.unique_edges(src, dst)
        b = synth.batch(n, cs, cd, bsize, seed + 1)
        G.apply_batch(*b)
        O.apply_batch(*b)
    return G, O, r0


# sizes: tiny, odd, not a multiple of 32, several quad tiles, an empty batch
CASES = [(1, 2, 2, 3, None), (6, 3, 5, 4, 37), (9, 8, 40, 5, None), (12, 16, 300, 6, None), (14, 16, 262, 7, None),
         (11, 24, 0, 8, None), (13, 4, 2000, 9, 5000)]


@pytest.fixture(scope="module")
def cases(lib):
    return [make_case(lib, *c) for c in CASES]


def solo(G, r0, method, **kw):
    G.set_ranks(r0)
    st = G.update(method, **kw)
    return G.ranks(), st


def same_stats(a, b):
    return (a.iterations, a.converged, a.vertices_ever_affected, a.edges_processed, a.vertices_processed) == \
        (b.iterations, b.converged, b.vertices_ever_affected, b.edges_processed, b.vertices_processed)


@pytest.mark.parametrize("method", ["dfp", "df", "nd", "static"])
def test_group_matches_oracle_and_solo_runs(lib, cases, method):
    graphs = [c[0] for c in cases]
    grp = lib.Group(graphs)
    try:
        for G, O, r0 in cases:
            G.set_ranks(r0)
        stats = grp.update(method)
        got = [G.ranks() for G in graphs]
        for (G, O, r0), r, st in zip(cases, got, stats):
            ref, ost = O.update(method, r_prev=r0)
            assert np.max(np.abs(r - ref)) < TOL
            assert st.iterations == ost.iterations
            assert st.converged == ost.converged
            r_solo, st_solo = solo(G, r0, method)
            assert np.array_equal(r, r_solo), (G.n, method)
            assert same_stats(st, st_solo), (st, st_solo)
            if method in ("df", "dfp"):
                assert st.vertices_ever_affected == ost.vertices_ever_affected
    finally:
        grp.close()


@pytest.mark.parametrize("method", ["dfp", "static"])
def test_group_host_loop_equals_device_loop(lib, cases, method):
    """The kernels launched one by one with the condition read back on the host
    and the whole loop in one cooperative kernel give the same bits as the
    CUDA graph with its WHILE node."""
    graphs = [c[0] for c in cases]
    grp = lib.Group(graphs)
    try:
        out = []
        for loop in ("device", "one", "host"):
            for G, O, r0 in cases:
                G.set_ranks(r0)
            st = grp.update(method, loop=loop)
            out.append(([G.ranks() for G in graphs], [(s.iterations, s.vertices_ever_affected) for s in st]))
        for o in out[1:]:
            assert all(np.array_equal(a, b) for a, b in zip(out[0][0], o[0]))
            assert out[0][1] == o[1]
    finally:
        grp.close()


def test_group_max_iter_and_empty_batch(lib, cases):
    graphs = [c[0] for c in cases]
    grp = lib.Group(graphs)
    try:
        for G, O, r0 in cases:
            G.set_ranks(r0)
        stats = grp.update("dfp", max_iter=0)
        for (G, O, r0), st in zip(cases, stats):
            assert st.iterations == 0 and not st.converged
            assert np.array_equal(G.ranks(), r0)
        stats = grp.update("dfp", max_iter=3)
        for (G, O, r0), st in zip(cases, stats):
            assert st.iterations <= 3
            ref, _ = O.update("dfp", r_prev=r0, max_iter=3)
            assert np.max(np.abs(G.ranks() - ref)) < TOL
        # the graph whose batch was empty: F_0 is empty, one iteration, ranks kept
        G, O, r0 = cases[5]
        G.set_ranks(r0)
        st = grp.update("dfp")[5]
        assert st.iterations == 1 and st.converged and st.vertices_ever_affected == 0
        assert np.array_equal(G.ranks(), r0)
    finally:
        grp.close()


def test_group_successive_batches(lib):
    """Chained batches: batch, group DF-P, batch, group DF-P, ... on every
    graph.  Before each update the group's graphs and the solo graphs get the
    oracle's previous ranks (the previous snapshot's ranks are an input of
    Alg. 1, injected identically into both sides); the group's ranks equal the
    solo graphs' bit for bit and the oracle's within 1e-9, with the same
    iterations and vertices ever affected."""
    specs = [(10, 8, 50, 21), (12, 16, 200, 22), (8, 4, 10, 23)]
    pairs = []
    for scale, ef, _, seed in specs:
        n = 1 << scale
        src, dst = synth.rmat(scale, ef * n, seed)
        pairs.append((n, src, dst, lib.Graph.from_edges(n, src, dst), lib.Graph.from_edges(n, src, dst),
                      oracle.Graph(n, src, dst)))
    grp = lib.Group([p[3] for p in pairs])
    try:
        grp.update("static")
        r_cpu = []
        for n, src, dst, G, S, O in pairs:
            r, _ = O.update("static")
            r_cpu.append(r)
            S.update("static")
            assert np.array_equal(G.ranks(), S.ranks())
        for step in range(3):
            for k, ((n, src, dst, G, S, O), (_, _, bsize, seed)) in enumerate(zip(pairs, specs)):
                cs, cd = synth.unique_edges(src, dst)
                b = synth.batch(n, cs, cd, bsize, seed * 100 + step)
                for x in (G, S, O):
                    x.apply_batch(*b)
            for k, (n, src, dst, G, S, O) in enumerate(pairs):
                G.set_ranks(r_cpu[k])
                S.set_ranks(r_cpu[k])
            gst = grp.update("dfp")
            for k, (n, src, dst, G, S, O) in enumerate(pairs):
                S.update("dfp")
                r_cpu[k], ost = O.update("dfp", r_prev=r_cpu[k])
                assert np.array_equal(G.ranks(), S.ranks()), (step, k)
                assert np.max(np.abs(G.ranks() - r_cpu[k])) < 1e-9, (step, k)
                assert_same_run(gst[k], ost, (step, k))
    finally:
        grp.close()


def test_group_errors(lib):
    n = 64
    src, dst = synth.rmat(6, 256, 5)
    A = lib.Graph.from_edges(n, src, dst)
    B = lib.Graph.from_edges(n, src, dst)
    with pytest.raises(lib.PRError):
        lib.Group([A, A])
    with pytest.raises(lib.PRError):
        lib.Group([])
    grp = lib.Group([A, B])
    try:
        with pytest.raises(lib.PRError) as e:
            grp.update("dfp")               # no ranks yet
        assert e.value.status == 4
        with pytest.raises(lib.PRError):
            grp.update("dt")                # not offered for groups
        grp.update("static")
        grp.update("dfp")
    finally:
        grp.close()


@pytest.mark.parametrize("method", ["dfp", "df", "nd"])
def test_every_unit_size_gives_the_same_bits(lib, cases, method):
    """Gather units of 32 x 2/4/8 quads (or four steps of 32 x 2) and epilogue
    units of 1/2/4 chunks change only how the group's work is cut: ranks and
    statistics are bit-identical across all twelve settings (and to the oracle
    within 1e-9)."""
    graphs = [c[0] for c in cases]
    grp = lib.Group(graphs)
    try:
        out = []
        for q, k in ((2, 1), (4, 1), (8, 1), (2, 4)):
            for f in (1, 2, 4):
                grp.set_tuning(q, f, k)
                tu = grp.tuning()
                assert (tu.quads_per_lane, tu.steps_per_unit, tu.chunks_per_unit) == (q, k, f)
                for G, O, r0 in cases:
                    G.set_ranks(r0)
                for loop in ("device", "host"):
                    if loop == "host":
                        for G, O, r0 in cases:
                            G.set_ranks(r0)
                    st = grp.update(method, loop=loop)
                    out.append(([G.ranks() for G in graphs], [(s.iterations, s.vertices_processed) for s in st]))
        for ranks, its in out[1:]:
            assert all(np.array_equal(a, b) for a, b in zip(ranks, out[0][0]))
            assert its == out[0][1]
        for (G, O, r0), got in zip(cases, out[0][0]):
            ref, _ = O.update(method, r_prev=r0)
            assert np.max(np.abs(got - ref)) < TOL
    finally:
        grp.close()


def test_group_autotune_keeps_the_ranks(lib, cases):
    graphs = [c[0] for c in cases]
    for G, O, r0 in cases:
        G.set_ranks(r0)
    grp = lib.Group(graphs)
    try:
        tu = grp.autotune("dfp")
        assert tu.candidates == 12 and tu.ms_update > 0
        assert tu.quads_per_lane in (2, 4, 8) and tu.chunks_per_unit in (1, 2, 4)
        assert grp.tuning() == tu
        for G, O, r0 in cases:
            assert np.array_equal(G.ranks(), r0)
        st = grp.update("dfp")
        for (G, O, r0), s in zip(cases, st):
            ref, _ = O.update("dfp", r_prev=r0)
            assert np.max(np.abs(G.ranks() - ref)) < TOL
        for bad in ((3, 4, 1), (4, 3, 1), (16, 4, 1), (4, 8, 1), (4, 4, 4), (8, 4, 2)):
            with pytest.raises(lib.PRError):
                grp.set_tuning(*bad)
        assert grp.tuning() == tu
        with pytest.raises(lib.PRError):
            grp.autotune("dt")
    finally:
        grp.close()


def test_batches_of_many_graphs_at_once(lib):
    """pr_apply_batches_device and pr_apply_batches (host arrays) give every
    graph the edges, effective change and ranks that pr_apply_batch_device on
    each graph gives: small and large batches, an empty one, a graph with a
    repack; a batch with a bad id fails with PR_ERANGE and leaves only its own
    graph unchanged."""
    torch = pytest.importorskip("torch")
    specs = [(10, 8, 40), (12, 16, 3000), (11, 4, 0), (13, 16, 9000), (9, 8, 120)]
    trios, dev_batches, host_batches = [], [], []
    for k, (scale, ef, bsize) in enumerate(specs):
        n = 1 << scale
        src, dst = synth.rmat(scale, ef * n, 300 + k)
        trio = [lib.Graph.from_edges(n, src, dst) for _ in range(3)]
        for G in trio:
            G.update("static")
        cs, cd = synth.unique_edges(src, dst)
        b = synth.batch(n, cs, cd, bsize, 400 + k) if bsize else tuple(np.zeros(0, np.int32) for _ in range(4))
        if k == 4:   # overflow one row: a repack inside the multi-graph call
            b = (b[0], b[1], np.concatenate([b[2], np.full(300, 5, np.int32)]),
                 np.concatenate([b[3], np.arange(300, dtype=np.int32) % n]))
        b = tuple(np.ascontiguousarray(x, np.int32) for x in b)
        trios.append(trio)
        host_batches.append(b)
        dev_batches.append(tuple(torch.from_numpy(x).cuda() for x in b))
    lib.pr_apply_batches_device([t[0].handle for t in trios], dev_batches)
    lib.pr_apply_batches([t[2].handle for t in trios], host_batches)
    for (A, B, C), b in zip(trios, dev_batches):
        B.apply_batch_device(*b)
        for G in (A, C):
            for x, y in ((G.out_csr(), B.out_csr()), (G.in_csr(), B.in_csr())):
                assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
            assert all(np.array_equal(p, q) for p, q in zip(G.effective_delta(), B.effective_delta()))
    grp = lib.Group([t[0] for t in trios])
    try:
        st = grp.update("dfp")
    finally:
        grp.close()
    for (A, B, C), s in zip(trios, st):
        sb = B.update("dfp")
        sc = C.update("dfp")
        assert np.array_equal(A.ranks(), B.ranks()) and np.array_equal(C.ranks(), B.ranks())
        assert (s.iterations, s.vertices_processed) == (sb.iterations, sb.vertices_processed)
    # a bad id in one batch, host and device forms
    n0 = 1 << specs[0][0]
    for form in ("device", "host"):
        bad = (None, None, np.array([1, n0 + 5], np.int32), np.array([2, 3], np.int32))
        good = (None, None, np.array([7], np.int32), np.array([8], np.int32))
        if form == "device":
            bad = (None, None) + tuple(torch.from_numpy(x).cuda() for x in bad[2:])
            good = (None, None) + tuple(torch.from_numpy(x).cuda() for x in good[2:])
        G0, G1 = trios[0][0], trios[1][0]
        before = G0.out_csr()
        m0, m1 = G0.m, G1.m
        call = lib.pr_apply_batches_device if form == "device" else lib.pr_apply_batches
        with pytest.raises(lib.PRError) as e:
            call([G0.handle, G1.handle], [bad, good])
        assert e.value.status == 2
        after = G0.out_csr()
        assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1]) and G0.m == m0
        assert G1.m in (m1, m1 + 1)                    # the other graph's batch was applied


def test_batches_of_graphs_on_their_own_streams(lib):
    """Graphs on different streams: pr_apply_batches_device orders each graph's
    batch after the work already queued on the graph's stream and before the
    work queued after the call.  A rank import is queued on each stream just
    before the call, a rank export just after, and the applied edges, the
    effective change and the DF-P ranks equal those of the same graph applied
    alone."""
    torch = pytest.importorskip("torch")
    streams = [torch.cuda.Stream() for _ in range(3)]
    graphs, twins, batches, r0s = [], [], [], []
    for k, (scale, bsize) in enumerate([(11, 50), (12, 2500), (10, 9)]):
        n = 1 << scale
        src, dst = synth.rmat(scale, 8 * n, 500 + k)
        G = lib.Graph.from_edges(n, src, dst, stream=streams[k])
        T = lib.Graph.from_edges(n, src, dst)
        T.update("static")
        r0 = torch.from_numpy(T.ranks()).cuda()
        cs, cd = synth.unique_edges(src, dst)
        b = synth.batch(n, cs, cd, bsize, 600 + k)
        graphs.append(G)
        twins.append(T)
        batches.append(tuple(torch.from_numpy(np.ascontiguousarray(x, np.int32)).cuda() for x in b))
        r0s.append(r0)
    torch.cuda.synchronize()
    outs = []
    for G, r0, s in zip(graphs, r0s, streams):
        with torch.cuda.stream(s):
            G.set_ranks_device(r0)
    lib.pr_apply_batches_device([G.handle for G in graphs], batches)
    for G, r0, s in zip(graphs, r0s, streams):
        with torch.cuda.stream(s):
            out = torch.empty_like(r0)
            G.ranks_device(out)
            outs.append(out)
    torch.cuda.synchronize()
    for G, T, b, r0, out in zip(graphs, twins, batches, r0s, outs):
        assert torch.equal(out, r0)                    # the import landed before the batch, the export after
        T.apply_batch_device(*b)
        for x, y in ((G.out_csr(), T.out_csr()), (G.in_csr(), T.in_csr())):
            assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
        assert all(np.array_equal(p, q) for p, q in zip(G.effective_delta(), T.effective_delta()))
        sg_ = G.update("dfp")
        st_ = T.update("dfp")
        assert np.array_equal(G.ranks(), T.ranks())
        assert (sg_.iterations, sg_.vertices_processed) == (st_.iterations, st_.vertices_processed)


def test_group_at_the_batched_workload_sizes(lib):
    """The batched configuration's graph sizes (R-MAT scales 12 .. 21, edge
    factors 8 .. 32, one 80/20 batch of 1e-4 |E| each): one group DF-P update
    of ten graphs spanning that range equals, graph by graph, the oracle's
    DF-P from the same previous ranks within 1e-9, with the same decisions of
    Alg. 1."""
    specs = [(12, 8), (13, 32), (14, 16), (15, 24), (16, 8), (17, 32), (18, 12), (19, 20), (20, 16), (21, 8)]
    graphs, refs = [], []
    for k, (scale, ef) in enumerate(specs):
        n = 1 << scale
        src, dst = synth.rmat(scale, ef * n, 7000 + k)
        G = lib.Graph.from_edges(n, src, dst)
        O = oracle.Graph(n, src, dst, parallel=True)
        r0, _ = O.update("static")
        cs, cd = synth.unique_edges(src, dst)
        b = synth.batch(n, cs, cd, max(1, int(round(1e-4 * O.m))), 7100 + k)
        G.apply_batch(*b)
        O.apply_batch(*b)
        G.set_ranks(r0)
        graphs.append(G)
        refs.append(O.update("dfp", r_prev=r0))
    grp = lib.Group(graphs)
    try:
        stats = grp.update("dfp")
    finally:
        grp.close()
    for k, (G, (ref, ost)) in enumerate(zip(graphs, refs)):
        assert np.max(np.abs(G.ranks() - ref)) < TOL, specs[k]
        assert_same_run(stats[k], ost, specs[k])
