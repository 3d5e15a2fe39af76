"""Parity of the CUDA library with the CPU oracle, element by element.

Integer work (CSR build, batch edit, effective change, affected sets) must be
bit-exact; ranks must agree within 1e-9 in L-infinity (the tolerance the
target states), for every method, from the same previous ranks.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-9
from cases import TIE_REL, assert_same_run  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    import paper_2401_15870_gb300 as pr
    pr.load()
    return pr


def make_pair(pr, n, src, dst, keep_order=False):
    return pr.Graph.from_edges(n, src, dst, keep_order=keep_order), oracle.Graph(n, src, dst)


def assert_same_graph(G, O):
    for mine, ref in ((G.out_csr(), O.out_csr()), (G.in_csr(), O.in_csr())):
        assert np.array_equal(mine[0], ref[0])
        assert np.array_equal(mine[1], ref[1])


# ------------------------------------------------------------- integer parity


@pytest.mark.parametrize("keep_order", [False, True])
@pytest.mark.parametrize("scale,m", [(1, 3), (5, 40), (10, 1 << 13), (14, 1 << 18)])
def test_build_matches_oracle(lib, scale, m, keep_order):
    n = 1 << scale
    src, dst = synth.rmat(scale, m, 100 + scale)
    G, O = make_pair(lib, n, src, dst, keep_order)
    assert G.m == O.m
    assert_same_graph(G, O)


def test_build_from_csr_and_ragged_sizes(lib):
    for n, m, seed in ((1, 0, 1), (3, 5, 2), (37, 300, 3), (1000, 7001, 4)):
        rng = np.random.default_rng(seed)
        s = np.sort(rng.integers(0, n, m)).astype(np.int32)
        d = rng.integers(0, n, m).astype(np.int32)
        off = np.zeros(n + 1, np.int64)
        np.add.at(off, s + 1, 1)
        off = np.cumsum(off)
        G = lib.Graph.from_csr(n, off, d)
        O = oracle.Graph(n, s, d)
        assert_same_graph(G, O)


def batches(n, src, dst, count, size, seed):
    cs, cd = synth.unique_edges(src, dst)
    out = []
    for i in range(count):
        ds, dd, is_, id_ = synth.batch(n, cs, cd, size, seed + i)
        # repeats, self-loops, a missing-edge deletion, an edge deleted and re-inserted
        if len(ds):
            ds = np.concatenate([ds, ds[:1], [3 % n], [(7 * i) % n]]).astype(np.int32)
            dd = np.concatenate([dd, dd[:1], [3 % n], [(11 * i + 1) % n]]).astype(np.int32)
            is_ = np.concatenate([is_, is_[:1], [5 % n], ds[:1]]).astype(np.int32)
            id_ = np.concatenate([id_, id_[:1], [5 % n], dd[:1]]).astype(np.int32)
        out.append((ds, dd, is_, id_))
    return out


@pytest.mark.parametrize("scale,size", [(6, 20), (10, 300), (14, 262), (12, 4000), (14, 20000)])
def test_batch_edit_matches_oracle(lib, scale, size):
    """Batches up to 4096 edges take the one-block ingest path, larger ones the
    multi-kernel path; both must be bit-exact."""
    n = 1 << scale
    src, dst = synth.rmat(scale, 16 * n, 200 + scale)
    G, O = make_pair(lib, n, src, dst)
    for b in batches(n, src, dst, 4, size, 300):
        G.apply_batch(*b)
        O.apply_batch(*b)
        gd, gp = G.effective_delta()
        od, op = O.effective_delta()
        assert np.array_equal(gd, od) and np.array_equal(gp, op)
        assert G.m == O.m
        assert_same_graph(G, O)


def test_small_batch_on_hub_rows(lib):
    """A small batch touching rows longer than the small path's first staging
    buffer (64K elements): the device skips the direction, the host grows the
    buffer and finishes it."""
    n = 1 << 18
    rng = np.random.default_rng(3)
    hub_out = np.arange(1, 150001, dtype=np.int32)
    src = np.concatenate([np.zeros(hub_out.size, np.int32), hub_out, rng.integers(0, n, 50000).astype(np.int32)])
    dst = np.concatenate([hub_out, np.zeros(hub_out.size, np.int32), rng.integers(0, n, 50000).astype(np.int32)])
    G, O = make_pair(lib, n, src, dst)
    G.update("static")
    r0 = G.ranks()
    b = (np.array([0, 5, 7], np.int32), np.array([10, 0, 0], np.int32),
         np.array([0, 200000, 0], np.int32), np.array([200001, 0, 5], np.int32))
    G.apply_batch(*b)
    O.apply_batch(*b)
    assert_same_graph(G, O)
    dm, dp = G.effective_delta()
    odm, odp = O.effective_delta()
    assert np.array_equal(dm, odm) and np.array_equal(dp, odp)
    G.set_ranks(r0)
    G.update("dfp")
    ref, _ = O.update("dfp", r_prev=r0)
    assert np.max(np.abs(G.ranks() - ref)) < TOL


def test_batch_overflow_repacks(lib):
    """Insertions that overflow a row's slack force a rebuild of that direction."""
    n = 512
    src, dst = synth.rmat(9, 4000, 7)
    G, O = make_pair(lib, n, src, dst)
    hub_ins_s = np.full(300, 17, np.int32)
    hub_ins_d = np.arange(300, dtype=np.int32) * 1 % n
    tgt_ins_s = np.arange(300, dtype=np.int32) % n
    tgt_ins_d = np.full(300, 99, np.int32)
    for b in ((hub_ins_s, hub_ins_d), (tgt_ins_s, tgt_ins_d)):
        G.apply_batch(ins_src=b[0], ins_dst=b[1])
        O.apply_batch(ins_src=b[0], ins_dst=b[1])
        assert_same_graph(G, O)
    # and deleting them again
    G.apply_batch(del_src=hub_ins_s, del_dst=hub_ins_d)
    O.apply_batch(del_src=hub_ins_s, del_dst=hub_ins_d)
    assert_same_graph(G, O)


def test_repack_spreads_hub_rows_and_matches_oracle(lib):
    """A batch that overflows rows of more than 16384 edges (an out-hub and an
    in-hub, with deletions and insertions in them) and rows of every other
    length: the repack splits the hub rows over many blocks, the short rows
    over single threads and the rest over warps; both CSRs equal the oracle's
    exactly and the DF-P ranks after it are within 1e-9."""
    n = 50000
    rng = np.random.default_rng(91)
    hub_out = rng.choice(np.arange(3, n), 30000, replace=False)      # 1 -> 30000 targets
    hub_in = rng.choice(np.arange(3, n), 30000, replace=False)       # 30000 sources -> 2
    mid_s = rng.integers(0, n, 200000)
    mid_d = rng.integers(0, n, 200000)
    src = np.concatenate([np.full(30000, 1), hub_in, mid_s]).astype(np.int32)
    dst = np.concatenate([hub_out, np.full(30000, 2), mid_d]).astype(np.int32)
    G, O = make_pair(lib, n, src, dst)
    r0, _ = O.update("static")
    free_out = np.setdiff1d(np.arange(3, n), hub_out)[:6000]
    free_in = np.setdiff1d(np.arange(3, n), hub_in)[:6000]
    ins_s = np.concatenate([np.full(6000, 1), free_in, rng.integers(0, n, 5000)]).astype(np.int32)
    ins_d = np.concatenate([free_out, np.full(6000, 2), rng.integers(0, n, 5000)]).astype(np.int32)
    del_s = np.concatenate([np.full(700, 1), hub_in[:700], mid_s[:900]]).astype(np.int32)
    del_d = np.concatenate([hub_out[:700], np.full(700, 2), mid_d[:900]]).astype(np.int32)
    G.apply_batch(del_s, del_d, ins_s, ins_d)
    O.apply_batch(del_s, del_d, ins_s, ins_d)
    assert_same_graph(G, O)
    G.set_ranks(r0)
    G.update("dfp")
    ref, _ = O.update("dfp", r_prev=r0)
    assert np.max(np.abs(G.ranks() - ref)) < TOL
    # the repacked graph takes further batches in place
    b = batches(n, src, dst, 1, 3000, 93)[0]
    G.apply_batch(*b)
    O.apply_batch(*b)
    assert_same_graph(G, O)


def test_batch_out_of_range_changes_nothing(lib):
    n = 64
    src, dst = synth.rmat(6, 300, 9)
    G, O = make_pair(lib, n, src, dst)
    with pytest.raises(lib.PRError) as e:
        G.apply_batch(ins_src=[1, 64], ins_dst=[2, 3])
    assert e.value.status == 2
    assert_same_graph(G, O)


@pytest.mark.parametrize("seed", range(3))
def test_affected_sets_match_oracle(lib, seed):
    n = 1 << 11
    src, dst = synth.rmat(11, 8 * n, 400 + seed)
    G, O = make_pair(lib, n, src, dst)
    b = batches(n, src, dst, 1, 5 + 20 * seed, 500 + seed)[0]
    G.apply_batch(*b)
    O.apply_batch(*b)
    assert np.array_equal(G.initial_affected(), O.initial_affected())
    assert np.array_equal(G.dt_affected(), O.dt_affected())


# -------------------------------------------------------------- rank parity


def rank_case(lib, scale, ef, bsize, seed, keep_order=False):
    n = 1 << scale
    src, dst = synth.rmat(scale, ef * n, seed)
    G, O = make_pair(lib, n, src, dst, keep_order)
    r0, _ = O.update("static")
    b = batches(n, src, dst, 1, bsize, seed + 1)[0]
    G.apply_batch(*b)
    O.apply_batch(*b)
    return G, O, r0


@pytest.mark.parametrize("method", ["static", "nd", "dt", "df", "dfp"])
def test_ranks_tiny_config(lib, method):
    """R-MAT 2^14 vertices, 2^18 edges, one batch of 1e-3 |E| (80/20)."""
    G, O, r0 = rank_case(lib, 14, 16, 262, 11)
    G.set_ranks(r0)
    st = G.update(method)
    ref, ost = O.update(method, r_prev=r0)
    got = G.ranks()
    assert np.max(np.abs(got - ref)) < TOL
    assert st.converged and ost.converged
    assert_same_run(st, ost, method)


@pytest.mark.parametrize("method", ["static", "nd", "dt", "df", "dfp"])
@pytest.mark.parametrize("scale,ef,bsize,keep", [(4, 3, 4, False), (9, 8, 50, True), (12, 24, 400, False)])
def test_ranks_ragged_and_small(lib, method, scale, ef, bsize, keep):
    G, O, r0 = rank_case(lib, scale, ef, bsize, 20 + scale, keep)
    G.set_ranks(r0)
    st = G.update(method)
    ref, ost = O.update(method, r_prev=r0)
    assert np.max(np.abs(G.ranks() - ref)) < TOL
    assert_same_run(st, ost, method)


def test_ranks_with_hub_rows_spanning_many_tiles(lib):
    """A vertex with ~20000 in-edges spans several 4096-slot tiles, so its sum
    is assembled from partial sums of different thread blocks."""
    n = 30000
    rng = np.random.default_rng(5)
    src = np.concatenate([np.arange(n), rng.integers(0, n, 60000)]).astype(np.int32)
    dst = np.concatenate([np.full(n, 7), rng.integers(0, n, 60000)]).astype(np.int32)
    src = np.concatenate([src, np.full(20000, 3)]).astype(np.int32)     # out-hub too
    dst = np.concatenate([dst, rng.integers(0, n, 20000)]).astype(np.int32)
    G, O = make_pair(lib, n, src, dst)
    for method in ("static",):
        G.update(method)
        ref, _ = O.update(method)
        assert np.max(np.abs(G.ranks() - ref)) < TOL
    r0 = ref
    b = (np.array([3, 11], np.int32), np.array([int(dst[-1]), 7], np.int32),
         np.array([7, 100, 3], np.int32), np.array([3, 7, 8], np.int32))
    G.apply_batch(*b)
    O.apply_batch(*b)
    for method in ("nd", "dt", "df", "dfp"):
        G.set_ranks(r0)
        G.update(method)
        ref, _ = O.update(method, r_prev=r0)
        assert np.max(np.abs(G.ranks() - ref)) < TOL, method


@pytest.mark.parametrize("direction", ["pull", "push", None])
@pytest.mark.parametrize("method", ["df", "dfp", "dt"])
@pytest.mark.parametrize("scale,bsize", [(12, 40), (14, 262), (13, 3000)])
def test_frontier_directions_agree_with_oracle(lib, method, direction, scale, bsize):
    """Pull sweeps (every vertex, membership test), push sweeps (frontier lists)
    and the automatic choice give the oracle's ranks and processed sets (DT:
    its affected set swept as a list or as the members of every-row sweeps)."""
    G, O, r0 = rank_case(lib, scale, 16, bsize, 50 + scale)
    G.set_ranks(r0)
    st = G.update(method, direction=direction)
    ref, ost = O.update(method, r_prev=r0)
    assert np.max(np.abs(G.ranks() - ref)) < TOL
    assert_same_run(st, ost, (method, direction))


@pytest.mark.parametrize("method", ["static", "nd", "df", "dfp"])
@pytest.mark.parametrize("scale,bsize", [(12, 40), (14, 262), (13, 3000)])
def test_device_and_host_loops_agree_bitwise(lib, method, scale, bsize):
    """The iteration loop on the device (CUDA graph, pull form), in one
    cooperative kernel and on the host give bit-identical ranks and
    statistics."""
    G, O, r0 = rank_case(lib, scale, 16, bsize, 70 + scale)
    out = []
    for loop in ("device", "one", "host"):
        G.set_ranks(r0)
        st = G.update(method, loop=loop)
        out.append((G.ranks(), st.iterations, st.converged, st.vertices_ever_affected, st.vertices_processed,
                    st.edges_processed))
    for o in out[1:]:
        assert np.array_equal(out[0][0], o[0])
        assert out[0][1:] == o[1:]
    ref, ost = O.update(method, r_prev=r0)
    assert np.max(np.abs(out[0][0] - ref)) < TOL
    assert (out[0][1], out[0][3], out[0][4]) == (ost.iterations, ost.vertices_ever_affected,
                                                 ost.vertices_processed) or ost.tie_rel < TIE_REL


@pytest.mark.parametrize("method", ["df", "dfp", "dt"])
@pytest.mark.parametrize("scale,bsize", [(12, 40), (14, 262), (13, 3000)])
def test_frontier_directions_agree_bitwise(lib, method, scale, bsize):
    """Both sweep forms sum the same fixed-point contributions exactly and
    evaluate Eq. 1 / Eq. 2 with the same roundings, so the direction taken in
    each iteration changes neither the ranks nor the frontier: pull, push and
    the automatic choice give bit-identical ranks and statistics."""
    G, O, r0 = rank_case(lib, scale, 16, bsize, 50 + scale)
    out = []
    for direction in ("pull", "push", None):
        G.set_ranks(r0)
        st = G.update(method, direction=direction)
        out.append((G.ranks(), st.iterations, st.vertices_ever_affected, st.vertices_processed,
                    st.edges_processed if method == "dt" else 0))
    for r, *rest in out[1:]:
        assert np.array_equal(r, out[0][0])
        assert tuple(rest) == out[0][1:]


def test_successive_batches_and_methods_from_same_ranks(lib):
    n = 1 << 12
    src, dst = synth.rmat(12, 16 * n, 77)
    G, O = make_pair(lib, n, src, dst)
    G.update("static")
    r_gpu = G.ranks()
    r_cpu, _ = O.update("static")
    for i, b in enumerate(batches(n, src, dst, 3, 120, 900)):
        G.apply_batch(*b)
        O.apply_batch(*b)
        for method in ("dfp", "df", "dt", "nd"):
            G.set_ranks(r_cpu)
            st = G.update(method)
            ref, ost = O.update(method, r_prev=r_cpu)
            assert np.max(np.abs(G.ranks() - ref)) < TOL, (i, method)
            assert_same_run(st, ost, (i, method))
        # chain DF-P results on both sides
        G.set_ranks(r_cpu)
        G.update("dfp")
        r_cpu, _ = O.update("dfp", r_prev=r_cpu)


def test_empty_batch_and_edge_cases(lib):
    n = 256
    src, dst = synth.rmat(8, 2000, 3)
    G, O = make_pair(lib, n, src, dst)
    r0, _ = O.update("static")
    G.set_ranks(r0)
    G.apply_batch()
    for method in ("df", "dfp", "dt"):
        G.set_ranks(r0)
        st = G.update(method)
        assert st.iterations == 1 and st.delta_R == 0.0 and st.vertices_ever_affected == 0
        assert np.array_equal(G.ranks(), r0)
    # max_iter = 0 leaves the ranks as set
    G.set_ranks(r0)
    st = G.update("nd", max_iter=0)
    assert st.iterations == 0 and not st.converged
    assert np.array_equal(G.ranks(), r0)
    # a single vertex
    one = lib.Graph.from_edges(1, [], [])
    one.update("static")
    assert one.ranks()[0] == pytest.approx(1.0, abs=1e-15)


def test_dynamic_method_without_ranks_is_rejected(lib):
    G = lib.Graph.from_edges(8, [0, 1], [1, 2])
    with pytest.raises(lib.PRError) as e:
        G.update("dfp")
    assert e.value.status == 4


def test_set_ranks_validation(lib):
    G = lib.Graph.from_edges(4, [0, 1], [1, 2])
    with pytest.raises(lib.PRError):
        G.set_ranks([0.5, -0.1, 0.3, 0.3])
    with pytest.raises(lib.PRError):
        G.set_ranks([1.0, 1.0, 1.0, 1.0])
    G.set_ranks([0.25] * 4)


def test_device_pointer_entry_points(lib):
    torch = pytest.importorskip("torch")
    n = 1 << 10
    src, dst = synth.rmat(10, 8 * n, 12)
    O = oracle.Graph(n, src, dst)
    G = lib.Graph.from_edges(n, torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), device=True)
    assert_same_graph(G, O)
    r0, _ = O.update("static")
    G.set_ranks_device(torch.from_numpy(r0).cuda())
    b = batches(n, src, dst, 1, 40, 13)[0]
    O.apply_batch(*b)
    G.apply_batch_device(*[torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in b])
    assert_same_graph(G, O)
    G.update("dfp")
    ref, _ = O.update("dfp", r_prev=r0)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    G.ranks_device(out)
    assert np.max(np.abs(out.cpu().numpy() - ref)) < TOL


def test_deterministic_across_runs(lib):
    """Fixed-point sums make repeated runs bitwise identical."""
    G, O, r0 = rank_case(lib, 13, 16, 200, 31)
    outs = []
    for _ in range(3):
        G.set_ranks(r0)
        G.update("dfp")
        outs.append(G.ranks())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])


# ------------------------------------------------------------- gather settings (pr_autotune)

SETTINGS = [(256, 4, 0, 0, 1), (256, 4, 0, 1, 1), (1024, 4, 27648, 1, 1), (512, 2, 13824, 0, 1),
            (256, 8, 3072, 1, 1), (1024, 8, 100, 0, 1), (512, 4, 1, 1, 1), (1024, 2, 6656, 1, 1), (512, 8, 0, 1, 1),
            (1024, 2, 0, 0, 1), (512, 4, 0, 0, 2), (256, 4, 0, 0, 4), (1024, 2, 3072, 0, 4), (256, 8, 0, 0, 2),
            (1024, 2, 0, 0, 8)]


@pytest.mark.parametrize("method,direction", [("static", None), ("nd", None), ("df", "pull"), ("dfp", "pull")])
@pytest.mark.parametrize("scale,bsize", [(12, 40), (14, 262)])
def test_every_gather_setting_gives_the_same_bits(lib, method, direction, scale, bsize):
    """Threads per block, quads per lane, the hub staged in shared memory
    (none, a ragged count, a count above n that covers every vertex and the
    sentinel), the epilogue inside or after the gather kernel and the sweep cut
    into vertex ranges on two streams change only the schedule of exact integer
    sums: ranks and statistics are bit-identical across settings, and within
    1e-9 of the oracle."""
    G, O, r0 = rank_case(lib, scale, 16, bsize, 90 + scale)
    out = []
    for t, q, hub, fused, ranges in SETTINGS:
        G.set_tuning(t, q, hub, fused, ranges)
        tu = G.tuning()
        assert (tu.threads, tu.quads_per_lane, tu.hub_vertices, tu.fused_epilogue, tu.ranges) == \
            (t, q, min(hub, G.n), fused, ranges)
        G.set_ranks(r0)
        st = G.update(method, direction=direction, loop="host")
        out.append((G.ranks(), st.iterations, st.vertices_ever_affected, st.vertices_processed, st.edges_processed))
    for r, *rest in out[1:]:
        assert np.array_equal(r, out[0][0])
        assert rest == list(out[0][1:])
    ref, _ = O.update(method, r_prev=r0)
    assert np.max(np.abs(out[0][0] - ref)) < TOL


def test_autotune_on_sweeps_keeps_the_graph_and_the_results(lib):
    G, O, r0 = rank_case(lib, 14, 16, 262, 97)
    G.set_ranks(r0)
    st0 = G.update("dfp", direction="pull", loop="host")
    r_default = G.ranks()
    tu = G.autotune("nd", reps=2)
    assert np.array_equal(G.ranks(), r_default)          # the trials leave the ranks as they were
    assert tu.threads in (256, 512, 1024) and tu.quads_per_lane in (2, 4, 8)
    assert 0 <= tu.hub_vertices <= G.n and tu.candidates >= 18 and tu.ms_gather > 0
    assert tu.fused_epilogue in (0, 1)
    # the staged hub is every vertex of out-degree >= hub_min_degree
    if tu.hub_vertices:
        deg = np.diff(G.rows(0, np.arange(G.n, dtype=np.int32), degrees_only=True))
        assert tu.hub_min_degree >= 1
        assert np.sum(deg > tu.hub_min_degree) <= tu.hub_vertices <= np.sum(deg >= tu.hub_min_degree)
    assert G.tuning() == tu
    G.set_ranks(r0)
    st1 = G.update("dfp", direction="pull", loop="host")
    assert np.array_equal(G.ranks(), r_default)
    assert (st1.iterations, st1.vertices_processed) == (st0.iterations, st0.vertices_processed)


@pytest.mark.parametrize("method", ["df", "dfp"])
@pytest.mark.parametrize("scale", [13, 12])
def test_autotune_on_updates_keeps_the_ranks(lib, method, scale):
    """Tuning on whole updates runs them from the entry ranks with the last
    batch and puts those ranks back; a graph small enough for the device loop
    also gets its one-graph group tuned.  The update that follows, with the
    device loop or the host loop, equals the oracle's."""
    G, O, r0 = rank_case(lib, scale, 16, 200, 98)
    G.set_ranks(r0)
    tu = G.autotune(method)
    assert tu.candidates >= 18
    assert np.array_equal(G.ranks(), r0)
    ref, _ = O.update(method, r_prev=r0)
    for loop in ("device", "one", "host"):
        G.set_ranks(r0)
        G.update(method, loop=loop)
        assert np.max(np.abs(G.ranks() - ref)) < TOL
    with pytest.raises(lib.PRError):
        G.autotune("dt")


def test_invalid_gather_settings_are_rejected(lib):
    G, _, _ = rank_case(lib, 10, 8, 20, 5)
    before = G.tuning()
    # a hub of 40000 vertices is above n here, but no block's shared memory holds it
    for t, q, hub, f, r in ((128, 4, 0, 1, 1), (256, 3, 0, 1, 1), (256, 4, -1, 1, 1), (256, 4, 40000, 1, 1),
                            (2048, 4, 0, 1, 1), (256, 4, 0, 2, 1), (256, 4, 0, 1, 2), (256, 4, 0, 0, 3),
                            (256, 4, 0, 0, 0)):
        with pytest.raises(lib.PRError):
            G.set_tuning(t, q, hub, f, r)
    assert G.tuning() == before


# ------------------------------------------------------------- frontier measures of Sec. 4.3


@pytest.mark.parametrize("measure,tol_f", [("absolute", 1e-12), ("contrib", 1e-13), ("relative", 1e-5)])
@pytest.mark.parametrize("method", ["df", "dfp"])
@pytest.mark.parametrize("scale,bsize", [(12, 40), (14, 262)])
def test_frontier_measures_match_oracle_in_every_form(lib, measure, tol_f, method, scale, bsize):
    """DF / DF-P with each measure of Sec. 4.3 (rank change, change of the
    contribution factor, relative change) against the oracle with the same
    measure, within 1e-9; pull, push, the automatic choice, the device loop
    and a group give bit-identical ranks and statistics."""
    G, O, r0 = rank_case(lib, scale, 16, bsize, 110 + scale)
    ref, ost = O.update(method, tau_f=tol_f, tau_p=tol_f, r_prev=r0, metric=measure)
    out, first = [], None
    for direction, loop in (("pull", "host"), ("push", "host"), (None, "host"), (None, "device")):
        G.set_ranks(r0)
        st = G.update(method, tau_f=tol_f, tau_p=tol_f, direction=direction, loop=loop, measure=measure)
        out.append((G.ranks(), st.iterations, st.vertices_ever_affected, st.vertices_processed))
        first = first or st
    G.set_ranks(r0)
    grp = lib.Group([G])
    try:
        st = grp.update(method, tau_f=tol_f, tau_p=tol_f, measure=measure)[0]
        out.append((G.ranks(), st.iterations, st.vertices_ever_affected, st.vertices_processed))
    finally:
        grp.close()
    for r, *rest in out[1:]:
        assert np.array_equal(r, out[0][0])
        assert rest == list(out[0][1:])
    assert np.max(np.abs(out[0][0] - ref)) < TOL
    assert_same_run(first, ost, measure)


def test_measure_flags_are_exclusive(lib):
    G, _, r0 = rank_case(lib, 10, 8, 20, 5)
    G.set_ranks(r0)
    import ctypes
    opts = lib.pr_options(1e-6, 1e-6, 500, 32 | 64)
    assert lib.load().pr_update(G.handle, 4, 0.85, 1e-10, ctypes.byref(opts), None) == 1
    # the measures change the frontier, not Eq. 1 / Eq. 2: ND ignores them
    a = G.update("nd", measure="absolute")
    ra = G.ranks()
    G.set_ranks(r0)
    b = G.update("nd")
    assert np.array_equal(ra, G.ranks()) and a.iterations == b.iterations


@pytest.mark.parametrize("method", ["df", "dfp"])
@pytest.mark.parametrize("direction", ["pull", "push", None])
def test_frontier_without_expansion_matches_oracle(lib, method, direction):
    """tau_f = inf, tau_p = 0: only the initially affected set is swept, every
    other vertex keeps R_{t-1} bitwise (the case the oracle pins to the linear
    system restricted to that set)."""
    G, O, r0 = rank_case(lib, 12, 16, 40, 91)
    G.set_ranks(r0)
    st = G.update(method, tau_f=float("inf"), tau_p=0.0, direction=direction)
    ref, ost = O.update(method, tau_f=float("inf"), tau_p=0.0, r_prev=r0)
    A = G.initial_affected()
    got = G.ranks()
    assert np.max(np.abs(got - ref)) < TOL
    assert np.array_equal(got[~A], r0[~A])
    assert st.vertices_ever_affected == ost.vertices_ever_affected == int(A.sum())


# ------------------------------------------------------------- prune against re-mark (reading C2)


@pytest.mark.parametrize("direction,loop", [("pull", "host"), ("push", "host"), (None, "device"), (None, "one")])
def test_pruned_vertex_re_marked_matches_oracle(lib, direction, loop):
    """The hand-made case of tests/golden/prune_vs_mark_6v.txt: vertex 2 is
    pruned in iteration 0 while its in-neighbour 1 expands into it, so it is
    swept again in iteration 1 (F_1 = M_0 u (F_0 \\ P_0) = {1, 2, 3}).  Every
    sweep form gives the oracle's ranks and the same vertex updates after
    one, two and three iterations."""
    from cases import load_prune_vs_mark, prune_vs_mark_case
    edges, _ = load_prune_vs_mark()
    O, r, meta = prune_vs_mark_case()
    G = lib.Graph.from_edges(6, [a for a, _ in edges], [b for _, b in edges])
    G.apply_batch(ins_src=[meta["insert"][0]], ins_dst=[meta["insert"][1]])
    for k in (1, 2, 3):
        G.set_ranks(r)
        st = G.update("dfp", tau=0.0, max_iter=k, direction=direction, loop=loop)
        ref, ost = O.update("dfp", tau=0.0, max_iter=k, r_prev=r)
        assert np.max(np.abs(G.ranks() - ref)) < TOL, k
        assert (st.vertices_processed, st.vertices_ever_affected) == (ost.vertices_processed,
                                                                      ost.vertices_ever_affected), k
    assert ost.vertices_processed >= meta["processed_after2"][0]
