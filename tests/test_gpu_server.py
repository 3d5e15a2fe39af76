"""The request loop (pr_server_*): every result must be the same alone and in
the mix.  Grouped mode merges the requests of a graph that queue up (per edge
the last operation wins) and updates many graphs in one group update; the test
rebuilds each round's merged batch from the request records with its own merge,
replays the rounds on a separate copy of the graph with plain pr_apply_batch +
pr_update, and requires bit-identical ranks, and ranks within 1e-9 of the
oracle's DF-P from the same previous ranks at every round."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def lib():
    import paper_2401_15870_gb300 as pr
    pr.load()
    return pr


SPECS = [(10, 8, 31), (12, 16, 32), (9, 4, 33), (13, 8, 34)]


def build(pr, specs):
    """Server copies, replay copies and oracle graphs, all at static ranks."""
    out = []
    for scale, ef, seed in specs:
        n = 1 << scale
        src, dst = synth.rmat(scale, ef * n, seed)
        A = pr.Graph.from_edges(n, src, dst)
        B = pr.Graph.from_edges(n, src, dst)
        O = oracle.Graph(n, src, dst, parallel=scale >= 18)
        A.update("static")
        B.set_ranks(A.ranks())
        out.append(dict(n=n, src=src, dst=dst, A=A, B=B, O=O, r0=A.ranks()))
    return out


def make_requests(cases, count, seed, max_size=300):
    """Random requests, with repeated edges across requests of a graph so that
    merging has to resolve insert-then-delete and delete-then-insert."""
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        g = int(rng.integers(0, len(cases)))
        c = cases[g]
        cs, cd = synth.unique_edges(c["src"], c["dst"])
        ds, dd, is_, id_ = synth.batch(c["n"], cs, cd, int(rng.integers(1, max_size)), seed * 1000 + i)
        if reqs and rng.random() < 0.5:
            # undo or redo some edges of an earlier request of the same graph
            prev = [r for r in reqs if r[0] == g]
            if prev:
                _, pds, pdd, pis, pid = prev[-1]
                k = min(5, len(pis))
                ds = np.concatenate([ds, pis[:k]]).astype(np.int32)
                dd = np.concatenate([dd, pid[:k]]).astype(np.int32)
                k = min(5, len(pds))
                is_ = np.concatenate([is_, pds[:k]]).astype(np.int32)
                id_ = np.concatenate([id_, pdd[:k]]).astype(np.int32)
        reqs.append((g, ds, dd, is_, id_))
    return reqs


def merge(batches):
    """Per edge the last operation wins; a request's deletions before its insertions."""
    last = {}
    for ds, dd, is_, id_ in batches:
        for u, v in zip(ds.tolist(), dd.tolist()):
            last[(u, v)] = 0
        for u, v in zip(is_.tolist(), id_.tolist()):
            last[(u, v)] = 1
    d = [e for e, op in last.items() if op == 0]
    i = [e for e, op in last.items() if op == 1]
    arr = lambda es, k: np.array([e[k] for e in es], np.int32)
    return arr(d, 0), arr(d, 1), arr(i, 0), arr(i, 1)


def replay(cases, reqs, infos):
    """Rounds of every graph in order, each merged batch applied to the replay
    copy and the oracle; DF-P on both from the replay copy's previous ranks."""
    by = {}
    for (g, *b), info in zip(reqs, infos):
        assert info.graph == g and info.status == 0
        by.setdefault((g, info.round), []).append((info.ticket, b))
    for (g, rnd) in sorted(by, key=lambda k: (k[0], k[1])):
        items = sorted(by[(g, rnd)], key=lambda t: t[0])
        for t, _ in items:
            assert infos[t].merged == len(items)
        b = merge([bb for _, bb in items])
        c = cases[g]
        r_prev = c["B"].ranks()
        c["B"].apply_batch(*b)
        c["O"].apply_batch(*b)
        c["B"].update("dfp")
        ref, _ = c["O"].update("dfp", r_prev=r_prev)
        assert np.max(np.abs(c["B"].ranks() - ref)) < TOL, (g, rnd)
    return by


def run_server(lib, cases, reqs, **kw):
    srv = lib.Server([c["A"] for c in cases], **kw)
    try:
        tickets = [srv.submit(g, ds, dd, is_, id_) for g, ds, dd, is_, id_ in reqs]
        assert tickets == list(range(len(reqs)))
        srv.drain(300)
        infos = [srv.wait(t, 10) for t in tickets]
    finally:
        srv.close()
    return infos


def test_grouped_server_equals_replay_alone(lib):
    cases = build(lib, SPECS)
    reqs = make_requests(cases, 60, 5)
    infos = run_server(lib, cases, reqs, mode="grouped")
    by = replay(cases, reqs, infos)
    assert max(i.merged for i in infos) > 1                      # requests were coalesced
    assert len({i.round for i in infos}) < len({k for k in by})   # and graphs shared rounds
    for c in cases:
        assert np.array_equal(c["A"].ranks(), c["B"].ranks())
    for i in infos:
        assert i.t_submit <= i.t_start <= i.t_done
        assert i.stats.iterations >= 1


def test_plain_server_equals_sequential(lib):
    cases = build(lib, SPECS[:2])
    reqs = make_requests(cases, 20, 6)
    infos = run_server(lib, cases, reqs, mode="plain")
    assert all(i.merged == 1 for i in infos)
    assert sorted(i.round for i in infos) == list(range(len(reqs)))
    replay(cases, reqs, infos)
    for c in cases:
        assert np.array_equal(c["A"].ranks(), c["B"].ranks())


def test_admission_by_free_memory(lib):
    """A reserve larger than the device: every round admits only its first
    graph, and the results are still those of the replay."""
    cases = build(lib, SPECS[:3])
    reqs = make_requests(cases, 24, 7)
    infos = run_server(lib, cases, reqs, mode="grouped", hbm_reserve=1 << 60)
    graphs_of_round = {}
    for i in infos:
        graphs_of_round.setdefault(i.round, set()).add(i.graph)
    assert all(len(v) == 1 for v in graphs_of_round.values())
    replay(cases, reqs, infos)
    for c in cases:
        assert np.array_equal(c["A"].ranks(), c["B"].ranks())


def test_server_errors(lib):
    n = 256
    src, dst = synth.rmat(8, 1024, 3)
    G = lib.Graph.from_edges(n, src, dst)
    with pytest.raises(lib.PRError) as e:
        lib.Server([G])                              # no ranks yet
    assert e.value.status == 4
    G.update("static")
    srv = lib.Server([G])
    try:
        with pytest.raises(lib.PRError) as e:
            srv.submit(0, [1], [n])                  # id out of range
        assert e.value.status == 2
        with pytest.raises(lib.PRError):
            srv.submit(1, [1], [2])                  # no graph 1
        with pytest.raises(lib.PRError):
            srv.wait(5, 0.1)                         # never issued
        t = srv.submit(0, [], [], [1, 2], [3, 4])
        info = srv.wait(t, 60)
        assert info.status == 0 and info.stats.eff_insertions <= 2
    finally:
        srv.close()
    G.update("dfp")                                  # the graph is usable again afterwards


def test_large_graph_is_served_beside_group_updates(lib):
    """A graph of at least PR_DEVICE_LOOP_SLOTS in-CSR slots is updated by the
    server's solo thread (pr_update, one large graph after another) while the
    small graphs go through group updates; every round still equals its
    replay with plain calls bit for bit and the oracle's DF-P within 1e-9."""
    cases = build(lib, [(20, 16, 41), (10, 8, 42), (12, 16, 43)])
    reqs = make_requests(cases, 30, 8, max_size=2000)
    infos = run_server(lib, cases, reqs, mode="grouped")
    by = replay(cases, reqs, infos)
    big_rounds = {i.round for i in infos if i.graph == 0}
    small_rounds = {i.round for i in infos if i.graph != 0}
    assert not (big_rounds & small_rounds)               # the large graph never joins a group update
    for c in cases:
        assert np.array_equal(c["A"].ranks(), c["B"].ranks())
