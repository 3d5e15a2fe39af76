"""Parity at full size: R-MAT scale 25, edge factor 32 (2^25 vertices, about
5.4e8 edges with the self-loops), one random batch of 1e-4 |E| edges (80%
insertions), run through the same entry points and launch configuration as
the benchmark step.  The whole DF-P update is compared with the oracle's
(its OpenMP build, about a minute); the other checks are (a) sampled outputs
that the oracle computes one by one from rows
exported by the library (Eq. 1 and Eq. 2 for single vertices), (b) exact
integer checks of sampled rows against set semantics (Sec. 3.2) and of the
initial marking (Alg. 1) on sampled vertices, and (c) properties that hold at
any size (mass, convergence, untouched vertices keep their ranks bitwise,
push and pull forms agree bitwise).

Tolerances of the one-sweep checks come from the arithmetic: the library sums
contributions R[u]/|out(u)| rounded to 2^-61 fixed point (at most 2^-62 error
per in-neighbour), then evaluates Eq. 1 or Eq. 2 in FP64; the oracle sums in
FP64.  So |library - oracle| <= f * alpha * (deg_in + 1) * 2^-61 + 8 ulp, with
f = 1 for Eq. 1 and f = 1 / (1 - alpha/d) <= 1/(1 - alpha) for Eq. 2.
"""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

SCALE, EDGE_FACTOR, BATCH_FRAC, SEED = 25, 32, 1e-4, 1
ALPHA, TAU, TAU_F, TAU_P = 0.85, 1e-10, 1e-6, 1e-6
N_RANDOM, N_TOUCHED, N_HUBS = 400, 200, 8


def in_sums(rows, outdeg_of, r):
    """c_v = sum over u in in(v) of r[u] / |out(u)|, exactly rounded (fsum)."""
    off, adj = rows
    c = np.empty(len(off) - 1)
    for k in range(len(off) - 1):
        u = adj[off[k]:off[k + 1]]
        c[k] = math.fsum((r[u] / outdeg_of(u)).tolist())
    return c


class Snapshot:
    """Rows and degrees of sampled vertices in one graph snapshot."""

    def __init__(self, G, sample, extra_out):
        self.sample = sample
        self.in_rows = G.rows(1, sample)
        self.out_rows = G.rows(0, extra_out)
        self.out_vertices = extra_out
        nb = np.unique(self.in_rows[1])
        deg = np.diff(G.rows(0, nb, degrees_only=True))
        self._nb, self._deg = nb, deg
        self.own_deg = np.diff(G.rows(0, sample, degrees_only=True))

    def outdeg_of(self, u):
        return self._deg[np.searchsorted(self._nb, u)]

    def row(self, which, v):
        off, adj = self.in_rows if which == 1 else self.out_rows
        verts = self.sample if which == 1 else self.out_vertices
        k = int(np.nonzero(verts == v)[0][0])
        return adj[off[k]:off[k + 1]]


@pytest.fixture(scope="module")
def full():
    import torch

    import paper_2401_15870_gb300 as pr
    import synth.gpu as sg

    pr.load()
    sg.build()
    n = 1 << SCALE
    src, dst = sg.rmat(SCALE, EDGE_FACTOR << SCALE, SEED)
    G = pr.Graph.from_edges(n, src, dst, device=True)
    m0 = G.m
    size = max(1, int(round(BATCH_FRAC * m0)))
    batch = sg.batch(n, src, dst, size, SEED + 1)
    torch.cuda.synchronize()
    del src, dst
    host_batch = [t.cpu().numpy() for t in batch]

    st_static = G.update("static", alpha=ALPHA, tau=TAU)
    r_prev = G.ranks()

    rng = np.random.default_rng(12345)
    ds, dd, is_, id_ = host_batch
    bsrc = np.unique(np.concatenate([ds, is_]))
    bdst = np.unique(np.concatenate([dd, id_]))
    hubs = np.argsort(r_prev)[-N_HUBS:].astype(np.int32)
    sample = np.unique(np.concatenate([rng.integers(0, n, N_RANDOM), hubs,
                                       rng.choice(bdst, min(N_TOUCHED, bdst.size), replace=False)])).astype(np.int32)
    touched_src = rng.choice(bsrc, min(N_TOUCHED, bsrc.size), replace=False).astype(np.int32)
    out_sample = np.unique(np.concatenate([touched_src, rng.integers(0, n, N_RANDOM)])).astype(np.int32)

    before = Snapshot(G, sample, out_sample)
    G.apply_batch_device(*batch)
    torch.cuda.synchronize()
    after = Snapshot(G, sample, out_sample)
    dm, dp = G.effective_delta()
    yield dict(pr=pr, G=G, n=n, m0=m0, batch=host_batch, st_static=st_static, r_prev=r_prev, sample=sample,
               out_sample=out_sample, before=before, after=after, dm=dm, dp=dp, hubs=hubs)
    G.close()


def test_static_solution_full_size(full):
    """Static from 1/n: converged within tau; mass 1 (self-loops, no dead ends);
    on sampled vertices the residual of Eq. 1 is within the bound a last change
    of at most tau allows: |r - T(r)|_v <= alpha * tau * sum_u 1/|out(u)|."""
    st, r, n = full["st_static"], full["r_prev"], full["n"]
    assert st.converged and st.delta_R <= TAU
    assert abs(float(np.sum(r)) - 1.0) < 1e-9
    assert np.all(r > 0)
    snap = full["before"]
    c = in_sums(snap.in_rows, snap.outdeg_of, r)
    off, adj = snap.in_rows
    for k, v in enumerate(snap.sample):
        u = adj[off[k]:off[k + 1]]
        assert v in u                                         # self-loop (Sec. 5.1.3)
        expect = oracle.rank_plain(ALPHA, n, c[k])
        bound = (ALPHA * TAU * float(np.sum(1.0 / snap.outdeg_of(u))) + ALPHA * (u.size + 1) * 2.0 ** -61
                 + 8 * np.spacing(expect))
        assert abs(r[v] - expect) <= bound, (v, r[v], expect, bound)


def expected_rows(old_rows, verts, dels, inss):
    """(old, new) row sets under E_t = (E_{t-1} minus D) united with I, the
    self-loops kept; dels / inss are (key, other endpoint) arrays."""
    out = {}
    for k, v in enumerate(verts):
        old = set(old_rows[1][old_rows[0][k]:old_rows[0][k + 1]].tolist())
        d = set(dels[1][dels[0] == v].tolist()) - {v}
        i = set(inss[1][inss[0] == v].tolist())
        out[v] = (old, (old - d) | i)
    return out


def test_batch_edit_full_size(full):
    """Sampled rows after the batch are exactly the set-semantics rows, out and
    in, and the effective change restricted to them is exactly new - old and
    old - new (Sec. 3.2); the edge count moves by |Delta+| - |Delta-|."""
    G, before, after = full["G"], full["before"], full["after"]
    ds, dd, is_, id_ = full["batch"]
    dm, dp = full["dm"], full["dp"]
    assert G.m == full["m0"] - len(dm) + len(dp)
    for which, verts, old_rows, new_rows, dels, inss, dmk, dpk in (
            (0, before.out_vertices, before.out_rows, after.out_rows, (ds, dd), (is_, id_), (dm[:, 0], dm[:, 1]),
             (dp[:, 0], dp[:, 1])),
            (1, before.sample, before.in_rows, after.in_rows, (dd, ds), (id_, is_), (dm[:, 1], dm[:, 0]),
             (dp[:, 1], dp[:, 0]))):
        exp = expected_rows(old_rows, verts, dels, inss)
        off, adj = new_rows
        for k, v in enumerate(verts):
            got = adj[off[k]:off[k + 1]]
            old, new = exp[v]
            assert np.all(np.diff(got) > 0)
            assert set(got.tolist()) == new, (which, v)
            assert set(dmk[1][dmk[0] == v].tolist()) == old - new, (which, v)
            assert set(dpk[1][dpk[0] == v].tolist()) == new - old, (which, v)


def test_initial_marking_full_size(full):
    """Alg. 1's initial marking on sampled vertices: v is marked exactly when
    some in-neighbour in G_{t-1} or G_t is the source of an effective change."""
    G, before, after = full["G"], full["before"], full["after"]
    A = G.initial_affected()
    srcs = np.unique(np.concatenate([full["dm"][:, 0], full["dp"][:, 0]]))
    assert srcs.size > 0 and A.sum() > 0
    for v in before.sample:
        nb = np.union1d(before.row(1, v), after.row(1, v))
        assert A[v] == bool(np.intersect1d(nb, srcs).size), v
    # a marked vertex is an out-neighbour of a changed source, so the count is
    # at most the sources' degree total
    deg = np.diff(G.rows(0, srcs, degrees_only=True))
    assert A.sum() <= int(deg.sum()) + len(full["dm"])


def one_sweep_bound(in_deg, closed):
    f = 1.0 / (1.0 - ALPHA) if closed else 1.0
    return f * ALPHA * (in_deg + 1) * 2.0 ** -61


def test_one_sweep_parity_full_size(full):
    """One synchronous sweep at full size, element by element on sampled
    vertices against the oracle's Eq. 1 (Naive-dynamic from R_{t-1}) and Eq. 2
    (DF-P's first sweep, pull and push forms); every vertex outside the
    initial marking keeps R_{t-1} bitwise, and the two forms agree bitwise."""
    G, snap, r_prev, n = full["G"], full["after"], full["r_prev"], full["n"]
    c = in_sums(snap.in_rows, snap.outdeg_of, r_prev)
    ideg = np.diff(snap.in_rows[0])
    A = G.initial_affected()

    G.set_ranks(r_prev)
    G.update("nd", alpha=ALPHA, tau=TAU, max_iter=1)
    r1 = G.ranks()
    for k, v in enumerate(snap.sample):
        expect = oracle.rank_plain(ALPHA, n, c[k])
        assert abs(r1[v] - expect) <= one_sweep_bound(ideg[k], False) + 8 * np.spacing(expect), v

    got = {}
    for direction in ("pull", "push"):
        G.set_ranks(r_prev)
        st = G.update("dfp", alpha=ALPHA, tau=TAU, tau_f=TAU_F, tau_p=TAU_P, max_iter=1, direction=direction)
        assert st.iterations == 1
        assert st.vertices_processed == int(A.sum())
        r1 = G.ranks()
        assert np.array_equal(r1[~A], r_prev[~A])
        for k, v in enumerate(snap.sample):
            if not A[v]:
                continue
            expect = oracle.rank_closed_loop(ALPHA, n, c[k], r_prev[v], int(snap.own_deg[k]))
            assert abs(r1[v] - expect) <= one_sweep_bound(ideg[k], True) + 8 * np.spacing(expect), (direction, v)
        got[direction] = r1
    assert np.array_equal(got["pull"], got["push"])


def test_dfp_full_run_full_size(full):
    """The whole DF-P update as the benchmark runs it: converged; vertices
    outside the Dynamic Traversal set keep R_{t-1} bitwise; the pull form, the
    push form and the per-iteration choice give bit-identical ranks; and the
    ranks stay within the soft-error bound 10 tau_p / (1 - alpha) of a Static
    solve of G_t."""
    G, r_prev = full["G"], full["r_prev"]
    DT = G.dt_affected()
    res = {}
    for direction in (None, "pull", "push"):
        G.set_ranks(r_prev)
        st = G.update("dfp", alpha=ALPHA, tau=TAU, tau_f=TAU_F, tau_p=TAU_P, direction=direction)
        assert st.converged and st.delta_R <= TAU
        assert st.vertices_ever_affected <= int(DT.sum())
        res[direction] = (G.ranks(), st)
    r = res[None][0]
    assert np.array_equal(r[~DT], r_prev[~DT])
    for d in ("pull", "push"):
        assert np.array_equal(res[d][0], r), d
        assert res[d][1].iterations == res[None][1].iterations
        assert res[d][1].vertices_ever_affected == res[None][1].vertices_ever_affected
    G.update("static", alpha=ALPHA, tau=TAU)
    r_static = G.ranks()
    assert np.max(np.abs(r - r_static)) < 10 * TAU_P / (1 - ALPHA)
    assert abs(float(np.sum(r)) - 1.0) < 1e-5          # sanity: pruning moves little mass


def test_dfp_whole_graph_matches_the_oracle(full):
    """The whole DF-P update at full size against the oracle element by
    element (Alg. 1, Eq. 2): the oracle (its OpenMP build, the same bits as
    the single-threaded one) builds G_{t-1} from the same drawn edges, both
    sides take the same R_{t-1} (the library's Static ranks) and the same
    batch; every rank within 1e-9, with the oracle's iterations, vertices ever
    affected and vertex updates unless the oracle reports a near-tie."""
    import synth.gpu as sg
    from cases import assert_same_run
    G, n, r_prev = full["G"], full["n"], full["r_prev"]
    src, dst = sg.rmat(SCALE, EDGE_FACTOR << SCALE, SEED)
    src_h, dst_h = src.cpu().numpy(), dst.cpu().numpy()
    del src, dst
    O = oracle.Graph(n, src_h, dst_h, parallel=True)
    del src_h, dst_h
    O.apply_batch(*full["batch"])
    G.set_ranks(r_prev)
    st = G.update("dfp", alpha=ALPHA, tau=TAU, tau_f=TAU_F, tau_p=TAU_P)
    ref, ost = O.update("dfp", alpha=ALPHA, tau=TAU, tau_f=TAU_F, tau_p=TAU_P, r_prev=r_prev)
    del O
    assert np.max(np.abs(G.ranks() - ref)) < 1e-9
    assert_same_run(st, ost, "full size")


def test_dt_full_run_full_size(full):
    """Dynamic Traversal at full size: its affected set (reachable from the
    changed sources in G_{t-1} or G_t) holds most in-edges here, so the
    automatic choice sweeps every row and updates the members; the list form
    gives the same bits.  Converged; every vertex outside the set keeps
    R_{t-1} bitwise; on sampled members the residual of Eq. 1 is within the
    bound a last change of at most tau allows (as for Static)."""
    G, r_prev, n = full["G"], full["r_prev"], full["n"]
    DT = G.dt_affected()
    res = {}
    for direction in (None, "push"):
        G.set_ranks(r_prev)
        st = G.update("dt", alpha=ALPHA, tau=TAU, direction=direction)
        assert st.converged and st.delta_R <= TAU
        assert st.vertices_ever_affected == int(DT.sum())
        res[direction] = (G.ranks(), st)
    r, st = res[None]
    assert np.array_equal(res["push"][0], r)
    assert (res["push"][1].iterations, res["push"][1].edges_processed) == (st.iterations, st.edges_processed)
    assert np.array_equal(r[~DT], r_prev[~DT])
    snap = full["after"]
    c = in_sums(snap.in_rows, snap.outdeg_of, r)
    off, adj = snap.in_rows
    checked = 0
    for k, v in enumerate(snap.sample):
        if not DT[v]:
            continue
        u = adj[off[k]:off[k + 1]]
        expect = oracle.rank_plain(ALPHA, n, c[k])
        bound = (ALPHA * TAU * float(np.sum(1.0 / snap.outdeg_of(u))) + ALPHA * (u.size + 1) * 2.0 ** -61
                 + 8 * np.spacing(expect))
        assert abs(r[v] - expect) <= bound, (v, r[v], expect, bound)
        checked += 1
    assert checked > 0
