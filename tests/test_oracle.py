"""Pins for the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the linear
system whose solution is the PageRank fixed point (numpy's LAPACK solver),
closed forms, conservation laws, the appendix's geometric series, brute-force
reachability and set arithmetic, and the worked example of Sec. 4.1.3.
"""
import os

import numpy as np
import pytest

import oracle
import synth

ALPHA = 0.85
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def edge_set(n, src, dst):
    """Edge set with one self-loop per vertex, as Python tuples."""
    e = {(int(u), int(v)) for u, v in zip(src, dst)}
    e |= {(v, v) for v in range(n)}
    return e


def pagerank_solve(n, edges, alpha=ALPHA):
    """Solve (I - alpha P^T) r = (1-alpha)/n 1 with P[u][w] = 1/|out(u)| (Eq. 1 at its fixed point)."""
    outdeg = np.zeros(n)
    for u, _ in edges:
        outdeg[u] += 1
    A = np.eye(n)
    for u, w in edges:
        A[w, u] -= alpha / outdeg[u]
    return np.linalg.solve(A, np.full(n, (1 - alpha) / n))


def random_graph(n, m, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, n, m), rng.integers(0, n, m)


def random_batch(n, edges, nd, ni, seed, with_noise=True):
    """Deletions of existing edges, uniform insertions, plus repeats, self-loops,
    missing-edge deletions and edges both deleted and inserted."""
    rng = np.random.default_rng(seed)
    ex = sorted(e for e in edges if e[0] != e[1])
    dels = [ex[i] for i in rng.integers(0, len(ex), nd)] if ex and nd else []
    ins = [(int(a), int(b)) for a, b in zip(rng.integers(0, n, ni), rng.integers(0, n, ni))]
    if with_noise:
        dels += [dels[0]] if dels else []
        dels += [(0, 0), (int(rng.integers(0, n)), int(rng.integers(0, n)))]
        ins += [ins[0]] if ins else []
        ins += [(1 % n, 1 % n)]
        if dels:
            ins += [dels[-1]]
    split = lambda lst: (np.array([a for a, _ in lst], np.int32), np.array([b for _, b in lst], np.int32))
    return split(dels), split(ins)


# ---------------------------------------------------------------- fixed point


@pytest.mark.parametrize("n,m,seed", [(1, 0, 0), (2, 1, 1), (7, 12, 2), (40, 160, 3), (120, 900, 4), (200, 400, 5)])
def test_static_matches_linear_solve(n, m, seed):
    src, dst = random_graph(n, m, seed)
    g = oracle.Graph(n, src, dst)
    r, st = g.update("static", tau=1e-15, max_iter=5000)
    ref = pagerank_solve(n, edge_set(n, src, dst))
    assert st.converged
    assert np.max(np.abs(r - ref)) < 1e-12


@pytest.mark.parametrize("method", ["nd", "dfp_zero", "df_zero"])
def test_nd_and_zero_tolerance_frontiers_reach_fixed_point(method):
    """ND from any start, and DF / DF-P with tau_f = tau_p = 0 (no pruning of a
    changing vertex, expansion on any change), reach the fixed point of G_t."""
    n = 150
    src, dst = random_graph(n, 700, 11)
    g = oracle.Graph(n, src, dst)
    E0 = edge_set(n, src, dst)
    r0 = pagerank_solve(n, E0)
    (ds, dd), (is_, id_) = random_batch(n, E0, 10, 40, 12)
    g.apply_batch(ds, dd, is_, id_)
    E1 = (E0 - {(int(a), int(b)) for a, b in zip(ds, dd) if a != b}) | {(int(a), int(b)) for a, b in zip(is_, id_)}
    ref = pagerank_solve(n, E1)
    if method == "nd":
        r, st = g.update("nd", tau=1e-15, max_iter=5000, r_prev=np.random.default_rng(0).random(n))
    else:
        r, st = g.update(method[:-5], tau=1e-15, tau_f=0.0, tau_p=0.0, max_iter=5000, r_prev=r0)
    assert st.converged
    assert np.max(np.abs(r - ref)) < 1e-12


def test_dt_reaches_fixed_point_and_leaves_others_bitwise():
    n = 160
    src, dst = random_graph(n, 260, 21)
    E0 = edge_set(n, src, dst)
    g = oracle.Graph(n, src, dst)
    r0 = pagerank_solve(n, E0)
    (ds, dd), (is_, id_) = random_batch(n, E0, 3, 5, 22)
    g.apply_batch(ds, dd, is_, id_)
    E1 = (E0 - {(int(a), int(b)) for a, b in zip(ds, dd) if a != b}) | {(int(a), int(b)) for a, b in zip(is_, id_)}
    r, st = g.update("dt", tau=1e-15, max_iter=5000, r_prev=r0)
    A = g.dt_affected()
    assert np.max(np.abs(r - pagerank_solve(n, E1))) < 1e-12
    assert np.array_equal(r[~A], r0[~A])
    assert st.vertices_ever_affected == A.sum()


# ---------------------------------------------------------------- closed forms


@pytest.mark.parametrize("method", ["static", "nd", "dfp", "df"])
@pytest.mark.parametrize("kind", ["cycle", "complete"])
def test_uniform_closed_forms(kind, method):
    """A directed cycle and a complete digraph, each with self-loops, have
    uniform PageRank 1/n: every vertex receives alpha/n in total from
    in-neighbours of equal rank and out-degree."""
    n = 37
    if kind == "cycle":
        src, dst = np.arange(n), (np.arange(n) + 1) % n
    else:
        src, dst = np.repeat(np.arange(n), n), np.tile(np.arange(n), n)
    g = oracle.Graph(n, src, dst)
    if method == "static":
        r, st = g.update("static")
        assert st.iterations == 1
    else:
        # 1/n is the fixed point: ND changes nothing beyond rounding, and a batch
        # that re-inserts an existing edge marks nothing for DF / DF-P
        g.apply_batch(ins_src=[0], ins_dst=[1])
        r, st = g.update(method, r_prev=np.full(n, 1.0 / n))
        assert st.iterations == 1 and st.delta_R < 1e-15
        if method != "nd":
            assert st.delta_R == 0.0 and st.vertices_ever_affected == 0
    assert np.max(np.abs(r - 1.0 / n)) < 1e-15


def test_mass_conservation_static_nd():
    """With a self-loop on every vertex there are no dead ends, so a Jacobi step
    of Eq. 1 maps a vector of sum 1 to a vector of sum 1."""
    src, dst = synth.rmat(10, 1 << 14, 5)
    g = oracle.Graph(1 << 10, src, dst)
    r, _ = g.update("static")
    assert abs(r.sum() - 1.0) < 1e-12
    cs, cd = synth.unique_edges(src, dst)
    g.apply_batch(*synth.batch(1 << 10, cs, cd, 100, 6))
    r2, _ = g.update("nd", r_prev=r)
    assert abs(r2.sum() - 1.0) < 1e-12


# ------------------------------------------------------- Eq. 2 and appendix


@pytest.mark.parametrize("d,c_ex,r0", [(1, 0.0, 0.5), (2, 1e-3, 1e-4), (7, 3.3e-6, 2e-6), (1000, 0.2, 0.01)])
def test_closed_loop_equals_repeated_self_update(d, c_ex, r0):
    """Appendix: repeating the standard update r <- alpha (c + r/d) + C0 with the
    in-neighbours frozen converges to the closed-loop value of Eq. 2."""
    n = 1000
    C0 = (1 - ALPHA) / n
    r = r0
    for _ in range(10000):
        r = ALPHA * (c_ex + r / d) + C0
    closed = oracle.rank_closed_loop(ALPHA, n, c_ex + r0 / d, r0, d)
    assert abs(closed - r) <= 1e-14 * abs(r)
    assert oracle.rank_plain(ALPHA, n, c_ex) == pytest.approx(C0 + ALPHA * c_ex, rel=0, abs=0)


# ------------------------------------------------------------ batch semantics


@pytest.mark.parametrize("seed", range(6))
def test_batch_effective_delta_is_set_difference(seed):
    n = 30
    src, dst = random_graph(n, 90, 100 + seed)
    E0 = edge_set(n, src, dst)
    g = oracle.Graph(n, src, dst)
    (ds, dd), (is_, id_) = random_batch(n, E0, 8, 12, 200 + seed)
    g.apply_batch(ds, dd, is_, id_)
    D = {(int(a), int(b)) for a, b in zip(ds, dd) if a != b}
    I = {(int(a), int(b)) for a, b in zip(is_, id_)}
    E1 = (E0 - D) | I
    dm, dp = g.effective_delta()
    assert {tuple(x) for x in dm.tolist()} == E0 - E1
    assert {tuple(x) for x in dp.tolist()} == E1 - E0
    off, adj = g.out_csr()
    got = {(u, int(adj[j])) for u in range(n) for j in range(off[u], off[u + 1])}
    assert got == E1
    ioff, iadj = g.in_csr()
    got_in = {(int(iadj[j]), v) for v in range(n) for j in range(ioff[v], ioff[v + 1])}
    assert got_in == E1
    for u in range(n):
        assert list(adj[off[u]:off[u + 1]]) == sorted(adj[off[u]:off[u + 1]])


def test_batch_rejects_out_of_range_and_leaves_graph():
    g = oracle.Graph(5, [0, 1], [1, 2])
    before = g.out_csr()
    with pytest.raises(oracle.OracleError):
        g.apply_batch(ins_src=[0, 5], ins_dst=[1, 1])
    with pytest.raises(oracle.OracleError):
        g.apply_batch(del_src=[-1], del_dst=[1])
    after = g.out_csr()
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])


# ------------------------------------------------------- affected-set pins


def reach(n, edges, sources):
    """Brute force: boolean transitive closure by repeated squaring."""
    M = np.zeros((n, n), bool)
    for u, v in edges:
        M[u, v] = True
    M |= np.eye(n, dtype=bool)
    while True:
        M2 = (M.astype(np.int32) @ M.astype(np.int32)) > 0
        if np.array_equal(M2, M):
            break
        M = M2
    out = np.zeros(n, bool)
    for s in sources:
        out |= M[s]
    return out


@pytest.mark.parametrize("seed", range(5))
def test_marking_and_dt_against_brute_force(seed):
    n = 40
    src, dst = random_graph(n, 70, 300 + seed)
    E0 = edge_set(n, src, dst)
    g = oracle.Graph(n, src, dst)
    (ds, dd), (is_, id_) = random_batch(n, E0, 3, 4, 400 + seed)
    g.apply_batch(ds, dd, is_, id_)
    D = {(int(a), int(b)) for a, b in zip(ds, dd) if a != b}
    E1 = (E0 - D) | {(int(a), int(b)) for a, b in zip(is_, id_)}
    S = {u for u, _ in (E0 - E1) | (E1 - E0)}
    init = np.zeros(n, bool)
    for u, v in E0 | E1:
        if u in S:
            init[v] = True
    assert np.array_equal(g.initial_affected(), init)
    assert np.array_equal(g.dt_affected(), reach(n, E0, S) | reach(n, E1, S))


def load_worked_example():
    edges, meta, cur = [], {}, None
    with open(os.path.join(GOLDEN, "worked_example_16v.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            if line == "edges":
                cur = "edges"
                continue
            if line == "end":
                cur = None
                continue
            if cur == "edges":
                a, b = line.split()
                edges.append((int(a) - 1, int(b) - 1))
            else:
                k, *vals = line.split()
                meta[k] = [int(x) - 1 for x in vals]
    return edges, meta


def test_worked_example_sec_4_1_3():
    """The 16-vertex example of Sec. 4.1.3.  The oracle adds self-loops, so the
    initial marking also contains the two sources 2 and 4 (their self-loops are
    out-edges); the narrated set is the marking without them."""
    edges, meta = load_worked_example()
    n = 16
    assert len(edges) == 23
    g = oracle.Graph(n, [a for a, _ in edges], [b for _, b in edges])
    g.apply_batch(del_src=[meta["delete"][0]], del_dst=[meta["delete"][1]],
                  ins_src=[meta["insert"][0]], ins_dst=[meta["insert"][1]])
    f0 = set(np.flatnonzero(g.initial_affected()).tolist())
    assert f0 - {1, 3} == set(meta["initial"])
    assert {1, 3} <= f0
    off, adj = g.out_csr()
    for k in ("1", "2"):
        marked = set()
        for v in meta["expanders" + k]:
            marked |= {int(w) for w in adj[off[v]:off[v + 1]] if w != v}
        assert marked == set(meta["marked" + k])
    dt = g.dt_affected()
    assert set(np.flatnonzero(~dt).tolist()) == set(meta["dt_unaffected"])


# ------------------------------------------------------------ DF invariants


def test_df_invariants_and_empty_batch():
    src, dst = synth.rmat(10, 1 << 13, 31)
    n = 1 << 10
    g = oracle.Graph(n, src, dst)
    r0, _ = g.update("static")
    g.apply_batch()                      # empty batch
    for m in ("df", "dfp", "dt"):
        r, st = g.update(m, r_prev=r0)
        assert np.array_equal(r, r0) and st.iterations == 1 and st.delta_R == 0.0
        assert st.vertices_ever_affected == 0
    cs, cd = synth.unique_edges(src, dst)
    g.apply_batch(*synth.batch(n, cs, cd, 20, 32))
    r_df, st = g.update("df", r_prev=r0)
    # vertices never marked keep R_{t-1} bitwise; DF's frontier only grows, so
    # a vertex outside the DT reachability set is never marked
    dt = g.dt_affected()
    assert np.array_equal(r_df[~dt], r0[~dt])
    assert st.vertices_ever_affected <= dt.sum()
    assert st.converged
    r_dfp, st_p = g.update("dfp", r_prev=r0)
    assert np.array_equal(r_dfp[~dt], r0[~dt])
    assert st_p.converged and st_p.edges_processed <= st.edges_processed


def test_dynamic_methods_require_previous_ranks():
    g = oracle.Graph(4, [0], [1])
    with pytest.raises(oracle.OracleError):
        g.update("df")


def test_error_ordering_soft_claim():
    """Sec. 5.2.1: DF error lies below Static's at the same tau and ND's below
    DF's (errors are L1 against a tightly converged static solve, Sec. 5.1.5).
    DF-P's error is governed by its relative prune tolerance: it stays within a
    small multiple of tau_p / (1 - alpha).  The paper's DF-P-below-Static
    ordering needs graphs large enough that tau = 1e-10 (absolute) is loose
    relative to the ranks; at this size it is not asserted (the paper itself
    reports DF-P above Static on web graphs, Sec. 5.2.2)."""
    n = 1 << 11
    src, dst = synth.rmat(11, 1 << 15, 41)
    g = oracle.Graph(n, src, dst)
    r0, _ = g.update("static")
    cs, cd = synth.unique_edges(src, dst)
    g.apply_batch(*synth.batch(n, cs, cd, 30, 42))
    ref, _ = g.update("static", tau=1e-100, max_iter=500)
    err = {m: np.abs(g.update(m, r_prev=r0)[0] - ref).sum() for m in ("static", "nd", "df", "dfp")}
    assert err["df"] < err["static"]
    assert err["nd"] <= err["df"] * 1.0001
    assert err["dfp"] < 10 * 1e-6 / (1 - ALPHA)


# ---------------------------------------------------------------- Sec. 4.3 measures, asynchronous order


@pytest.mark.parametrize("metric", ["relative", "absolute", "contrib"])
@pytest.mark.parametrize("order", ["sync", "async"])
@pytest.mark.parametrize("method", ["df", "dfp"])
def test_every_measure_and_order_reaches_fixed_point_at_zero_tolerance(metric, order, method):
    """With tau_f = tau_p = 0 every measure expands on any change and prunes
    nothing that changes, in either order, so DF and DF-P reach the fixed
    point of G_t (the linear solve)."""
    n = 150
    src, dst = random_graph(n, 700, 31)
    g = oracle.Graph(n, src, dst)
    E0 = edge_set(n, src, dst)
    r0 = pagerank_solve(n, E0)
    (ds, dd), (is_, id_) = random_batch(n, E0, 10, 40, 32)
    g.apply_batch(ds, dd, is_, id_)
    E1 = (E0 - {(int(a), int(b)) for a, b in zip(ds, dd) if a != b}) | {(int(a), int(b)) for a, b in zip(is_, id_)}
    r, st = g.update(method, tau=1e-15, tau_f=0.0, tau_p=0.0, max_iter=5000, r_prev=r0, metric=metric, order=order)
    assert st.converged
    assert np.max(np.abs(r - pagerank_solve(n, E1))) < 1e-12


@pytest.mark.parametrize("method", ["static", "nd"])
def test_async_sweeps_reach_fixed_point(method):
    """Gauss-Seidel sweeps (one rank vector, ascending id) converge to the
    same linear-system solution as the synchronous ones.  (Not necessarily in
    fewer sweeps: on a well-mixing random graph the power iteration's error
    shrinks by about alpha |lambda_2| per sweep, with nothing along the Perron
    vector, and beats Gauss-Seidel; the DAG test below shows the opposite.)"""
    n = 120
    src, dst = random_graph(n, 900, 41)
    g = oracle.Graph(n, src, dst)
    ref = pagerank_solve(n, edge_set(n, src, dst))
    start = np.full(n, 1.0 / n) if method == "nd" else None
    ra, sa = g.update(method, tau=1e-15, max_iter=5000, r_prev=start, order="async")
    assert sa.converged and np.max(np.abs(ra - ref)) < 1e-12


def test_async_closed_loop_solves_a_dag_in_one_sweep():
    """On a graph whose edges all go from a lower to a higher id (plus the
    self-loops), Eq. 2 visited in ascending id reads only final in-neighbour
    ranks and removes the self term exactly: one asynchronous DF-P sweep over
    every vertex gives the fixed point, and the second one only confirms it.
    The synchronous order needs one sweep per level of the DAG at least."""
    n = 60
    rng = np.random.default_rng(51)
    u = rng.integers(0, n - 1, 200)
    v = u + 1 + (rng.integers(0, n, 200) % (n - 1 - u))
    g = oracle.Graph(n, u, v)
    E0 = edge_set(n, u, v)
    r0 = pagerank_solve(n, E0)
    # insert (k, k+1) for every k: every vertex becomes a source, so all are marked
    ins = [(k, k + 1) for k in range(n - 1) if (k, k + 1) not in E0]
    ins += [(0, 1)] if not ins else []
    g.apply_batch([], [], [a for a, _ in ins], [b for _, b in ins])
    E1 = E0 | set(ins)
    ref = pagerank_solve(n, E1)
    assert g.initial_affected().all()
    r1, s1 = g.update("dfp", tau=1e-14, tau_f=0.0, tau_p=0.0, max_iter=1, r_prev=r0, order="async")
    assert np.max(np.abs(r1 - ref)) < 1e-14
    r2, s2 = g.update("dfp", tau=1e-14, tau_f=0.0, tau_p=0.0, max_iter=50, r_prev=r0, order="async")
    assert s2.converged and s2.iterations == 2
    _, s3 = g.update("dfp", tau=1e-14, tau_f=0.0, tau_p=0.0, max_iter=500, r_prev=r0, order="sync")
    assert s3.iterations > 2


def test_contribution_measure_on_constant_out_degree():
    """dr / d > tau_f with every out-degree equal to d is dr > d * tau_f: on
    such a graph DF with the contribution measure at tau_f takes the same steps
    as DF with the rank-change measure at d * tau_f (tau_f a power of two,
    so both thresholds are exact)."""
    n, k = 300, 6   # out-degree k with the self-loop
    rng = np.random.default_rng(61)
    src, dst = [], []
    for a in range(n):
        others = rng.choice(np.delete(np.arange(n), a), k - 1, replace=False)
        src += [a] * (k - 1)
        dst += list(others)
    g = oracle.Graph(n, src, dst)
    off, _ = g.out_csr()
    assert np.all(np.diff(off) == k)
    r0, _ = g.update("static", tau=1e-14)
    # a batch that keeps every out-degree at k: move one edge of each of a few sources
    E = edge_set(n, src, dst)
    dels, ins = [], []
    for a in rng.choice(n, 8, replace=False):
        old = next(w for (x, w) in sorted(E) if x == a and w != a)
        new = next(w for w in rng.permutation(n) if w != a and (int(a), int(w)) not in E)
        dels.append((int(a), int(old)))
        ins.append((int(a), int(new)))
    g.apply_batch([a for a, _ in dels], [b for _, b in dels], [a for a, _ in ins], [b for _, b in ins])
    assert np.all(np.diff(g.out_csr()[0]) == k)
    t = 2.0 ** -30   # d * t ~ 5.6e-9: inside the range the rank changes pass through before tau = 1e-10
    for method in ("df", "dfp"):
        rc, sc = g.update(method, tau_f=t, tau_p=t, r_prev=r0, metric="contrib")
        ra, sa = g.update(method, tau_f=t * k, tau_p=t * k, r_prev=r0, metric="absolute")
        assert np.array_equal(rc, ra)
        assert (sc.iterations, sc.vertices_processed) == (sa.iterations, sa.vertices_processed)
        rr, sr = g.update(method, tau_f=t, tau_p=t, r_prev=r0, metric="absolute")
        assert sr.vertices_processed >= sc.vertices_processed   # a lower threshold processes at least as much here


@pytest.mark.parametrize("metric", ["relative", "absolute", "contrib"])
@pytest.mark.parametrize("order", ["sync", "async"])
def test_prune_everything_expand_nothing(metric, order):
    """Every measure is at most 1 here (dr <= max(r, R[v]) for non-negative
    ranks, and dr <= 1, dr / d <= 1 for ranks below 1), so DF-P with
    tau_f = tau_p = 1 expands nothing and prunes every vertex at its first
    visit: each initially affected vertex is processed exactly once, with one
    step of Eq. 2 from R_{t-1}, and the second iteration finds an empty
    frontier."""
    n = 200
    src, dst = random_graph(n, 1200, 71)
    g = oracle.Graph(n, src, dst)
    r0, _ = g.update("static", tau=1e-14)
    E0 = edge_set(n, src, dst)
    (ds, dd), (is_, id_) = random_batch(n, E0, 3, 6, 72, with_noise=False)
    g.apply_batch(ds, dd, is_, id_)
    F0 = g.initial_affected()
    r, st = g.update("dfp", tau_f=1.0, tau_p=1.0, r_prev=r0, metric=metric, order=order)
    assert st.vertices_processed == F0.sum() == st.vertices_ever_affected
    assert st.iterations == 2 and st.converged
    assert np.array_equal(r[~F0], r0[~F0])
    # the processed vertices moved by one Eq. 2 step from R_{t-1} (in the
    # synchronous order every in-neighbour still has its R_{t-1} rank)
    if order == "sync":
        off, adj = g.in_csr()
        oo, _ = g.out_csr()
        d = np.diff(oo)
        for v in np.flatnonzero(F0)[:20]:
            c = sum(r0[u] / d[u] for u in adj[off[v]:off[v + 1]])
            assert r[v] == oracle.rank_closed_loop(ALPHA, n, c, r0[v], int(d[v]))


@pytest.mark.parametrize("method", ["df", "dfp"])
@pytest.mark.parametrize("seed", [81, 82])
def test_frontier_without_expansion_solves_the_restricted_system(method, seed):
    """With expansion switched off (tau_f = inf) and no pruning (tau_p = 0),
    DF and DF-P sweep exactly the initially affected set F_0 (Alg. 1) with every
    other vertex held at R_{t-1}.  Their limit is then the solution of the
    linear system restricted to F_0: x_v = (1-alpha)/n + alpha sum_{u in in(v)}
    x_u / |out(u)| for v in F_0, with x_u = R_{t-1}[u] outside F_0 (Eq. 1; Eq. 2
    has the same fixed point), solved here with numpy's LAPACK solver."""
    n = 150
    src, dst = random_graph(n, 700, seed)
    g = oracle.Graph(n, src, dst)
    r0, _ = g.update("static", tau=1e-15, max_iter=5000)
    E0 = edge_set(n, src, dst)
    (ds, dd), (is_, id_) = random_batch(n, E0, 2, 4, seed + 100, with_noise=False)
    g.apply_batch(ds, dd, is_, id_)
    F0 = g.initial_affected().astype(bool)
    assert 0 < F0.sum() < n
    E1 = (E0 - set(zip(ds.tolist(), dd.tolist()))) | set(zip(is_.tolist(), id_.tolist()))
    E1 |= {(v, v) for v in range(n)}
    outdeg = np.zeros(n)
    for u, _ in E1:
        outdeg[u] += 1
    A = np.eye(n)
    for u, w in E1:
        A[w, u] -= ALPHA / outdeg[u]
    b = np.full(n, (1 - ALPHA) / n)
    F, O = np.flatnonzero(F0), np.flatnonzero(~F0)
    x = np.linalg.solve(A[np.ix_(F, F)], b[F] - A[np.ix_(F, O)] @ r0[O])
    r, st = g.update(method, tau=1e-15, tau_f=np.inf, tau_p=0.0, max_iter=5000, r_prev=r0)
    assert st.converged
    assert st.vertices_ever_affected == F0.sum()
    assert np.array_equal(r[O], r0[O])
    assert np.max(np.abs(r[F] - x)) < 1e-12


# ------------------------------------------------------------ prune against re-mark (reading C2)


from cases import prune_vs_mark_case  # noqa: E402


def test_pruned_vertex_re_marked_by_expanding_in_neighbour():
    """Alg. 1, Sec. 4.1.2: a vertex pruned in iteration i but marked by an
    expanding in-neighbour in the same iteration is swept in iteration i + 1
    (F_{i+1} = M_i u (F_i \\ P_i)).  The expected sets are derived by hand in
    the fixture; a 'prune wins' order would drop vertex 2 from F_1 (5 vertices
    processed in two iterations instead of 6, R[2] unchanged in iteration 1)."""
    g, r, meta = prune_vs_mark_case()
    assert set(np.flatnonzero(g.initial_affected()).tolist()) == set(meta["initial"])
    r1, s1 = g.update("dfp", tau=0.0, max_iter=1, r_prev=r)
    r2, s2 = g.update("dfp", tau=0.0, max_iter=2, r_prev=r)
    # iteration 0: 0 and 2 keep their ranks (pruned), 1 moves (expands)
    for v in meta["pruned0"]:
        assert abs(r1[v] - r[v]) <= 1e-6 * r[v]
    for v in meta["expanders0"]:
        assert abs(r1[v] - r[v]) > 1e-6 * max(r1[v], r[v])
    assert s1.vertices_processed == len(meta["initial"])
    # F_1 = {1, 2, 3} is swept in iteration 1.  2 and 3 change (they read the
    # new R[1]); 1 is swept but Eq. 2 gives it the same value, since its only
    # other in-neighbour, 0, did not change; 0 is not swept and keeps its bits
    f1 = set(meta["frontier1"])
    assert s2.vertices_processed - s1.vertices_processed == len(f1) == meta["processed_after2"][0] - 3
    changed = set(np.flatnonzero(r2 != r1).tolist())
    assert changed == f1 - {1}
    assert r2[0] == r1[0]
    assert s2.vertices_ever_affected == meta["ever_after2"][0]
    # Eq. 2 for vertex 2 in iteration 1 reads the new R[1]
    C0 = (1 - ALPHA) / 6
    expect2 = (C0 + ALPHA * (r1[0] / 3 + r1[1] / 3)) / (1 - ALPHA)
    assert r2[2] == pytest.approx(expect2, rel=1e-14)


# ------------------------------------------------------------ the OpenMP build of the oracle


@pytest.mark.parametrize("seed", [1, 2])
def test_openmp_build_gives_the_same_bits(seed):
    """The oracle built with -fopenmp (threaded sweeps, sorts and adjacency
    rebuild) returns exactly what the single-threaded build returns: the same
    edge sets, effective changes, affected sets, ranks and statistics for every
    method, measure and order, over a chain of batches."""
    oracle.set_threads(4)
    assert oracle.threads() == 4
    scale = 12
    n = 1 << scale
    src, dst = synth.rmat(scale, 16 * n, 600 + seed)
    A, B = oracle.Graph(n, src, dst), oracle.Graph(n, src, dst, parallel=True)
    for x, y in zip(A.out_csr() + A.in_csr(), B.out_csr() + B.in_csr()):
        assert np.array_equal(x, y)
    ra, sa = A.update("static")
    rb, sb = B.update("static")
    assert np.array_equal(ra, rb) and sa == sb
    cs, cd = synth.unique_edges(src, dst)
    for step in range(3):
        b = synth.batch(n, cs, cd, 50 + 400 * step, 700 + seed * 10 + step)
        A.apply_batch(*b)
        B.apply_batch(*b)
        for x, y in zip(A.out_csr() + A.in_csr() + A.effective_delta(), B.out_csr() + B.in_csr() + B.effective_delta()):
            assert np.array_equal(x, y)
        assert np.array_equal(A.initial_affected(), B.initial_affected())
        for method in ("static", "nd", "dt", "df", "dfp"):
            for metric, order in (("relative", "sync"), ("absolute", "sync"), ("relative", "async")):
                tf = 1e-12 if metric == "absolute" else 1e-6
                x, s1 = A.update(method, r_prev=ra, metric=metric, order=order, tau_f=tf, tau_p=tf)
                y, s2 = B.update(method, r_prev=ra, metric=metric, order=order, tau_f=tf, tau_p=tf)
                assert np.array_equal(x, y), (step, method, metric, order)
                assert s1 == s2, (step, method, metric, order)
        ra, _ = A.update("dfp", r_prev=ra)


def test_openmp_build_sorts_large_edge_lists():
    """Edge lists long enough for the threaded sort (runs sorted per thread,
    then merged) build the same graph as the single-threaded build."""
    oracle.set_threads(3)
    n = 1 << 16
    src, dst = synth.rmat(16, 5_000_000, 77)
    A, B = oracle.Graph(n, src, dst), oracle.Graph(n, src, dst, parallel=True)
    assert A.m == B.m
    for x, y in zip(A.out_csr() + A.in_csr(), B.out_csr() + B.in_csr()):
        assert np.array_equal(x, y)


# ------------------------------------------------------------ vertex insertion and deletion


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_resize_carries_the_fixed_point_over(seed):
    """Adding isolated vertices (self-loop only) to a graph: the linear-system
    solution of the grown graph equals the old solution times n / n_new, with
    1 / n_new on the new vertices (numpy LAPACK on both graphs), and the
    oracle's resize gives the grown edge set."""
    n, n_new = 40, 57
    src, dst = random_graph(n, 160, 80 + seed)
    g = oracle.Graph(n, src, dst)
    r_old = pagerank_solve(n, edge_set(n, src, dst))
    g.resize(n_new)
    assert g.n == n_new
    off, adj = g.out_csr()
    grown = {(u, int(w)) for u in range(n_new) for w in adj[off[u]:off[u + 1]]}
    assert grown == edge_set(n_new, src, dst)
    exact_new = pagerank_solve(n_new, grown)
    carried = oracle.resize_ranks(r_old, n_new)
    assert np.max(np.abs(carried - exact_new)) < 1e-14
    assert np.all(carried[n:] == 1.0 / n_new)
    # the carried ranks are a fixed point: ND stops after one sweep
    r, st = g.update("nd", tau=1e-13, r_prev=carried)
    assert st.iterations == 1 and np.max(np.abs(r - exact_new)) < 1e-14
    # the last batch is cleared: DF-P processes nothing
    r, st = g.update("dfp", r_prev=carried)
    assert st.vertices_processed == 0 and np.array_equal(r, carried)


def test_resize_removes_isolated_tail_only():
    """Removing vertices: allowed only once their edges are deleted; the
    solution of the smaller graph is the isolated-tail solution times
    n / n_new, and DF-P after a batch that connects a grown graph's new
    vertices reaches the linear-system solution at zero tolerance."""
    n = 30
    src, dst = random_graph(n, 120, 7)
    g = oracle.Graph(n, src, dst)
    before = (g.out_csr(), g.in_csr())
    with pytest.raises(oracle.OracleError):
        g.resize(20)                     # vertices 20..29 still have edges
    assert all(np.array_equal(a, b) for a, b in zip(g.out_csr() + g.in_csr(), before[0] + before[1]))
    # delete every edge touching 20..29, then remove them
    E = edge_set(n, src, dst)
    gone = [(u, v) for u, v in E if u != v and (u >= 20 or v >= 20)]
    g.apply_batch(del_src=[u for u, _ in gone], del_dst=[v for _, v in gone])
    E2 = E - set(gone)
    r_iso = pagerank_solve(n, E2)
    g.resize(20)
    E3 = {(u, v) for u, v in E2 if u < 20 and v < 20}
    exact = pagerank_solve(20, E3)
    assert np.max(np.abs(oracle.resize_ranks(r_iso, 20) - exact)) < 1e-14
    # grow again and connect the new vertices with a batch: DF-P at zero
    # tolerance from the carried ranks reaches the new fixed point
    g.resize(26)
    carried = oracle.resize_ranks(exact, 26)
    ins = [(20, 3), (3, 21), (22, 20), (25, 0), (24, 24), (5, 23)]
    g.apply_batch(ins_src=[u for u, _ in ins], ins_dst=[v for _, v in ins])
    E4 = edge_set(26, [u for u, _ in E3] + [u for u, _ in ins], [v for _, v in E3] + [v for _, v in ins])
    r, _ = g.update("dfp", tau=1e-15, tau_f=0.0, tau_p=0.0, r_prev=carried)
    assert np.max(np.abs(r - pagerank_solve(26, E4))) < 1e-12


# ------------------------------------------------------------ the ranges order (Alg. 1, one rank vector, eight id ranges in turn)


def range_bounds(in_off, P=8):
    """The ranges of the ranges order on in-rows with offsets in_off: cut at
    multiples of 128 where the in-degree prefix first reaches k / P of all
    in-edges (one range below 128 P vertices)."""
    n = len(in_off) - 1
    P = P if n >= 128 * P else 1
    W = int(in_off[n])
    b = [0]
    for k in range(1, P):
        j = 0
        while 128 * j < n and int(in_off[128 * j]) * P < k * W:
            j += 1
        b.append(min(128 * j, n))
    return b + [n]


@pytest.mark.parametrize("method", ["static", "nd", "df", "dfp"])
def test_ranges_order_reaches_fixed_point_at_zero_tolerance(method):
    """Eight ranges of 1280 vertices: every method in the ranges order reaches
    the linear-system solution of G_t (numpy LAPACK) at zero tolerances."""
    n = 1280
    src, dst = random_graph(n, 6000, 41)
    g = oracle.Graph(n, src, dst)
    E0 = edge_set(n, src, dst)
    r0 = pagerank_solve(n, E0)
    (ds, dd), (is_, id_) = random_batch(n, E0, 30, 120, 42)
    g.apply_batch(ds, dd, is_, id_)
    off, adj = g.out_csr()
    E1 = {(u, int(w)) for u in range(n) for w in adj[off[u]:off[u + 1]]}
    r, st = g.update(method, tau=1e-15, tau_f=0.0, tau_p=0.0, max_iter=5000, r_prev=r0, order="ranges")
    assert st.converged
    assert np.max(np.abs(r - pagerank_solve(n, E1))) < 1e-12


@pytest.mark.parametrize("skewed", [False, True])
def test_ranges_order_reads_earlier_ranges_only(skewed):
    """What sets the ranges order apart, checked against the synchronous order:
    (a) one sweep gives range 0 exactly the synchronous values (it reads only
    start-of-sweep ranks) and gives a later vertex the synchronous value
    whenever none of its in-neighbours lies in an earlier range;
    (b) a later vertex with an in-neighbour in an earlier range gets Eq. 1
    evaluated on the updated ranks of that range;
    (c) a graph with no edge between ranges, and any graph below 1024
    vertices (one range), gives the synchronous result bit for bit.
    skewed: most in-edges go to low ids, so the ranges, which hold equal
    shares of the in-edges, are far from equal in vertices."""
    n = 1280
    src, dst = random_graph(n, 5000, 43)
    if skewed:
        dst = np.minimum(np.random.default_rng(46).geometric(1.0 / 150, dst.size) - 1, n - 1)
    g = oracle.Graph(n, src, dst)
    b = range_bounds(g.in_csr()[0])
    if skewed:
        assert b[1] == 128 and b[-2] <= n // 2, b   # not the ranges of equal vertex counts
    r0 = np.random.default_rng(44).random(n)
    r0 /= r0.sum()
    rs, _ = g.update("nd", tau=0.0, max_iter=1, r_prev=r0)
    rr, _ = g.update("nd", tau=0.0, max_iter=1, r_prev=r0, order="ranges")
    rng_of = np.searchsorted(b, np.arange(n), side="right") - 1
    off, adj = g.in_csr()
    ooff, _ = g.out_csr()
    deg = np.diff(ooff)
    for v in range(n):
        ins = adj[off[v]:off[v + 1]]
        early = ins[rng_of[ins] < rng_of[v]]
        if early.size == 0:
            assert rr[v] == rs[v], v
        else:
            mixed = np.where(rng_of[ins] < rng_of[v], rr[ins], r0[ins]) / deg[ins]
            expect = (1 - ALPHA) / n + ALPHA * mixed.sum()
            assert rr[v] == pytest.approx(expect, rel=1e-12, abs=0), v
    # (c) no edge between ranges: none crosses a multiple of 128, where every
    # range bound lies
    keep = src // 128 == dst // 128
    g2 = oracle.Graph(n, src[keep], dst[keep])
    for m in ("static", "dfp"):
        x, sx = g2.update(m, r_prev=r0)
        y, sy = g2.update(m, r_prev=r0, order="ranges")
        assert np.array_equal(x, y) and sx == sy
    s3, d3 = random_graph(900, 4000, 45)
    g3 = oracle.Graph(900, s3, d3)
    x, sx = g3.update("static")
    y, sy = g3.update("static", order="ranges")
    assert np.array_equal(x, y) and sx == sy


@pytest.mark.parametrize("tau,stop_at_change", [(1e-6, False), (None, False), (1e-6, True)])
def test_tie_distance_is_the_nearest_decision(tau, stop_at_change):
    """The oracle's tie_rel (the relative distance of the nearest expand,
    prune or stop decision from its threshold, which the GPU tests use to tell
    a near-tie from a different frontier) equals a brute-force minimum over one
    DF-P iteration: every processed vertex's relative change against tau_f and
    tau_p, and the iteration's L-inf change against tau.  With tau_f = tau_p set
    to one vertex's own relative change the nearest decision is exactly on its
    threshold (0), and so it is with the iteration tolerance set to the
    iteration's own L-inf change."""
    n = 300
    src, dst = random_graph(n, 1500, 91)
    g = oracle.Graph(n, src, dst)
    r0, _ = g.update("static")
    E0 = edge_set(n, src, dst)
    (ds, dd), (is_, id_) = random_batch(n, E0, 20, 60, 92, with_noise=False)
    g.apply_batch(ds, dd, is_, id_)
    F0 = np.nonzero(g.initial_affected())[0]
    r1, _ = g.update("dfp", tau=1e-10, tau_f=1e-6, tau_p=1e-6, max_iter=1, r_prev=r0)
    dr = np.abs(r1[F0] - r0[F0])
    rel = dr / np.maximum(r1[F0], r0[F0])
    if tau is None:                     # a threshold exactly at one vertex's change
        tau = float(rel[len(rel) // 2])
    tau_stop = float(dr.max()) if stop_at_change else 1e-10
    r, st = g.update("dfp", tau=tau_stop, tau_f=tau, tau_p=tau, max_iter=1, r_prev=r0)
    assert np.array_equal(r, r1)        # one iteration: the ranks do not depend on the tolerances
    expect = min(float(np.min(np.abs(rel / tau - 1.0))), abs(float(dr.max()) / tau_stop - 1.0))
    assert st.tie_rel == expect
    if stop_at_change or tau == float(rel[len(rel) // 2]):
        assert st.tie_rel == 0.0
