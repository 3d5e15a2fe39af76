"""The asynchronous order of Alg. 1 on the GPU (PR_OPT_ASYNC, Sec. 4.4): eight
consecutive vertex ranges swept in turn, each reading the ranks of the
ranges before it as updated in the sweep.  On graphs that keep the caller's
vertex order the ranges are the oracle's ranges order, so ranks must agree
within 1e-9 with the same decisions of Alg. 1; on relabelled graphs (ranges
of the internal order) the checks are what holds for any such schedule: at
zero tolerances every method reaches the linear-system solution of Eq. 1
(the oracle's Static at tau = 1e-15 is pinned to numpy's LAPACK solve), and
at the default tolerances DF / DF-P stay as close to that solution as the
synchronous order does.  Vertices outside every frontier keep their previous
ranks bit for bit."""
import numpy as np
import pytest

import oracle
import synth
from cases import assert_same_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2401_15870_gb300 as pr
    pr.load()
    return pr


def case(lib, scale, ef, bsize, seed, keep_order=False):
    n = 1 << scale
    src, dst = synth.rmat(scale, ef * n, seed)
    G = lib.Graph.from_edges(n, src, dst, keep_order=keep_order)
    O = oracle.Graph(n, src, dst)
    r0, _ = O.update("static")
    cs, cd = synth.unique_edges(src, dst)
    b = synth.batch(n, cs, cd, bsize, seed + 1)
    G.apply_batch(*b)
    O.apply_batch(*b)
    exact, _ = O.update("static", tau=1e-15, max_iter=500)
    return G, O, r0, exact


@pytest.mark.parametrize("scale,ef", [(7, 4), (10, 8), (13, 16)])
@pytest.mark.parametrize("method", ["static", "nd", "df", "dfp"])
def test_async_reaches_the_fixed_point_at_zero_tolerance(lib, scale, ef, method):
    G, O, r0, exact = case(lib, scale, ef, 3 * scale, 40 + scale)
    G.set_ranks(r0)
    st = G.update(method, tau=1e-14, tau_f=0.0, tau_p=0.0, order="async")
    assert st.converged
    assert np.max(np.abs(G.ranks() - exact)) < 1e-12


@pytest.mark.parametrize("method", ["df", "dfp"])
def test_async_default_tolerances_within_the_convergence_bound(lib, method):
    """R-MAT 2^14 vertices, one batch of 1e-3 |E|: the asynchronous update is
    within 10 tau_p / (1 - alpha) of the fixed point (the bound the oracle's
    pins use for DF-P), no further from it than twice the synchronous
    update's error, and it leaves every vertex outside the reachable set of
    the batch at its previous rank."""
    G, O, r0, exact = case(lib, 14, 16, 262, 11)
    G.set_ranks(r0)
    st_s = G.update(method)
    sync = G.ranks()
    G.set_ranks(r0)
    st_a = G.update(method, order="async")
    asy = G.ranks()
    assert st_a.converged and st_s.converged
    bound = 10 * 1e-6 / (1 - 0.85)
    assert np.max(np.abs(asy - exact)) < bound
    e_sync, e_async = np.sum(np.abs(sync - exact)), np.sum(np.abs(asy - exact))
    assert e_async <= 2 * e_sync + 1e-12, (e_async, e_sync)
    outside = ~O.dt_affected()
    assert np.array_equal(asy[outside], r0[outside])


def test_async_static_and_nd_agree_with_oracle(lib):
    """Static and ND at tau = 1e-12 in either order land within the power
    iteration's bound of the same fixed point."""
    G, O, r0, exact = case(lib, 13, 16, 100, 12)
    for method in ("static", "nd"):
        G.set_ranks(r0)
        st = G.update(method, tau=1e-12, order="async")
        assert st.converged
        assert np.max(np.abs(G.ranks() - exact)) < 1e-10
        assert abs(np.sum(G.ranks()) - 1.0) < 1e-9


def test_async_argument_errors(lib):
    G, O, r0, _ = case(lib, 8, 4, 10, 13)
    G.set_ranks(r0)
    for kw in ({"method": "dt"}, {"method": "dfp", "loop": "device"}, {"method": "dfp", "direction": "push"}):
        kw = dict(kw)
        m = kw.pop("method")
        with pytest.raises(lib.PRError) as e:
            G.update(m, order="async", **kw)
        assert e.value.status == 1
    grp = lib.Group([G])
    try:
        import ctypes
        opts = lib.pr_options(1e-6, 1e-6, 500, lib.PR_OPT_ASYNC)
        assert lib.load().pr_group_update(grp._q, 4, 0.85, 1e-10, ctypes.byref(opts), None) == 1
    finally:
        grp.close()


@pytest.mark.parametrize("method", ["static", "nd", "df", "dfp"])
@pytest.mark.parametrize("scale,bsize", [(9, 30), (12, 120), (14, 262)])
def test_async_matches_the_oracle_ranges_order(lib, method, scale, bsize):
    """Graphs that keep the caller's vertex order: the GPU's asynchronous
    order is the oracle's ranges order (one range below 1024 vertices, eight
    above), so ranks agree within 1e-9 and Alg. 1 takes the same decisions."""
    G, O, r0, _ = case(lib, scale, 16, bsize, 60 + scale, keep_order=True)
    G.set_ranks(r0)
    st = G.update(method, order="async")
    ref, ost = O.update(method, r_prev=r0, order="ranges")
    assert np.max(np.abs(G.ranks() - ref)) < 1e-9
    assert_same_run(st, ost, method)


def test_async_is_reproducible(lib):
    G, O, r0, _ = case(lib, 13, 16, 200, 14)
    out = []
    for _ in range(2):
        G.set_ranks(r0)
        st = G.update("dfp", order="async")
        out.append((G.ranks(), st.iterations, st.vertices_processed))
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1:] == out[1][1:]
