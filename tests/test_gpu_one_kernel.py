"""The iteration loop in one cooperative kernel (PR_OPT_ONE_KERNEL): init,
marking and every iteration's gather, epilogue and control as phases of one
launch separated by grid barriers.  Its ranks and statistics must be the bits
of the CUDA-graph loop and of the host loop, and within 1e-9 of the oracle
with the oracle's iterations and frontier (Alg. 1, Eq. 1, Eq. 2)."""
import ctypes

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


def case(pr, scale, ef, bsize, seed, n=None):
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


def run(G, r0, method, **kw):
    G.set_ranks(r0)
    st = G.update(method, **kw)
    return G.ranks(), (st.iterations, st.converged, st.vertices_ever_affected, st.vertices_processed,
                       st.edges_processed)


# n = 2, ragged n, several warp steps, an empty batch
SIZES = [(1, 2, 2, 11, None), (7, 5, 9, 12, 101), (10, 16, 60, 13, 1000), (12, 8, 0, 14, None),
         (13, 16, 500, 15, 7000)]


@pytest.mark.parametrize("method", ["static", "nd", "df", "dfp"])
@pytest.mark.parametrize("max_iter", [0, 1, 3, 500])
def test_one_kernel_equals_the_other_loops(lib, method, max_iter):
    for spec in SIZES:
        G, O, r0 = case(lib, *spec)
        # the host loop's statistics of a run cut short are its own (it picks
        # the sweep form per iteration), so it is compared at full runs only
        loops = ("one", "device", "host") if max_iter == 500 else ("one", "device")
        out = {loop: run(G, r0, method, loop=loop, max_iter=max_iter) for loop in loops}
        for loop in loops[1:]:
            assert np.array_equal(out["one"][0], out[loop][0]), (spec, loop)
            assert out["one"][1] == out[loop][1], (spec, loop, out["one"][1], out[loop][1])


@pytest.mark.parametrize("method", ["static", "nd", "df", "dfp"])
@pytest.mark.parametrize("spec", [(12, 16, 262, 21, None), (14, 16, 262, 22, None), (11, 12, 40, 23, 1999)])
def test_one_kernel_matches_the_oracle(lib, method, spec):
    G, O, r0 = case(lib, *spec)
    G.set_ranks(r0)
    st = G.update(method, loop="one")
    ref, ost = O.update(method, r_prev=r0)
    assert np.max(np.abs(G.ranks() - ref)) < TOL
    assert_same_run(st, ost, (method, spec))


def test_one_kernel_above_the_default_size(lib):
    """Forced on a graph that by default takes the CUDA graph: same bits."""
    G, O, r0 = case(lib, 17, 24, 2000, 31)
    assert G.m >= lib.PR_ONE_KERNEL_SLOTS
    for method in ("dfp", "nd"):
        a = run(G, r0, method, loop="one")
        b = run(G, r0, method, loop="device")
        assert np.array_equal(a[0], b[0])
        assert a[1] == b[1]


def test_default_loop_choice(lib):
    """Small graphs run the whole update as one launch; graphs of at least
    PR_ONE_KERNEL_SLOTS in-CSR slots (below PR_DEVICE_LOOP_SLOTS) run the CUDA
    graph, init and mark plus three kernels per iteration."""
    small, _, rs = case(lib, 12, 16, 262, 41)
    large, _, rl = case(lib, 17, 24, 2000, 43)
    for G, r0, one in ((small, rs, True), (large, rl, False)):
        G.set_ranks(r0)
        G.update("dfp")   # tables for this alpha
        G.set_ranks(r0)
        k0 = lib.pr_kernel_launches()
        st = G.update("dfp")
        launched = lib.pr_kernel_launches() - k0
        assert launched == (1 if one else 2 + 3 * st.iterations), (G.n, launched, st.iterations)


def test_group_in_one_kernel_equals_solo_runs(lib):
    """A group of graphs of different sizes in one launch: every graph gets
    the bits of its own update."""
    cs = [case(lib, *spec) for spec in SIZES]
    graphs = [c[0] for c in cs]
    grp = lib.Group(graphs)
    try:
        for method in ("dfp", "static"):
            for G, O, r0 in cs:
                G.set_ranks(r0)
            st = grp.update(method, loop="one")
            got = [G.ranks() for G in graphs]
            for (G, O, r0), r, s in zip(cs, got, st):
                r_solo, st_solo = run(G, r0, method, loop="device")
                assert np.array_equal(r, r_solo), (G.n, method)
                assert (s.iterations, s.converged, s.vertices_ever_affected, s.vertices_processed,
                        s.edges_processed) == st_solo
    finally:
        grp.close()


def test_one_kernel_option_errors(lib):
    G, O, r0 = case(lib, 9, 8, 20, 51)
    G.set_ranks(r0)
    with pytest.raises(lib.PRError):
        G.update("dt", loop="one")
    with pytest.raises(lib.PRError):
        G.update("dfp", loop="one", time_sweeps=True)
    with pytest.raises(lib.PRError):
        G.update("dfp", loop="one", direction="push")
    with pytest.raises(lib.PRError):
        G.update("dfp", loop="one", order="async")
    opts = lib.pr_options(1e-6, 1e-6, 500, lib.PR_OPT_ONE_KERNEL | lib.PR_OPT_HOST_LOOP)
    st = lib.pr_stats()
    assert lib.load().pr_update(G._h, 4, 0.85, 1e-10, ctypes.byref(opts), ctypes.byref(st)) == 1   # PR_EINVAL
    # the graph is untouched and still updates
    G.set_ranks(r0)
    G.update("dfp", loop="one")
    ref, _ = O.update("dfp", r_prev=r0)
    assert np.max(np.abs(G.ranks() - ref)) < TOL


def test_one_kernel_updates_from_two_threads(lib):
    """Two graphs on streams of their own, updated at the same time from two
    threads: the library orders their cooperative launches one after the
    other on the device, and every result is the one of the update alone."""
    import threading

    torch = pytest.importorskip("torch")
    specs = [(12, 16, 262, 61, None), (11, 12, 100, 62, 1500)]
    streams = [torch.cuda.Stream() for _ in specs]
    cases_ = []
    for spec, s in zip(specs, streams):
        scale, ef, bsize, seed, n = spec
        n = n or (1 << scale)
        src, dst = synth.rmat(scale, ef * n, seed)
        src, dst = src % n, dst % n
        G = lib.Graph.from_edges(n, src, dst, stream=s)
        O = oracle.Graph(n, src, dst)
        r0, _ = O.update("static")
        cs, cd = synth.unique_edges(src, dst)
        b = synth.batch(n, cs, cd, bsize, seed + 1)
        G.apply_batch(*b)
        cases_.append((G, r0))
    alone = [run(G, r0, "dfp", loop="one") for G, r0 in cases_]
    errors = []

    def worker(k):
        G, r0 = cases_[k]
        try:
            for _ in range(20):
                got = run(G, r0, "dfp", loop="one")
                if not (np.array_equal(got[0], alone[k][0]) and got[1] == alone[k][1]):
                    errors.append((k, got[1], alone[k][1]))
                    return
        except Exception as e:   # a barrier that gave up would raise here (PR_ETIMEOUT)
            errors.append((k, repr(e)))

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(len(cases_))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
