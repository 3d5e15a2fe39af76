"""Failure handling, tested on the host: allocation failures injected with
pr_debug_fail_alloc (the device is never exhausted or faulted), invalid
inputs, and checkpoint / resume of a graph through the C ABI's exports."""
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
    yield pr
    pr.pr_debug_fail_alloc(0)


def small_graph(n=1 << 10, seed=3):
    src, dst = synth.rmat(10, 8 * n, seed)
    return n, src, dst


def test_every_allocation_of_graph_creation_can_fail_cleanly(lib):
    """Whichever device allocation of pr_graph_create_edges fails, the call
    returns PR_ENOMEM with a message and no graph; afterwards the library
    works as before."""
    n, src, dst = small_graph()
    O = oracle.Graph(n, src, dst)
    ref, _ = O.update("static")
    failed = 0
    for k in range(1, 200):
        lib.pr_debug_fail_alloc(k)
        try:
            G = lib.Graph.from_edges(n, src, dst)
        except lib.PRError as e:
            assert e.status == 3, e           # PR_ENOMEM
            failed += 1
            continue
        finally:
            lib.pr_debug_fail_alloc(0)
        G.update("static")                    # k was past the last allocation
        assert np.max(np.abs(G.ranks() - ref)) < TOL
        G.close()
        break
    else:
        pytest.fail("graph creation never completed")
    assert failed >= 10
    G = lib.Graph.from_edges(n, src, dst)
    G.update("static")
    assert np.max(np.abs(G.ranks() - ref)) < TOL


def test_allocation_failure_in_a_repack_and_in_tuning(lib):
    """A batch whose repack cannot allocate returns PR_ENOMEM (the graph is
    then to be destroyed, as documented); tuning and group creation that
    cannot allocate return PR_ENOMEM and leave the graph usable."""
    n, src, dst = small_graph(seed=5)
    G = lib.Graph.from_edges(n, src, dst)
    G.update("static")
    r0 = G.ranks()
    lib.pr_debug_fail_alloc(1)
    with pytest.raises(lib.PRError) as e:
        G.autotune("dfp")
    assert e.value.status == 3
    lib.pr_debug_fail_alloc(1)
    with pytest.raises(lib.PRError) as e:
        lib.Group([G])
    assert e.value.status == 3
    lib.pr_debug_fail_alloc(0)
    assert np.array_equal(G.ranks(), r0)
    G.update("nd", max_iter=2)                # still usable
    # overflow one row far past its slack so the direction is repacked
    hub = np.full(600, 17, np.int32)
    tgt = np.arange(600, dtype=np.int32) % n
    lib.pr_debug_fail_alloc(1)
    try:
        with pytest.raises(lib.PRError) as e:
            G.apply_batch(ins_src=hub, ins_dst=tgt)
        assert e.value.status == 3
    finally:
        lib.pr_debug_fail_alloc(0)
    G.close()
    H = lib.Graph.from_edges(n, src, dst)     # the library is fine
    H.apply_batch(ins_src=hub, ins_dst=tgt)
    O = oracle.Graph(n, src, dst)
    O.apply_batch(ins_src=hub, ins_dst=tgt)
    for mine, ref in ((H.out_csr(), O.out_csr()), (H.in_csr(), O.in_csr())):
        assert np.array_equal(mine[0], ref[0]) and np.array_equal(mine[1], ref[1])


def test_checkpoint_and_resume(lib, tmp_path):
    """A graph saved after batches and updates, and loaded into a new handle,
    continues with the same results: the next batch and DF-P update give the
    same ranks, bit for bit, as on the original graph."""
    n = 1 << 12
    src, dst = synth.rmat(12, 16 * n, 61)
    G = lib.Graph.from_edges(n, src, dst)
    G.set_tuning(512, 4, 0, 0, 2)
    G.update("static")
    cs, cd = synth.unique_edges(src, dst)
    for i in range(2):
        G.apply_batch(*synth.batch(n, cs, cd, 300, 62 + i))
        G.update("dfp")
    path = tmp_path / "graph.npz"
    G.save(path)
    H = lib.Graph.load(path)
    assert H.tuning() == G.tuning()
    assert np.array_equal(H.ranks(), G.ranks())
    for a, b in ((H.out_csr(), G.out_csr()), (H.in_csr(), G.in_csr())):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    b = synth.batch(n, cs, cd, 300, 70)
    for X in (G, H):
        X.apply_batch(*b)
        X.update("dfp")
    assert np.array_equal(H.ranks(), G.ranks())
