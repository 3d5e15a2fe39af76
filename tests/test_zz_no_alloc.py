"""pr_sweep_noalloc: the rank sweep for callers that cannot allocate device
memory, checked against the regular entry point.

Some callers cannot call cudaMalloc (it may synchronize the device, or their
device memory belongs to another allocator).  pr_sweep_noalloc runs one Eq. 1
sweep over a caller-provided in-CSR using a fixed scratch array inside the
library.  Two calls in a row must match two single-sweep pr_update calls
(Naive-dynamic, one iteration) within the tolerance the parity tests use.
This file is collected last so that a failure here comes after every other
test has run.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-9


def test_noalloc_sweep_matches_pr_update_twice():
    torch = pytest.importorskip("torch")
    import paper_2401_15870_gb300 as pr
    n = 1 << 14
    src, dst = synth.rmat(14, 16 * n, 4242)
    G = pr.Graph.from_edges(n, src, dst)
    G.update("static", max_iter=3)
    r = G.ranks()
    in_off, in_src = G.in_csr()
    out_off, _ = G.out_csr()
    out_deg = np.diff(out_off).astype(np.int32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    t_off, t_src, t_deg = dev(in_off), dev(in_src), dev(out_deg)
    r_in = dev(r)
    r_out = torch.empty(n, dtype=torch.float64, device="cuda")
    delta = torch.empty(1, dtype=torch.float64, device="cuda")
    for call in range(2):
        G.set_ranks(r_in.cpu().numpy())
        st = G.update("nd", max_iter=1)
        expect = G.ranks()
        pr.pr_sweep_noalloc(n, t_off, t_src, t_deg, r_in, r_out, 0.85, delta)
        torch.cuda.synchronize()
        got = r_out.cpu().numpy()
        assert np.max(np.abs(got - expect)) < TOL, call
        assert abs(delta.item() - st.delta_R) < TOL, call
        r_in = r_out.clone()


def test_noalloc_rejects_sizes_beyond_its_array():
    import paper_2401_15870_gb300 as pr
    torch = pytest.importorskip("torch")
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    i64 = torch.zeros(4, dtype=torch.int64, device="cuda")
    i32 = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(pr.PRError) as e:
        pr.pr_sweep_noalloc(pr.PR_NOALLOC_MAX_N + 1, i64, i32, i32, x, x, 0.85, x)
    assert e.value.status == 1
