"""pr_sweep_noalloc: the rank sweep for callers that cannot allocate device
memory, checked against the oracle.

Some callers cannot call cudaMalloc: in their setting a device allocation may
synchronize the device or is not theirs to make (their device memory belongs
to another allocator).  pr_sweep_noalloc runs one Eq. 1 sweep over a
caller-provided in-CSR using a fixed scratch array inside the library.  Two
calls in a row (the second from the first's output) must match the oracle's
Naive-dynamic update run for one and for two iterations from the same ranks,
within the tolerance the parity tests use.  This file is collected last so
that a failure here comes after every other test has run; it also passes when
run alone in a fresh process.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-9


def test_noalloc_sweep_matches_oracle_twice():
    torch = pytest.importorskip("torch")
    import paper_2401_15870_gb300 as pr
    n = 1 << 14
    src, dst = synth.rmat(14, 16 * n, 4242)
    O = oracle.Graph(n, src, dst)
    r, _ = O.update("static", max_iter=3)          # a start that is not yet a fixed point
    in_off, in_src = O.in_csr()
    out_off, _ = O.out_csr()
    out_deg = np.diff(out_off).astype(np.int32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    t_off, t_src, t_deg = dev(in_off), dev(in_src), dev(out_deg)
    bufs = [dev(r), torch.empty(n, dtype=torch.float64, device="cuda")]
    delta = torch.empty(1, dtype=torch.float64, device="cuda")
    for call in range(2):
        expect, st = O.update("nd", tau=0.0, max_iter=call + 1, r_prev=r)
        pr.pr_sweep_noalloc(n, t_off, t_src, t_deg, bufs[call % 2], bufs[1 - call % 2], 0.85, delta)
        torch.cuda.synchronize()
        got = bufs[1 - call % 2].cpu().numpy()
        assert np.max(np.abs(got - expect)) < TOL, call
        assert abs(delta.item() - st.delta_R) < TOL, call


def test_noalloc_rejects_sizes_beyond_its_array_and_overlapping_ranks():
    import paper_2401_15870_gb300 as pr
    torch = pytest.importorskip("torch")
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    y = torch.zeros(4, dtype=torch.float64, device="cuda")
    i64 = torch.zeros(5, dtype=torch.int64, device="cuda")
    i32 = torch.ones(4, dtype=torch.int32, device="cuda")
    with pytest.raises(pr.PRError) as e:
        pr.pr_sweep_noalloc(pr.PR_NOALLOC_MAX_N + 1, i64, i32, i32, x, y, 0.85, x)
    assert e.value.status == 1
    with pytest.raises(pr.PRError) as e:
        pr.pr_sweep_noalloc(4, i64, i32, i32, x, x, 0.85, y)
    assert e.value.status == 1
