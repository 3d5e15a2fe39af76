"""Helpers shared by the oracle's pins and the GPU parity tests: hand-made
cases read from tests/golden, and the check that a GPU run took the same
decisions of Alg. 1 as the oracle's run."""
import os

import numpy as np

import oracle

ALPHA = 0.85
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_prune_vs_mark():
    edges, meta, cur = [], {}, None
    with open(os.path.join(GOLDEN, "prune_vs_mark_6v.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            if line in ("edges", "end"):
                cur = "edges" if line == "edges" else None
                continue
            if cur == "edges":
                a, b = line.split()
                edges.append((int(a), int(b)))
            else:
                k, *vals = line.split()
                meta[k] = [float(x) if "." in x else int(x) for x in vals]
    return edges, meta


def prune_vs_mark_case():
    """The graph after the batch, and the previous ranks the fixture defines."""
    edges, meta = load_prune_vs_mark()
    n, a = 6, ALPHA
    g = oracle.Graph(n, [x for x, _ in edges], [y for _, y in edges])
    g.apply_batch(ins_src=[meta["insert"][0]], ins_dst=[meta["insert"][1]])
    C0 = (1 - a) / n
    r = np.full(n, meta["rank_rest"][0])
    r[1] = meta["rank1"][0]
    r[0] = C0 / (1 - a / 3)
    r[2] = (C0 + a * (r[0] / 3 + r[1] / 3)) / (1 - a)
    return g, r, meta


# The GPU sums contributions in 2^-61 fixed point and the oracle in FP64, so
# their ranks differ by about 1e-18 .. 1e-16 absolute (at most 2^-62 per
# in-edge term, accumulated over the iterations by at most 1 / (1 - alpha)).
# A frontier measure is a rank change of about tau_f * r, r >= (1 - alpha)/n,
# so its relative error stays below about 1e-7 on the graphs of these tests
# (n <= 2^18, in-degrees of a few thousand at most), and Delta R's against
# tau = 1e-10 below 1e-6.  A decision of Alg. 1 (expand, prune, stop) can go
# the other way only where the oracle's quantity is within that relative
# distance of its threshold.
TIE_REL = 1e-6


def assert_same_run(st, ost, what=""):
    """Iterations, vertices ever affected and vertex updates of a GPU run
    equal the oracle's: the same decisions of Alg. 1 in every iteration.  They
    may differ only when the oracle reports a decision within TIE_REL of its
    threshold (a near-tie), and then by one iteration at most."""
    got = (st.iterations, st.vertices_ever_affected, st.vertices_processed)
    ref = (ost.iterations, ost.vertices_ever_affected, ost.vertices_processed)
    if got != ref:
        assert ost.tie_rel < TIE_REL, ("different run without a near-tie", what, got, ref, ost.tie_rel)
        assert abs(got[0] - ref[0]) <= 1, (what, got, ref, ost.tie_rel)
