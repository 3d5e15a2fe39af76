"""Error of the synchronous and the asynchronous order (Sec. 4.4) on a small
temporal stream, from the oracle alone (CPU, single thread).

Base graph: the first 90% of a copying / preferential-attachment stream of
20,000 vertices and 400,000 timestamped edges; then three consecutive
insertion-only batches of 1e-3 |E_T| (400 edges).  Every method starts from
the exact fixed point of G_{t-1} (Static at tau = 0, 500 iterations) and is
compared, in L1, with the exact fixed point of G_t.

    python oracle/compare_orders.py
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
import synth  # noqa: E402


def main():
    n, m = 20000, 400000
    s, d = synth.temporal(n, m, 5)
    base = int(0.9 * m)
    g = oracle.Graph(n, s[:base], d[:base])
    r_prev, _ = g.update("static", tau=0.0, max_iter=500)
    pos, size = base, 400
    print("batch method order   L1 error  iterations  vertex updates")
    for k in range(3):
        g.apply_batch([], [], s[pos:pos + size], d[pos:pos + size])
        pos += size
        ref, _ = g.update("static", tau=0.0, max_iter=500)
        rs, ss = g.update("static")
        print("%5d %-6s %-6s %9.2e %11d %15d" % (k, "static", "sync", np.abs(rs - ref).sum(), ss.iterations,
                                                   ss.vertices_processed))
        for meth in ("nd", "df", "dfp"):
            for order in ("sync", "async"):
                r, st = g.update(meth, r_prev=r_prev, order=order)
                print("%5d %-6s %-6s %9.2e %11d %15d" % (k, meth, order, np.abs(r - ref).sum(), st.iterations,
                                                           st.vertices_processed))
        r_prev = ref


if __name__ == "__main__":
    main()
