"""Checks of the seeded input generators (shapes, ranges, determinism)."""
import numpy as np

import synth


def test_rmat_deterministic_in_range_and_skewed():
    s1, d1 = synth.rmat(12, 1 << 16, 7)
    s2, d2 = synth.rmat(12, 1 << 16, 7)
    s3, _ = synth.rmat(12, 1 << 16, 8)
    assert np.array_equal(s1, s2) and np.array_equal(d1, d2)
    assert not np.array_equal(s1, s3)
    assert s1.min() >= 0 and s1.max() < 4096 and d1.min() >= 0 and d1.max() < 4096
    deg = np.bincount(s1, minlength=4096)
    # power law: the top 1 % of sources carry far more than 1 % of the edges
    top = np.sort(deg)[::-1][:41].sum() / deg.sum()
    assert top > 0.15
    # relabelling spreads the hubs: the largest out-degree is not at id 0
    assert np.argmax(deg) != 0


def test_permutation_is_a_bijection():
    for n in (1, 2, 3, 17, 1000, 4096):
        img = sorted(synth.perm(x, n, 99) for x in range(n))
        assert img == list(range(n))


def test_batch_composition():
    src, dst = synth.rmat(10, 1 << 13, 3)
    cs, cd = synth.unique_edges(src, dst)
    ds, dd, is_, id_ = synth.batch(1024, cs, cd, 1000, 5)
    assert len(is_) == 800 and len(ds) == 200
    assert np.all(is_ != id_)
    assert is_.min() >= 0 and is_.max() < 1024
    cand = set(zip(cs.tolist(), cd.tolist()))
    assert all((a, b) in cand for a, b in zip(ds.tolist(), dd.tolist()))
    again = synth.batch(1024, cs, cd, 1000, 5)
    assert all(np.array_equal(a, b) for a, b in zip((ds, dd, is_, id_), again))


def test_temporal_stream_has_repeats_and_heavy_tail():
    n, m = 20000, 200000
    s, d = synth.temporal(n, m, 11)
    assert s.min() >= 0 and s.max() < n and d.min() >= 0 and d.max() < n
    keys = s.astype(np.int64) << 32 | d
    uniq = np.unique(keys).size / m
    assert 0.4 < uniq < 0.8
    deg = np.bincount(s, minlength=n)
    assert deg.max() > 50 * deg.mean()
