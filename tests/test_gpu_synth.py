"""The GPU generators draw the same arrays as the host generators."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_gpu_rmat_and_batch_equal_host():
    torch = pytest.importorskip("torch")
    import synth.gpu as sg
    sg.build()
    for scale, m, seed in ((1, 5, 1), (12, 1 << 15, 2), (17, 100003, 3)):
        hs, hd = synth.rmat(scale, m, seed)
        gs, gd = sg.rmat(scale, m, seed)
        assert np.array_equal(hs, gs.cpu().numpy()) and np.array_equal(hd, gd.cpu().numpy())
        hb = synth.batch(1 << scale, hs, hd, 997, seed + 5)
        gb = sg.batch(1 << scale, gs, gd, 997, seed + 5)
        for x, y in zip(hb, gb):
            assert np.array_equal(x, y.cpu().numpy())
