"""Seeded workload generators (inputs only): shapes, ranges and determinism."""
import numpy as np

from paper_1902_05875_gb300 import workloads as W


def test_batched_instances_recipe():
    a = W.batched_instances(32, seed=5)
    b = W.batched_instances(32, seed=5)
    assert all(np.array_equal(x.src, y.src) and np.array_equal(x.q, y.q) for x, y in zip(a, b))
    for w in a:
        nl = len(w.k)
        assert nl in (2, 3)
        d = np.asarray(w.interfaces)
        assert np.all(d <= 0.0) and np.all(d >= -2.0) and np.all(np.diff(d) < 0)
        if nl == 3:
            assert d[0] - d[1] >= 0.3
        assert all(1.0 <= k <= 4.0 for k in w.k)
        assert 1000 <= len(w.src) <= 64000
        z = w.src[:, 2]
        lay = (z[:, None] < d[None, :]).sum(1)
        for l, (lo, hi) in enumerate(w.zext):
            zl = z[lay == l]
            assert len(zl) > 0 and zl.min() >= lo and zl.max() <= hi
            if l > 0:
                assert hi <= d[l - 1] - 0.1 + 1e-12
            if l < nl - 1:
                assert lo >= d[l] + 0.1 - 1e-12
    total = sum(len(w.src) for w in W.batched_instances(256))
    assert 3.0e6 < total < 4.5e6


def test_three_layer_slabs_recipe():
    w = W.three_layer_slabs(3000, 4, 64, seed=1)
    z = w.src[:, 2]
    for (lo, hi) in w.zext:
        assert np.count_nonzero((z >= lo) & (z <= hi)) == 1000
    assert np.all(np.abs(w.src[:, :2]) <= 2.0)
