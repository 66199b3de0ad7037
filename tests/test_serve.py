"""Serving workload generation (no GPU): viewer mix and Poisson arrival traces."""
import numpy as np

from paper_2510_03964_gb300 import serve


def test_viewer_mix_shapes():
    sp = serve.viewer_mix(64, 60.0, seed=0)
    assert len(sp) == 64
    assert {(v.width, v.height) for v in sp} == {(c[0], c[1]) for c in serve.CLASSES}
    assert [v.K for v in sp[:4]] == [8, 4, 8, 4]
    for v in sp:
        assert 72.0 <= v.rate_hz <= 120.0
        assert 0.0 <= v.join_s < v.leave_s <= 60.0
        assert v.color_fp16
    assert sp[0].state_bytes() > sp[1].state_bytes()  # K = 8 vs 4 at 4K


def test_arrivals_are_poisson_per_viewer():
    sp = serve.viewer_mix(8, 200.0, seed=3)
    tr = serve.arrivals(sp, seed=3)
    assert all(a[0] <= b[0] for a, b in zip(tr, tr[1:]))
    assert tr == serve.arrivals(sp, seed=3)
    for v in sp:
        ts = np.array([t for t, vid in tr if vid == v.vid])
        assert np.all((ts > v.join_s) & (ts < v.leave_s))
        gaps = np.diff(ts)
        rate = 1.0 / gaps.mean()
        assert abs(rate - v.rate_hz) < 0.1 * v.rate_hz
        # exponential gaps: coefficient of variation near 1
        assert 0.85 < gaps.std() / gaps.mean() < 1.15
