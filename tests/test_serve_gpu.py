"""Serving on the GPU: continuous batching and the plain path serve the same
trace; every viewer's reservoirs are bit-identical to serving it alone; the
HBM budget queues viewers that do not fit, or parks idle ones in host memory
(wrs_export_state / wrs_import_state) to admit them."""
import numpy as np
import pytest
import torch

from paper_2510_03964_gb300 import serve

pytestmark = pytest.mark.gpu

SMALL = ((64, 32, (6.0, 15.0)), (96, 40, (8.0, 20.0)), (128, 24, (10.0, 25.0)), (32, 16, (4.0, 10.0)))


@pytest.mark.parametrize("source", ["frames", "render"])
@pytest.mark.parametrize("mode,single_direct", [("batched", True), ("batched", False), ("plain", True)])
def test_served_viewers_equal_alone(mode, single_direct, source):
    # "render": every request's frame is foveated on the device from its
    # class's image (foveate + batched update, or the update foveating on read).
    # single_direct: a launch of one frame is the viewer's own update, or
    # (False) every launch is a batch, even of one.
    dev = torch.device("cuda")
    specs = serve.viewer_mix(12, 1.5, seed=1, rate_hz=(150.0, 300.0), classes=SMALL)
    trace = serve.arrivals(specs, seed=1)
    pool = (serve.RenderPool(SMALL, 6, dev, seed=1) if source == "render"
            else serve.FramePool(SMALL, 6, dev, seed=1))
    srv = serve.Server(specs, pool, budget_bytes=10**10, mode=mode, device=dev, keep_states=True,
                       single_direct=single_direct)
    stats = srv.run(trace, 1.5)
    s = stats.summary()
    assert stats.frames_served + stats.frames_rejected + stats.frames_shed == len(trace)
    assert stats.frames_served > 0 and s["p99_ms"] >= s["p50_ms"] > 0
    if mode == "batched":
        assert s["frames_per_launch"] >= 1.0
        if not single_direct:
            assert s["single_frame_launches"] == 0
    for vid, st in srv.kept.items():
        # the viewer's reservoirs and its last resolved frame, alone and in the mix
        alone, out = serve.replay_alone(srv.specs[vid], srv.pushed[vid], pool, device=dev)
        torch.cuda.synchronize()
        assert st.frame_index == alone.frame_index == len(srv.pushed[vid])
        assert np.array_equal(st.export_raw(), alone.export_raw()), f"viewer {vid}"
        if srv.pushed[vid]:
            assert torch.equal(srv.kept_out[vid].view(torch.int32), out.view(torch.int32)), f"viewer {vid}"
        alone.close()
    srv.close()


@pytest.mark.parametrize("mode", ["batched", "plain"])
def test_overload_sheds_late_frames_and_bounds_latency(mode):
    # far more frames than the GPU can take: frames that wait longer than the
    # deadline are dropped on the host, so the served frames' latency stays
    # near the deadline instead of growing with the queue
    dev = torch.device("cuda")
    big = ((1920, 1080, (120.0, 300.0)),)
    specs = serve.viewer_mix(24, 1.5, seed=4, rate_hz=(900.0, 900.0), classes=big)
    trace = serve.arrivals(specs, seed=4)
    pool = serve.FramePool(big, 4, dev, seed=4)
    srv = serve.Server(specs, pool, budget_bytes=10**11, mode=mode, device=dev, deadline_ms=10.0,
                       n_streams=4, depth=3)
    stats = srv.run(trace, 1.5)
    s = stats.summary()
    assert stats.frames_served + stats.frames_rejected + stats.frames_shed == len(trace)
    assert stats.frames_shed > 0 and stats.frames_served > 0
    # a served frame waited at most the deadline before its launch, then its
    # launch and at most the launches queued ahead of it
    assert s["p99_ms"] < 60.0, s
    srv.close()


def test_budget_queues_viewers():
    dev = torch.device("cuda")
    specs = serve.viewer_mix(8, 1.0, seed=2, rate_hz=(100.0, 100.0), classes=SMALL)
    trace = serve.arrivals(specs, seed=2)
    pool = serve.FramePool(SMALL, 4, dev, seed=2)
    budget = max(v.state_bytes() for v in specs) * 2  # room for about two viewers
    srv = serve.Server(specs, pool, budget_bytes=budget, mode="batched", device=dev)
    stats = srv.run(trace, 1.0)
    assert stats.peak_state_bytes <= budget
    assert stats.viewers_queued_max > 0 and stats.frames_rejected > 0
    assert stats.frames_served + stats.frames_rejected == len(trace)
    srv.close()


def _phased_trace(vids_by_phase, phase_s, rate_hz):
    # viewers take turns: in phase i only vids_by_phase[i % len] send frames
    ev = []
    n = int(round(phase_s * rate_hz))
    for i, vids in enumerate(vids_by_phase):
        for vid in vids:
            for k in range(n):
                ev.append((i * phase_s + (k + 0.5 + 0.1 * vid) / rate_hz, vid))
    ev.sort()
    return ev


@pytest.mark.parametrize("mode", ["batched", "plain"])
def test_budget_parks_idle_viewers_and_restores_them_bit_exact(mode):
    # four viewers, room for two: viewers 0, 1 and 2, 3 take turns sending
    # frames. A waiting viewer is admitted by parking idle ones in host memory;
    # a parked viewer whose frame is due is restored by parking others. Every
    # viewer's reservoirs and last resolved frame equal those of the viewer
    # served alone with the same frames.
    dev = torch.device("cuda")
    w, h, radii = SMALL[1]
    phases = [(0, 1), (2, 3), (0, 1), (2, 3)]
    phase_s, duration = 0.25, 1.0
    specs = [serve.ViewerSpec(vid=i, width=w, height=h, K=8 if i % 2 == 0 else 4, radii=radii, seed=i + 1,
                              rate_hz=200.0, join_s=0.0, leave_s=duration, cls=0) for i in range(4)]
    trace = _phased_trace(phases, phase_s, 200.0)
    pool = serve.FramePool((SMALL[1],), 4, dev, seed=3)
    budget = 2 * max(v.state_bytes() + v.frame_bytes() for v in specs)
    srv = serve.Server(specs, pool, budget_bytes=budget, mode=mode, device=dev, keep_states=True,
                       park_idle_ms=40.0)
    stats = srv.run(trace, duration)
    s = stats.summary()
    assert stats.frames_served + stats.frames_rejected + stats.frames_shed == len(trace)
    assert stats.peak_device_bytes <= budget
    assert s["viewers_parked"] >= 2 and s["viewers_restored"] >= 1, s
    assert set(srv.kept) == {0, 1, 2, 3}
    for vid, st in srv.kept.items():
        alone, out = serve.replay_alone(srv.specs[vid], srv.pushed[vid], pool, device=dev)
        torch.cuda.synchronize()
        assert st.frame_index == alone.frame_index == len(srv.pushed[vid])
        assert np.array_equal(st.export_raw(), alone.export_raw()), f"viewer {vid}"
        if srv.pushed[vid]:
            assert torch.equal(srv.kept_out[vid].view(torch.int32), out.view(torch.int32)), f"viewer {vid}"
        alone.close()
    srv.close()
