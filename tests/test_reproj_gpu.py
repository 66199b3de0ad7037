"""Temporal reprojection (Sec. 4.3) through the C-ABI against the oracle.

Both sides gather each pixel's history from the previous frame's reservoirs
through the same motion vectors and depth test, so every plane must match bit
for bit after every frame. The frames come from the panning 2.5-D scene
(foveated on the CPU by the oracle), with parallax, screen-edge entries and
disk wrap-arounds producing flushes.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2510_03964_gb300 as wrs
from parity import check_resolve, compare_states
from synth import PanScene, gaze_path, workload

pytestmark = pytest.mark.gpu


class ReprojRun:
    def __init__(self, w, h, K, radii, frames, seed=0, velocity=(3.25, 0.75), color_fp16=False,
                 temporal_bias=True, update_rule=0, depth=True, motion=True, tol=0.05,
                 flush_every=0):
        self.scene = PanScene(w, h, seed=seed, velocity=velocity)
        self.gaze = gaze_path(w, h, frames, seed=seed, model="jitter", jitter_px=w / 4)
        self.radii = radii
        self.w, self.h, self.K = w, h, K
        self.fp16 = color_fp16
        self.use_depth, self.use_motion, self.tol = depth, motion, tol
        self.flush_every = flush_every
        self.gpu = wrs.Stream(w, h, K, radii[0], seed=seed, color_fp16=color_fp16,
                              temporal_bias=temporal_bias, update_rule=update_rule)
        self.gpu.set_reprojection_buffer()
        self.orc = oracle.OracleStream(w, h, K, radii[0], seed=seed, temporal_bias=temporal_bias,
                                       rule=update_rule, color_fp16=color_fp16, nthreads=8)
        self.prev_depth = None
        self.out = torch.empty((h, w, 3), device="cuda")

    def step(self, t, reproject=True):
        img, mv, depth = (a.numpy() for a in self.scene.render(t))
        g = self.gaze[t]
        frame, ring = oracle.foveate(img, self.radii, g[0], g[1], oracle.FILTER_BILINEAR)
        if self.flush_every and t % self.flush_every == self.flush_every - 1:
            ring = ring.copy()
            ring[::3, ::2] = 0xFF
        mv = mv if self.use_motion else None
        d, pd = (depth, self.prev_depth) if (self.use_depth and self.prev_depth is not None) else (None, None)
        dev = {k: (None if v is None else torch.from_numpy(np.ascontiguousarray(v)).cuda())
               for k, v in (("frame", frame), ("mv", mv), ("d", d), ("pd", pd), ("ring", ring))}
        if reproject and t > 0:
            self.gpu.push_frame_reproject(dev["frame"], g, dev["mv"], dev["d"], dev["pd"], self.tol,
                                          dev["ring"], self.out)
            self.orc.push_frame_reproject(frame, g, mv, d, pd, self.tol, ring)
        else:
            self.gpu.push_frame(dev["frame"], g, dev["ring"], self.out)
            self.orc.push_frame(frame, g, ring)
        self.prev_depth = depth

    def compare(self, check_out=True):
        assert self.gpu.check_status() == 0, "a wait gave up or the checked build skipped an access"
        torch.cuda.synchronize()
        o = self.orc.state()
        compare_states(self.gpu.export_state(), o, None, self.fp16)
        if check_out:
            check_resolve(self.out.cpu().numpy(), self.orc, o, self.fp16)


@pytest.mark.parametrize("opts", [
    {},
    {"color_fp16": True},
    {"K": 1, "update_rule": 1},
    {"K": 1},
    {"K": 2, "color_fp16": True},
    {"K": 3, "temporal_bias": 2},
    {"depth": False},
    {"motion": False},
    {"flush_every": 3},
    {"K": 16, "velocity": (-7.5, 2.25)},
])
def test_reprojected_stream_bit_exact(opts):
    kw = dict(K=4, velocity=(3.25, 0.75))
    kw.update(opts)
    K = kw.pop("K")
    run = ReprojRun(96, 64, K, (8.0, 20.0, 35.0), frames=12, seed=7, **kw)
    for t in range(12):
        run.step(t)
        run.compare()


@pytest.mark.parametrize("wh", [(37, 23), (1, 1), (5, 2)])
def test_ragged_sizes(wh):
    w, h = wh
    run = ReprojRun(w, h, 4, (max(1.0, w / 6), max(2.0, w / 3)), frames=8, seed=2,
                    velocity=(1.5, -0.5))
    for t in range(8):
        run.step(t)
    run.compare()


def test_mixed_plain_and_reprojected_pushes():
    # buffers swap only on reprojected pushes; plain pushes act on whichever
    # buffer holds the current reservoirs
    run = ReprojRun(64, 40, 4, (6.0, 15.0), frames=10, seed=3)
    for t, rp in enumerate([False, True, True, False, True, False, False, True, True, True]):
        run.step(t, reproject=rp)
        run.compare()


def test_export_import_and_detach_with_state_in_the_spare():
    run = ReprojRun(48, 32, 4, (6.0, 15.0), frames=6, seed=4)
    for t in range(4):
        run.step(t)  # three reprojected pushes: the current state sits in the spare
    run.compare()
    raw = run.gpu.export_raw()
    st2 = wrs.Stream(48, 32, 4, 6.0, seed=4)
    st2.import_raw(raw, run.gpu.frame_index)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(st2.export_raw(), raw)
    run.gpu.set_reprojection_buffer(None)  # copies the current reservoirs home
    run.compare()
    run.gpu.set_reprojection_buffer()
    run.step(4)
    run.step(5)
    run.compare()


def test_errors():
    st = wrs.Stream(16, 8, 4, 3.0)
    fr = torch.zeros((8, 16, 3), device="cuda")
    with pytest.raises(wrs.WrsError, match="spare"):
        st.push_frame_reproject(fr, (8.0, 4.0))
    st.set_reprojection_buffer()
    d = torch.ones((8, 16), device="cuda")
    with pytest.raises(wrs.WrsError, match="together"):
        st.push_frame_reproject(fr, (8.0, 4.0), depth=d)
    with pytest.raises(wrs.WrsError, match="depth_tol"):
        st.push_frame_reproject(fr, (8.0, 4.0), depth=d, prev_depth=d, depth_tol=-1.0)
    with pytest.raises(wrs.WrsError, match="BUDGET|holds"):
        st.set_reprojection_buffer(torch.empty(256, dtype=torch.uint8, device="cuda"))
    assert st.frame_index == 0


def test_4k_pan_frames_bit_exact():
    # full 4K frames of the pan workload through the bench's entry point
    s = workload("4k_pan").streams[0]
    run = ReprojRun(s.width, s.height, s.K, s.radii, frames=3, seed=s.seed,
                    velocity=s.pan_velocity)
    for t in range(3):
        run.step(t)
    run.compare()
