"""Pipelined host-buffer frames (wrs_host_pipe_*): every frame's resolved
output and the final reservoirs equal the synchronous host path's, bit for
bit, whatever overlap the three streams achieve."""
import numpy as np
import pytest
import torch

import paper_2510_03964_gb300 as wrs
from synth import Foveator, gaze_path

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("with_fov,color_fp16", [(False, False), (True, False), (False, True)])
def test_pipeline_equals_synchronous_host_path(with_fov, color_fp16):
    w, h, K, frames = 96, 64, 4, 9
    fv = Foveator(w, h, (8.0, 20.0), seed=3)
    gz = gaze_path(w, h, frames, seed=3, model="jitter", jitter_px=10.0)
    h_frames = [fv.frame(*gz[t])[0].contiguous().pin_memory() for t in range(frames)]
    h_fovs = []
    for t in range(frames):
        m = torch.zeros((h, w), dtype=torch.uint8)
        if with_fov and t == 5:
            m[10:30, 20:60] = 0xFF
        h_fovs.append(m.pin_memory())
    a = wrs.Stream(w, h, K, 8.0, seed=4, color_fp16=color_fp16)
    b = wrs.Stream(w, h, K, 8.0, seed=4, color_fp16=color_fp16)
    pipe = wrs.HostPipeline(a, with_fov=with_fov)
    outs_a = [torch.empty((h, w, 3)).pin_memory() for _ in range(frames)]
    for t in range(frames):
        pipe.push(h_frames[t], gz[t], outs_a[t], h_fovs[t] if with_fov else None)
    pipe.finish()
    d_in = torch.empty((h, w, 3), device="cuda")
    d_out = torch.empty((h, w, 3), device="cuda")
    d_fov = torch.empty((h, w), dtype=torch.uint8, device="cuda")
    for t in range(frames):
        out_b = torch.empty((h, w, 3)).pin_memory()
        b.push_frame_host(h_frames[t], gz[t], out_b, d_in, d_out,
                          h_fov_map=h_fovs[t] if with_fov else None, d_fov_stage=d_fov if with_fov else None)
        assert torch.equal(outs_a[t].view(torch.int32), out_b.view(torch.int32)), f"frame {t}"
    assert a.frame_index == b.frame_index == frames
    assert np.array_equal(a.export_raw(), b.export_raw())
    pipe.close()


def test_pipeline_reuses_host_buffers_after_three_frames():
    # the pipeline waits for frame n-3 before enqueuing frame n, so a caller
    # cycling four host buffers never overwrites one still in flight
    w, h, K = 64, 32, 4
    fv = Foveator(w, h, (6.0, 15.0), seed=5)
    gz = gaze_path(w, h, 14, seed=5, model="jitter", jitter_px=5.0)
    a = wrs.Stream(w, h, K, 6.0, seed=6)
    b = wrs.Stream(w, h, K, 6.0, seed=6)
    pipe = wrs.HostPipeline(a)
    ring_in = [torch.empty((h, w, 3)).pin_memory() for _ in range(4)]
    ring_out = [torch.empty((h, w, 3)).pin_memory() for _ in range(4)]
    d_in = torch.empty((h, w, 3), device="cuda")
    d_out = torch.empty((h, w, 3), device="cuda")
    for t in range(14):
        if t >= 4:
            # frame t-4's output is complete: check it before its buffer is reused
            ref = torch.empty((h, w, 3)).pin_memory()
            b.push_frame_host(fv.frame(*gz[t - 4])[0].contiguous(), gz[t - 4], ref, d_in, d_out)
            assert torch.equal(ring_out[t % 4].view(torch.int32), ref.view(torch.int32)), f"frame {t - 4}"
        ring_in[t % 4].copy_(fv.frame(*gz[t])[0])
        pipe.push(ring_in[t % 4], gz[t], ring_out[t % 4])
    pipe.finish()
    pipe.close()
