"""The host-buffer push that allocates nothing (wrs_push_frame_host_noalloc)
against the existing host-buffer push (wrs_push_frame_host): the same outputs
and reservoirs, bit for bit, on two calls in a row. Collected last, so it also
runs after every other test has used the library."""
import numpy as np
import pytest
import torch

import paper_2510_03964_gb300 as wrs
from synth import Foveator, gaze_path

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("with_fov", [False, True])
def test_noalloc_equals_host_push_on_two_calls(with_fov):
    w, h, K = 160, 90, 4
    fv = Foveator(w, h, (10.0, 25.0), seed=2)
    gz = gaze_path(w, h, 2, seed=2, model="jitter", jitter_px=8.0)
    a = wrs.Stream(w, h, K, 10.0, seed=11)
    b = wrs.Stream(w, h, K, 10.0, seed=11)
    d_in = torch.empty((h, w, 3), device="cuda")
    d_out = torch.empty((h, w, 3), device="cuda")
    d_fov = torch.empty((h, w), dtype=torch.uint8, device="cuda")
    for t in range(2):
        frame = fv.frame(*gz[t])[0].contiguous().pin_memory()
        fov = None
        if with_fov:
            fov = torch.zeros((h, w), dtype=torch.uint8)
            fov[20:40, 30:90] = 0xFF if t == 1 else 0
            fov = fov.pin_memory()
        out_a = torch.full((h, w, 3), -1.0).pin_memory()
        out_b = torch.full((h, w, 3), -2.0).pin_memory()
        a.push_frame_host_noalloc(frame, gz[t], out_a, h_fov_map=fov)
        b.push_frame_host(frame, gz[t], out_b, d_in, d_out, h_fov_map=fov,
                          d_fov_stage=d_fov if with_fov else None)
        assert torch.equal(out_a.view(torch.int32), out_b.view(torch.int32)), f"call {t}"
    assert a.frame_index == b.frame_index == 2
    assert np.array_equal(a.export_raw(), b.export_raw())


def test_noalloc_steady_calls_take_no_device_memory():
    # the first call on the device maps the library's staging array (the
    # runtime backs it when the module loads); later calls must not change the
    # device's free memory: any device allocation takes at least a 2 MB page
    w, h, K = 160, 90, 4
    fv = Foveator(w, h, (10.0, 25.0), seed=4)
    gz = gaze_path(w, h, 3, seed=4, model="jitter", jitter_px=8.0)
    st = wrs.Stream(w, h, K, 10.0, seed=13)
    frames = [fv.frame(*gz[t])[0].contiguous().pin_memory() for t in range(3)]
    out = torch.empty((h, w, 3)).pin_memory()
    st.push_frame_host_noalloc(frames[0], gz[0], out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for t in (1, 2):
        st.push_frame_host_noalloc(frames[t], gz[t], out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free0 - free1) < (1 << 20), (free0, free1)
    assert st.frame_index == 3


def test_noalloc_rejects_frames_above_its_staging():
    st = wrs.Stream(8294401, 1, 1, 5.0)
    h_frame = torch.zeros((1, 8294401, 3))
    h_out = torch.zeros((1, 8294401, 3))
    with pytest.raises(wrs.WrsError, match="static staging"):
        st.push_frame_host_noalloc(h_frame, (1.0, 0.5), h_out)
    assert st.frame_index == 0
