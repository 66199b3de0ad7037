"""The benchmark's resolve-error report (CPU): the oracle leg compares a
stream's resolved colours with the oracle's FP64 resolve of the exact colours.
A second oracle stream stands in for the GPU here, with a planted relative
error, so the report's arithmetic is checked without a device."""
import numpy as np
import pytest
import torch

import bench
import oracle
from synth import Foveator, frame_pixels, gaze_path, workload


def _run(scale):
    spec = workload("tiny").streams[0]
    fv = Foveator(spec.width, spec.height, spec.radii, seed=spec.seed, device="cpu")
    gaze = gaze_path(spec.width, spec.height, spec.frames, seed=spec.seed, model=spec.gaze_model,
                     jitter_px=spec.jitter_px)
    pixels = bench.sample_pixels(spec, 2048)
    twin = oracle.OracleStream(spec.width, spec.height, spec.K, spec.r_f, seed=spec.seed,
                               stream_id=spec.stream_id, temporal_bias=spec.temporal_bias,
                               pixels=pixels, rule=spec.update_rule)
    host = np.zeros((spec.height, spec.width, 3), np.float32)

    def stand_in(t, g):
        host.reshape(-1, 3)[pixels] = frame_pixels(fv, float(g[0]), float(g[1]),
                                                   torch.as_tensor(pixels)).numpy()
        twin.push_frame(host, g)
        return twin.resolve() * scale

    return bench.oracle_ms_per_frame(spec, pixels, 4, 1, fv, gaze, gpu_out=stand_in)


def test_identical_stream_reports_zero_error():
    ms, frames, err = _run(1.0)
    assert ms > 0 and frames == 4
    assert err["max_abs"] == 0.0 and err["max_rel"] == 0.0 and err["within_tolerance"]
    assert err["pixels"] == 2048 and err["colour_storage"] == "fp32"


@pytest.mark.parametrize("scale,ok", [(1 + 3e-6, True), (1 + 3e-5, False)])
def test_planted_relative_error_is_measured(scale, ok):
    _, _, err = _run(scale)
    assert err["max_rel"] == pytest.approx(scale - 1, rel=1e-3)
    assert err["within_tolerance"] is ok
