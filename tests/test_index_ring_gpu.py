"""Sample indices kept as per-frame replacement codes (a ring of one-byte
planes) and folded into the index planes a band of blocks at a time: whatever
the frame at which a state is exported, imported or reprojected, the index
planes must equal the oracle's, which writes every index directly (Alg. 2,
one sample per slot). Sizes span ragged final blocks, more frames than the
ring holds, flushes and every kernel path."""
import numpy as np
import pytest
import torch

import oracle
import paper_2510_03964_gb300 as wrs
from parity import PairedRun, compare_states

pytestmark = pytest.mark.gpu


def _flush_map(w, h, t):
    m = np.zeros((h, w), np.uint8)
    if t % 7 == 3:
        m[5:25, 40:120] = 0xFF
    return m


@pytest.mark.parametrize("shape,K,fp16,pipeline", [
    ((300, 70), 4, False, None),                 # pipelined kernel, ragged last block
    ((300, 70), 8, True, None),
    ((300, 70), 4, False, (False, 0, 0, 0)),     # plain kernel, 4 pixels per thread
    ((301, 67), 3, False, None),                 # odd width: plain kernel, generic K
    ((300, 70), 1, False, None),                 # one or two slots: indices written
    ((300, 70), 2, True, None),                  # directly, no ring
    ((301, 67), 2, False, (False, 0, 0, 0)),
])
def test_exports_at_any_frame_match_the_oracle(shape, K, fp16, pipeline):
    w, h = shape
    run = PairedRun(w, h, K, 12.0, frames=41, seed=5, color_fp16=fp16, pipeline=pipeline)
    checkpoints = {1, 5, 15, 16, 17, 31, 40}
    for t in range(41):
        run.step(t, fov_map=_flush_map(w, h, t))
        if t in checkpoints:
            torch.cuda.synchronize()
            run.compare()


def test_literal_rule_indices_over_many_frames():
    run = PairedRun(256, 96, 1, 10.0, frames=37, seed=9, update_rule=1)
    for t in range(37):
        run.step(t, fov_map=_flush_map(256, 96, t))
        if t in (16, 36):
            torch.cuda.synchronize()
            run.compare()


def test_import_mid_ring_then_continue():
    w, h, K = 320, 64, 4
    run = PairedRun(w, h, K, 12.0, frames=45, seed=11)
    for t in range(21):
        run.step(t)
    torch.cuda.synchronize()
    snap = run.gpu.export_raw()
    # a second context imports the state at frame 21 and both go on: the
    # imported indices are complete and the stale ring must not be applied
    twin = wrs.Stream(w, h, K, 12.0, seed=11)
    twin.import_raw(snap, 21)
    for t in range(21, 45):
        gx, gy = run.gaze[t]
        fr, _ = run.fv.frame(float(gx), float(gy))
        twin.push_frame(fr.to("cuda").contiguous(), (gx, gy))
        run.step(t)
    torch.cuda.synchronize()
    g, o, _ = run.compare(check_out=False)
    compare_states(twin.export_state(), o, None, False)
    twin.close()


def test_export_twice_without_pushes_is_stable():
    run = PairedRun(256, 64, 4, 10.0, frames=19, seed=2)
    run.run()
    a = run.gpu.export_raw()
    b = run.gpu.export_raw()
    assert np.array_equal(a, b)
    run.compare(check_out=False)
