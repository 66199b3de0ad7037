"""Failure detection without a GPU fault: a device-side wait that runs out
returns an error status the host reads, and the context stays usable.

The pipelined kernel's copy barriers are bounded by a wall-clock limit. With
``test_extra_tx`` each barrier expects a few bytes more than are copied, so it
can never complete: the kernel must give up after the (short) limit, record
WRS_ERR_TIMEOUT, let its copies land and return. No trap, no fault, no hang.
"""
import numpy as np
import pytest
import torch

import paper_2510_03964_gb300 as wrs
from paper_2510_03964_gb300._lib import WRS_ERR_TIMEOUT, WRS_OK

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_recovers():
    dev = torch.device("cuda")
    W, H, K = 256, 64, 4
    st = wrs.Stream(W, H, K, 16.0, seed=1, device=dev)
    assert st.get_pipeline()[0], "the pipelined kernel must be selected for this frame shape"
    frame = torch.rand((H, W, 3), device=dev)
    out = torch.empty_like(frame)
    st.push_frame(frame, (100.0, 30.0), out=out)
    assert st.check_status() == WRS_OK
    snap = st.export_raw()
    st.set_wait_limit(timeout_ns=2_000_000, test_extra_tx=16)  # 2 ms, barriers never complete
    st.push_frame(frame, (100.0, 30.0), out=out)
    assert st.check_status() == WRS_ERR_TIMEOUT
    assert "gave up" in wrs.load().wrs_last_error().decode()
    assert st.check_status() == WRS_OK  # the word was cleared
    # the reservoirs are undefined: pushes are refused until a state is imported
    with pytest.raises(wrs.WrsError):
        st.push_frame(frame, (100.0, 30.0), out=out)
    st.set_wait_limit(0, 0)
    st.import_raw(snap, 1)
    st.push_frame(frame, (100.0, 30.0), out=out)
    torch.cuda.synchronize()
    assert st.check_status() == WRS_OK
    assert torch.isfinite(out).all()
    st.close()


def test_wait_limit_arguments():
    st = wrs.Stream(64, 8, 2, 4.0, device=torch.device("cuda"))
    with pytest.raises(wrs.WrsError):
        st.set_wait_limit(61 * 10 ** 9, 0)
    with pytest.raises(wrs.WrsError):
        st.set_wait_limit(10 ** 6, 5000)
    st.close()


def test_timed_out_push_is_refused_until_a_saved_state_is_restored():
    """A timed-out push leaves the reservoirs undefined. After the host has
    seen the timeout, the library refuses further pushes (WRS_ERR_STATE)
    until wrs_import_state restores a saved state. Pushing the same frames
    again then gives the oracle's reservoirs bit for bit."""
    from parity import PairedRun, compare_states
    from paper_2510_03964_gb300._lib import WRS_ERR_STATE
    run = PairedRun(256, 64, 4, 16.0, frames=8, seed=3)
    for t in range(3):
        run.step(t)
    torch.cuda.synchronize()
    snap = run.gpu.export_raw()
    st = run.gpu
    gx, gy = run.gaze[3]
    fr, _ = run.fv.frame(float(gx), float(gy))
    fr = fr.to("cuda").contiguous()
    st.set_wait_limit(timeout_ns=2_000_000, test_extra_tx=16)
    st.push_frame(fr, (gx, gy))          # its waits give up
    st.push_frame(fr, (gx, gy))          # enqueued before the host knows: left alone on the device
    assert st.check_status() == WRS_ERR_TIMEOUT
    with pytest.raises(wrs.WrsError) as e:
        st.push_frame(fr, (gx, gy))
    assert e.value.code == WRS_ERR_STATE
    with pytest.raises(wrs.WrsError):
        st.resolve()
    assert st.frame_index == 5
    st.set_wait_limit(0, 0)
    st.import_raw(snap, 3)
    assert st.frame_index == 3
    for t in range(3, 8):
        run.step(t)
    torch.cuda.synchronize()
    assert st.check_status() == WRS_OK
    run.compare()
