"""CUDA path (through the C-ABI) against the CPU oracle, element by element.

Reservoir planes must match bit for bit; resolved colours within the
tolerance stated in tests/parity.py. Sizes run from one pixel to full 4K; the
4K and HD streams use the same launch configuration as bench.py and compare
a sample of pixels that the oracle simulates one by one (every pixel is an
independent stream, so a sample evolves exactly as inside the full frame).
"""
import numpy as np
import pytest
import torch

import oracle
from parity import PairedRun, assert_bits_equal, check_resolve, compare_states
from synth import workload

pytestmark = pytest.mark.gpu


def _sample_pixels(w, h, n, seed):
    rng = np.random.default_rng(seed)
    pix = set(rng.choice(w * h, size=n, replace=False).tolist())
    # whole rows through the image centre and the last row, first/last pixels
    for y in (0, h // 2, h - 1):
        pix.update(range(y * w, y * w + w))
    pix.update([0, w * h - 1])
    return np.array(sorted(pix), np.int64)


def test_tiny_workload_bit_exact():
    s = workload("tiny").streams[0]
    run = PairedRun(s.width, s.height, s.K, s.r_f, radii=s.radii, frames=s.frames, seed=s.seed,
                    gaze_model=s.gaze_model, jitter_px=s.jitter_px)
    for t in range(s.frames):
        run.step(t)
        torch.cuda.synchronize()
        run.compare()  # every frame, including frame 0 (all inserts)


@pytest.mark.parametrize("K", [1, 2, 3, 4, 5, 8, 16])
@pytest.mark.parametrize("wh", [(37, 23), (64, 20), (1, 1), (3, 1)])
def test_k_and_ragged_sizes(K, wh):
    w, h = wh
    run = PairedRun(w, h, K, r_f=max(1.0, w / 6), frames=K + 5, seed=K, stream_id=K,
                    jitter_px=w / 3)
    run.run()
    run.compare()


@pytest.mark.parametrize("launch", [(64, 1), (128, 2), (256, 4), (96, 4), (256, 1)])
@pytest.mark.parametrize("K", [4, 8, 6])
def test_launch_shapes_agree(launch, K):
    run = PairedRun(96, 40, K, r_f=10.0, frames=12, seed=3, launch=launch, jitter_px=20)
    run.run()
    run.compare()


@pytest.mark.parametrize("pipeline", [(True, 1, 1, 0), (True, 1, 4, 0), (True, 2, 2, 0), (True, 4, 2, 0),
                                      (True, 2, 3, 0), (True, 1, 2, 1), (True, 1, 2, 3),
                                      (False, 0, 0, 0)])
@pytest.mark.parametrize("K,fp16", [(4, False), (8, False), (3, False), (8, True), (1, True)])
def test_pipeline_shapes_agree(pipeline, K, fp16):
    """The pipelined kernel (tiles of 256*px pixels through `stages` shared-memory
    stages; 3840 pixels = a ragged last tile for every tile size) and the plain
    kernel give the same planes. Shapes the library rejects for shared memory
    are skipped."""
    import paper_2510_03964_gb300 as wrs
    try:
        run = PairedRun(96, 40, K, r_f=10.0, frames=12, seed=5, jitter_px=20, color_fp16=fp16,
                        pipeline=pipeline)
    except wrs.WrsError as e:
        assert "shared memory" in str(e)
        pytest.skip("these stages do not fit in shared memory")
    run.run()
    run.compare()


def test_pipeline_rejects_oversized_stages():
    import paper_2510_03964_gb300 as wrs
    st = wrs.Stream(64, 16, 8, 8.0, device=torch.device("cuda"))
    with pytest.raises(wrs.WrsError):
        st.set_pipeline(True, 4, 2)  # 2 x 184 KB
    st.set_pipeline(True, 2, 2)
    assert st.get_pipeline() == (True, 2, 2, 0)
    st.set_pipeline(True, 1, 3, 1)
    assert st.get_pipeline() == (True, 1, 3, 1)
    st.close()


@pytest.mark.parametrize("K,fp16,px,stages", [(8, False, 1, 2), (8, True, 1, 3), (4, False, 1, 4),
                                               (4, True, 1, 4), (16, False, 1, 2), (1, False, 2, 4),
                                               (2, True, 2, 4)])
def test_default_stages_keep_two_ctas_per_sm(K, fp16, px, stages):
    # as many stages (up to four) as keep two CTAs on an SM, else what one CTA
    # holds; one or two slots take two pixels per thread
    import paper_2510_03964_gb300 as wrs
    st = wrs.Stream(64, 16, K, 8.0, color_fp16=fp16, device=torch.device("cuda"))
    assert st.get_pipeline() == (True, px, stages, 0)
    st.set_pipeline(True, 0, 0)
    assert st.get_pipeline() == (True, px, stages, 0)
    st.close()


def test_pipeline_many_tiles_per_cta():
    """More tiles than CTAs: every CTA walks several tiles through its stages."""
    run = PairedRun(640, 480, 4, r_f=40.0, frames=6, seed=8, jitter_px=60, pipeline=(True, 2, 3, 0),
                    pixels=np.arange(0, 640 * 480, 7))
    run.run()
    run.compare()


def test_pipeline_without_fused_resolve():
    """Without an output the pipelined kernel copies only frame, W, P and keys."""
    run = PairedRun(128, 32, 8, r_f=12.0, frames=9, seed=13, jitter_px=30)
    for t in range(9):
        run.step(t, fused=(t == 8))
    torch.cuda.synchronize()
    run.compare()


@pytest.mark.parametrize("K", [1, 4, 8, 3])
def test_fp16_colour(K):
    run = PairedRun(128, 72, K, r_f=12.0, frames=10, seed=11, color_fp16=True, jitter_px=25)
    run.run()
    _, _, err = run.compare()
    assert err <= 2.0 ** -11


@pytest.mark.parametrize("K", [1, 4])
def test_without_temporal_bias(K):
    run = PairedRun(80, 48, K, r_f=9.0, frames=14, seed=2, temporal_bias=False, jitter_px=15)
    run.run()
    run.compare()


def test_flush_map():
    run = PairedRun(64, 32, 4, r_f=6.0, frames=10, seed=9, jitter_px=10)
    rng = np.random.default_rng(0)
    for t in range(10):
        fm = rng.integers(0, 4, size=(32, 64), dtype=np.uint8)
        if t in (3, 7):
            fm[rng.random((32, 64)) < 0.3] = 0xFF
        run.step(t, fov_map=fm)
    torch.cuda.synchronize()
    run.compare()


def test_padded_pitch_and_standalone_resolve():
    run = PairedRun(52, 30, 4, r_f=7.0, frames=9, seed=4, jitter_px=12)
    for t in range(9):
        run.step(t, pitch_pad=5 if t % 2 else 0, fused=(t != 8))
    torch.cuda.synchronize()
    g, o, _ = run.compare(check_out=False)
    out = run.gpu.resolve()
    torch.cuda.synchronize()
    check_resolve(out.cpu().numpy(), run.orc, o, False, "standalone resolve")
    # fused and standalone resolves agree bit for bit
    run2 = PairedRun(52, 30, 4, r_f=7.0, frames=9, seed=4, jitter_px=12)
    run2.run()
    out2 = run2.gpu.resolve()
    torch.cuda.synchronize()
    assert_bits_equal(out2.cpu().numpy(), run2.out.cpu().numpy(), "fused vs standalone")


def test_gaze_far_outside_and_eccentricity_clamp():
    gaze = np.array([[-5000.0, 30.0], [1e6, -1e6], [10.0, 10.0], [64.5, 0.0]], np.float32)
    run = PairedRun(64, 24, 3, r_f=4.0, deg_per_px=3.0, gaze=gaze, seed=6)
    run.run()
    run.compare()


def test_resolve_before_any_push_is_zero():
    run = PairedRun(16, 8, 2, r_f=2.0, frames=1)
    out = run.gpu.resolve()
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0
    g = run.gpu.export_state()
    assert np.all(g["idx"] == oracle.EMPTY) and np.all(np.isinf(g["key"]))
    assert np.all(g["W"] == 0) and np.all(g["P"] == 1)


def test_bias_product_rescale_on_device():
    """A long stream at full weight drives P below 2^-64, so the rescale path
    runs on the GPU; the planes must still match."""
    frames = 1200
    gaze = np.tile(np.float32([[8.0, 4.0]]), (frames, 1))  # whole image inside the fovea: w = 1
    run = PairedRun(16, 8, 4, r_f=40.0, gaze=gaze, seed=12)
    run.run()
    g, o, _ = run.compare()
    assert np.all(g["P"] < 1.0) and np.all(o["P"] >= 2.0 ** -64)


def test_hd_workload_sampled_pixels():
    s = workload("hd").streams[0]
    pix = _sample_pixels(s.width, s.height, 20000, 1)
    run = PairedRun(s.width, s.height, s.K, s.r_f, radii=s.radii, frames=s.frames, seed=s.seed,
                    gaze_model=s.gaze_model, jitter_px=s.jitter_px, pixels=pix, frame_device="cuda")
    run.run()
    g, _, _ = run.compare()
    occ = (g["idx"] != oracle.EMPTY).sum(axis=0)
    assert np.all(occ == s.K)  # after 120 frames every pixel's reservoir is full


@pytest.mark.parametrize("name", ["4k", "4k_fp16"])
def test_4k_workload_sampled_pixels(name):
    s = workload(name).streams[0]
    pix = _sample_pixels(s.width, s.height, 16384, 2)
    run = PairedRun(s.width, s.height, s.K, s.r_f, radii=s.radii, frames=s.frames, seed=s.seed,
                    gaze_model=s.gaze_model, jitter_px=s.jitter_px, pixels=pix,
                    color_fp16=s.color_fp16, frame_device="cuda")
    run.run()
    g, _, err = run.compare()
    assert np.all((g["idx"] != oracle.EMPTY).sum(axis=0) == s.K)
    assert np.all((g["W"] > 0) & np.isfinite(g["W"]))
    if s.color_fp16:
        assert err <= 2.0 ** -11


def test_oracle_philox_matches_curand_through_library_stream():
    """Keys come from Philox: the library's draws reproduce the oracle's
    uniforms, checked through the slot keys of a one-frame K=1 stream with
    w = 1 everywhere (key = -ln u)."""
    w, h = 64, 16
    gaze = np.float32([[32.0, 8.0]])
    run = PairedRun(w, h, 1, r_f=100.0, gaze=gaze, seed=0xDEADBEEF12345678, stream_id=77)
    run.run()
    g = run.gpu.export_state()
    u = oracle.uniforms(0xDEADBEEF12345678, 77, 0, 0, w * h)
    assert_bits_equal(g["key"][0], -oracle.log32(u), "keys = -ln u")


@pytest.mark.parametrize("pipeline", [(True, 0, 0, 0), (False, 0, 0, 0)])
@pytest.mark.parametrize("fp16", [False, True])
def test_replacement_counter_matches_oracle(pipeline, fp16):
    """The stream's replacement count equals the number of (pixel, frame)
    pairs whose candidate entered a slot, counted from the oracle's states."""
    run = PairedRun(96, 40, 4, r_f=10.0, frames=14, seed=21, jitter_px=20, color_fp16=fp16,
                    pipeline=pipeline)
    expected = 0
    rng = np.random.default_rng(5)
    for t in range(14):
        before = run.orc.idx.copy()
        fm = None
        if t == 9:
            fm = np.zeros((40, 96), np.uint8)
            fm[rng.random((40, 96)) < 0.2] = 0xFF
        run.step(t, fov_map=fm)
        expected += int((run.orc.idx == t).any(axis=1).sum())
        assert not np.any((run.orc.idx != before) & (run.orc.idx != t) & (run.orc.idx != oracle.EMPTY))
    torch.cuda.synchronize()
    run.compare()
    assert run.gpu.replacements() == expected


@pytest.mark.parametrize("pipeline", [(True, 0, 0, 0), (True, 2, 2, 0), (False, 0, 0, 0)])
@pytest.mark.parametrize("fp16", [False, True])
def test_literal_rule_bit_exact(pipeline, fp16):
    """The paper's n = 1 rule taken literally (rand * (R1 + R2) <= R1 keeps R1
    after Eq. temporal-bias): planes bit-exact with the oracle, every frame."""
    run = PairedRun(96, 40, 1, r_f=10.0, frames=10, seed=31, jitter_px=20, color_fp16=fp16,
                    pipeline=pipeline, update_rule=1)
    for t in range(10):
        fm = None
        if t == 6:
            fm = np.zeros((40, 96), np.uint8)
            fm[::3, ::5] = 0xFF
        run.step(t, fov_map=fm)
        torch.cuda.synchronize()
        run.compare()


@pytest.mark.parametrize("wh", [(37, 23), (1, 1), (5, 3)])
def test_literal_rule_ragged(wh):
    run = PairedRun(wh[0], wh[1], 1, r_f=3.0, frames=7, seed=32, jitter_px=5, update_rule=1)
    run.run()
    run.compare()


def test_literal_rule_4k_sampled():
    s = workload("4k").streams[0]
    pix = _sample_pixels(s.width, s.height, 8192, 3)
    run = PairedRun(s.width, s.height, 1, s.r_f, radii=s.radii, frames=60, seed=s.seed,
                    gaze_model=s.gaze_model, jitter_px=s.jitter_px, pixels=pix, frame_device="cuda",
                    update_rule=1)
    run.run()
    run.compare()


def test_literal_rule_matches_key_race_in_distribution():
    """With K = 1 the key race and the literal rule select with the same law:
    whole image inside the fovea (w = 1), 24 frames, the final sample's frame
    index over 12288 pixels (independent streams) is compared by a two-sample
    chi-square at alpha = 1e-3."""
    from scipy import stats
    import paper_2510_03964_gb300 as wrs
    w, h, frames = 128, 96, 24
    dev = torch.device("cuda")
    hist = []
    for rule, seed in ((0, 101), (1, 202)):
        st = wrs.Stream(w, h, 1, 1000.0, seed=seed, device=dev, update_rule=rule)
        fr = torch.zeros((h, w, 3), device=dev)
        for t in range(frames):
            st.push_frame(fr, (w / 2, h / 2))
        torch.cuda.synchronize()
        idx = st.export_state()["idx"][0].astype(np.int64)
        hist.append(np.bincount(idx, minlength=frames))
    # the law itself: with equal weights under the bias, later frames are favoured
    assert hist[0][-1] > hist[0][0] and hist[1][-1] > hist[1][0]
    table = np.array(hist)
    keep = table.sum(axis=0) >= 10
    res = stats.chi2_contingency(table[:, keep])
    assert res.pvalue > 1e-3


@pytest.mark.parametrize("K,rule,fp16,pipeline", [
    (1, 0, False, (True, 0, 0, 0)), (4, 0, False, (True, 0, 0, 0)), (8, 0, True, (True, 0, 0, 0)),
    (4, 0, False, (False, 0, 0, 0)), (1, 1, False, (True, 0, 0, 0)), (1, 1, True, (False, 0, 0, 0)),
    (3, 0, True, (True, 2, 2, 0))])
def test_full_temporal_bias_bit_exact(K, rule, fp16, pipeline):
    """Eq. (full-temporal-bias) across a scene cut at frame 6 (large Delta L):
    planes bit-exact with the oracle before, at and after the cut."""
    run = PairedRun(96, 40, K, r_f=10.0, frames=12, seed=41, jitter_px=20, color_fp16=fp16,
                    pipeline=pipeline, update_rule=rule, temporal_bias=2, switch_scene_at=6)
    for t in range(12):
        run.step(t)
        if t in (5, 6, 7, 11):
            torch.cuda.synchronize()
            run.compare()


@pytest.mark.parametrize("K,rule,fp16,pipeline", [
    (4, 0, False, (True, 0, 0, 0)), (8, 0, True, (True, 2, 2, 0)), (1, 1, False, (True, 0, 0, 0)),
    (3, 0, False, (False, 0, 0, 0))])
def test_full_temporal_bias_without_fused_resolve(K, rule, fp16, pipeline):
    """Eq. (full-temporal-bias) needs the slots' colours even when no output
    is written: pushes without `out` must give the same planes."""
    run = PairedRun(96, 40, K, r_f=10.0, frames=10, seed=43, jitter_px=20, color_fp16=fp16,
                    pipeline=pipeline, update_rule=rule, temporal_bias=2, switch_scene_at=5)
    for t in range(10):
        run.step(t, fused=False)
    torch.cuda.synchronize()
    run.compare(check_out=False)


def test_full_temporal_bias_4k_sampled():
    s = workload("4k").streams[0]
    pix = _sample_pixels(s.width, s.height, 8192, 4)
    run = PairedRun(s.width, s.height, s.K, s.r_f, radii=s.radii, frames=40, seed=s.seed,
                    gaze_model=s.gaze_model, jitter_px=s.jitter_px, pixels=pix, frame_device="cuda",
                    temporal_bias=2, switch_scene_at=20)
    run.run()
    run.compare()
