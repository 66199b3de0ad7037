"""Foveation post-process kernels (Sec. 4.3) through the C-ABI against the oracle.

Mip texels, foveated frames and ring maps must match the oracle bit for bit:
both sides follow the same FP32 operation sequence (quad-tree block sums, one
division, the FP32 ring test and the bilinear weights). Sizes run from a
single pixel to full 4K, with ragged edges, padded pitches and gazes inside,
at the edge of and outside the image.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2510_03964_gb300 as wrs
from parity import check_resolve, compare_states
from synth import Foveator, ground_truth, workload

pytestmark = pytest.mark.gpu

FILTERS = (("box", oracle.FILTER_BOX), ("bilinear", oracle.FILTER_BILINEAR))


def _bits(a):
    return np.ascontiguousarray(a, np.float32).view(np.uint32)


def _assert_equal(got, ref, what):
    g, r = _bits(got), _bits(ref)
    bad = np.flatnonzero(g.reshape(-1) != r.reshape(-1))
    assert bad.size == 0, f"{what}: {bad.size} words differ, first at {bad[:5]}"


def _image(w, h, seed, pitch_pad=0):
    img = ground_truth(w, h, seed)
    if pitch_pad == 0:
        return img, torch.from_numpy(img).cuda()
    buf = torch.zeros((h, w + pitch_pad, 3), dtype=torch.float32, device="cuda")
    view = buf[:, :w, :]
    view.copy_(torch.from_numpy(img))
    return img, view


@pytest.mark.parametrize("wh", [(1, 1), (3, 2), (37, 21), (64, 32), (333, 129), (1000, 7)])
@pytest.mark.parametrize("levels", [2, 3, 4, 6])
def test_mip_levels_bit_exact(wh, levels):
    w, h = wh
    img, dimg = _image(w, h, seed=w + h)
    mip = wrs.mip_build(dimg, levels)
    torch.cuda.synchronize()
    for L, lv in enumerate(wrs.mip_levels(mip, w, h, levels), start=1):
        got = lv.cpu().numpy()
        _assert_equal(got[:, :, :3], oracle.mip_means(img, L), f"level {L} of {w}x{h}")
        assert np.all(got[:, :, 3] == 0.0)


def test_mip_padded_pitch_and_large():
    # pad 5: scalar staging; pad 4: 16-byte staging with a pitch; pad 0: packed rows
    for (w, h, pad) in ((1920, 1080, 5), (333, 77, 4), (3840, 2160, 0)):
        img, dimg = _image(w, h, seed=9, pitch_pad=pad)
        mip = wrs.mip_build(dimg, 4)
        torch.cuda.synchronize()
        for L, lv in enumerate(wrs.mip_levels(mip, w, h, 4), start=1):
            _assert_equal(lv.cpu().numpy()[:, :, :3], oracle.mip_means(img, L), f"{w}x{h} L{L}")


@pytest.mark.parametrize("name,f", FILTERS)
@pytest.mark.parametrize("case", [
    (37, 21, (4.0, 9.0), (10.3, 12.7)),
    (53, 29, (4.0, 9.0, 15.0), (0.0, 0.0)),           # gaze at a corner
    (64, 40, (5.0, 11.0, 17.0, 23.0, 30.0), (31.5, 20.0)),  # six levels, dyadic gaze
    (97, 31, (6.0, 14.0, 40.0), (-20.0, 50.0)),        # gaze outside the image
    (1, 1, (0.25,), (5.0, 5.0)),
    (5, 3, (1.0, 2.0, 3.0, 4.0, 5.0), (2.5, 1.5)),     # level-5 blocks larger than the image
])
def test_foveate_bit_exact(name, f, case):
    w, h, radii, gaze = case
    img, dimg = _image(w, h, seed=w * h)
    fov = wrs.Foveation(dimg, radii, filter=name)
    frame, ring = fov.frame(gaze)
    torch.cuda.synchronize()
    ref, ref_ring = oracle.foveate(img, radii, gaze[0], gaze[1], f)
    assert np.array_equal(ring.cpu().numpy(), ref_ring)
    _assert_equal(frame.cpu().numpy(), ref, f"{name} {w}x{h}")


@pytest.mark.parametrize("name,f", FILTERS)
def test_foveate_4k_full_frame(name, f):
    s = workload("4k").streams[0]
    img, dimg = _image(s.width, s.height, seed=s.seed)
    fov = wrs.Foveation(dimg, s.radii, filter=name)
    for gaze in ((1920.0, 1080.0), (3700.25, 100.5)):
        frame, ring = fov.frame(gaze)
        torch.cuda.synchronize()
        ref, ref_ring = oracle.foveate(img, s.radii, gaze[0], gaze[1], f)
        assert np.array_equal(ring.cpu().numpy(), ref_ring)
        _assert_equal(frame.cpu().numpy(), ref, f"4k {name} {gaze}")


@pytest.mark.parametrize("w,pad", [(70, 3), (64, 4), (64, 1)])
def test_foveate_pitched_output_and_no_ring_map(w, pad):
    # (64, 4): four pixels per thread with a pitch; the others one pixel per thread
    h = 33
    img, dimg = _image(w, h, seed=4, pitch_pad=pad)
    radii = (6.0, 15.0)
    mip = wrs.mip_build(dimg, 3)
    out_buf = torch.full((h, w + pad, 3), -1.0, device="cuda")
    out = out_buf[:, :w, :]
    frame, ring = wrs.foveate(dimg, mip, radii, (30.0, 16.0), "bilinear", out=out,
                              want_ring_map=False)
    torch.cuda.synchronize()
    assert ring is None
    ref, _ = oracle.foveate(img, radii, 30.0, 16.0, oracle.FILTER_BILINEAR)
    _assert_equal(out.cpu().numpy(), ref, "pitched")
    assert torch.all(out_buf[:, w:, :] == -1.0)  # padding untouched


@pytest.mark.parametrize("name", ["box", "bilinear"])
def test_matches_the_input_generator_on_gpu(name):
    # the product kernels and the seeded input generator produce the same
    # frames, so a stream fed by either evolves identically
    s = workload("hd").streams[0]
    fv = Foveator(s.width, s.height, s.radii, seed=s.seed, device="cuda", filter=name)
    fov = wrs.Foveation(fv.ground_truth, s.radii, filter=name)
    for gaze in ((960.0, 540.0), (17.3, 1001.9)):
        a, ra = fv.frame(*gaze)
        b, rb = fov.frame(gaze)
        assert torch.equal(ra, rb)
        assert torch.equal(a.view(torch.int32), b.view(torch.int32))


def test_mip_rebuild_after_image_change():
    w, h = 128, 64
    img, dimg = _image(w, h, seed=1)
    fov = wrs.Foveation(dimg, (10.0, 20.0), filter="bilinear")
    img2 = ground_truth(w, h, seed=2)
    dimg.copy_(torch.from_numpy(img2))
    fov.rebuild()
    frame, _ = fov.frame((40.0, 30.0))
    torch.cuda.synchronize()
    ref, _ = oracle.foveate(img2, (10.0, 20.0), 40.0, 30.0, oracle.FILTER_BILINEAR)
    _assert_equal(frame.cpu().numpy(), ref, "rebuilt")


def test_gpu_resident_stream_matches_oracle():
    # foveate -> push -> resolve entirely on the device, against the oracle
    # fed by the oracle's own foveation
    w, h, K = 96, 64, 4
    radii = (8.0, 20.0, 35.0)
    img, dimg = _image(w, h, seed=12)
    fov = wrs.Foveation(dimg, radii, filter="bilinear")
    st = wrs.Stream(w, h, K, radii[0], seed=12)
    ost = oracle.OracleStream(w, h, K, radii[0], seed=12)
    rng = np.random.default_rng(5)
    out = torch.empty((h, w, 3), device="cuda")
    for t in range(10):
        gaze = (float(rng.uniform(0, w)), float(rng.uniform(0, h)))
        frame, ring = fov.frame(gaze)
        st.push_frame(frame, gaze, ring, out)
        ref_frame, ref_ring = oracle.foveate(img, radii, gaze[0], gaze[1], oracle.FILTER_BILINEAR)
        ost.push_frame(ref_frame, gaze, ref_ring)
    torch.cuda.synchronize()
    o = ost.state()
    compare_states(st.export_state(), o, None, False)
    check_resolve(out.cpu().numpy(), ost, o, False)


def test_foveate_argument_errors():
    w, h = 16, 8
    _, dimg = _image(w, h, seed=0)
    mip = wrs.mip_build(dimg, 2)  # room for one radius only
    with pytest.raises(wrs.WrsError, match="mip buffer"):
        wrs.foveate(dimg, mip, (2.0, 4.0), (8.0, 4.0))
    with pytest.raises(wrs.WrsError, match="ascending"):
        wrs.foveate(dimg, mip, (2.0, 1.0), (8.0, 4.0))
    with pytest.raises(wrs.WrsError, match="gaze"):
        wrs.foveate(dimg, mip, (2.0,), (float("nan"), 4.0))
    with pytest.raises(wrs.WrsError, match="buffer holds"):
        wrs.mip_build(dimg, 4, out=torch.empty(256, dtype=torch.uint8, device="cuda"))


@pytest.mark.parametrize("name", ["box", "bilinear"])
@pytest.mark.parametrize("opts", [
    {"K": 8}, {"K": 4}, {"K": 3}, {"K": 8, "color_fp16": True}, {"K": 1, "update_rule": 1},
    {"K": 4, "temporal_bias": 2},
])
def test_push_foveated_equals_foveate_then_push(name, opts):
    # foveating on read gives the reservoirs and output of wrs_foveate followed
    # by wrs_push_frame, bit for bit, and both match the oracle
    w, h = 160, 72
    radii = (10.0, 25.0, 45.0)
    opts = dict(opts)
    K = opts.pop("K")
    img, dimg = _image(w, h, seed=21)
    fov = wrs.Foveation(dimg, radii, filter=name)
    a = wrs.Stream(w, h, K, radii[0], seed=3, **opts)
    b = wrs.Stream(w, h, K, radii[0], seed=3, **opts)
    ost = oracle.OracleStream(w, h, K, radii[0], seed=3, rule=opts.get("update_rule", 0),
                              temporal_bias=opts.get("temporal_bias", True),
                              color_fp16=opts.get("color_fp16", False))
    oa = torch.empty((h, w, 3), device="cuda")
    ob = torch.empty((h, w, 3), device="cuda")
    rng = np.random.default_rng(8)
    f_id = oracle.FILTER_BOX if name == "box" else oracle.FILTER_BILINEAR
    for t in range(9):
        gaze = (float(rng.uniform(-10, w + 10)), float(rng.uniform(0, h)))
        flush = None
        if t == 6:
            flush = torch.zeros((h, w), dtype=torch.uint8, device="cuda")
            flush[10:30, 40:100] = 0xFF
        a.push_foveated(fov, gaze, flush, oa)
        frame, _ = fov.frame(gaze)
        b.push_frame(frame, gaze, flush, ob)
        ref, _ = oracle.foveate(img, radii, gaze[0], gaze[1], f_id)
        ost.push_frame(ref, gaze, None if flush is None else flush.cpu().numpy())
    torch.cuda.synchronize()
    assert np.array_equal(a.export_raw(), b.export_raw())
    assert torch.equal(oa.view(torch.int32), ob.view(torch.int32))
    o = ost.state()
    compare_states(a.export_state(), o, None, opts.get("color_fp16", False))
    check_resolve(oa.cpu().numpy(), ost, o, opts.get("color_fp16", False))


def test_push_foveated_4k_and_errors():
    s = workload("4k").streams[0]
    img, dimg = _image(s.width, s.height, seed=s.seed)
    fov = wrs.Foveation(dimg, s.radii, filter="bilinear")
    a = wrs.Stream(s.width, s.height, s.K, s.r_f, seed=1)
    b = wrs.Stream(s.width, s.height, s.K, s.r_f, seed=1)
    out_a = torch.empty((s.height, s.width, 3), device="cuda")
    out_b = torch.empty_like(out_a)
    for gaze in ((1920.0, 1080.0), (400.5, 1999.25), (3000.0, 20.0)):
        a.push_foveated(fov, gaze, None, out_a)
        frame, _ = fov.frame(gaze)
        b.push_frame(frame, gaze, None, out_b)
    torch.cuda.synchronize()
    assert np.array_equal(a.export_raw(), b.export_raw())
    assert torch.equal(out_a.view(torch.int32), out_b.view(torch.int32))
    odd = wrs.Stream(70, 8, 4, 3.0)
    _, dodd = _image(70, 8, seed=0)
    with pytest.raises(wrs.WrsError, match="width"):
        odd.push_foveated(wrs.Foveation(dodd, (3.0,)), (5.0, 4.0))
    assert odd.frame_index == 0
