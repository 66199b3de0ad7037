"""The seeded input generators: determinism, ranges and ring structure."""
import numpy as np
import torch

from synth import Foveator, box_pyramid, gaze_path, ground_truth, workload


def test_ground_truth_deterministic_and_in_range():
    a = ground_truth(97, 53, seed=3)
    b = ground_truth(97, 53, seed=3)
    c = ground_truth(97, 53, seed=4)
    assert a.shape == (53, 97, 3) and a.dtype == np.float32
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= 0.0 and a.max() <= 1.0


def test_box_pyramid_block_means():
    img = ground_truth(37, 21, seed=1)
    pyr = box_pyramid(img, 4)
    assert np.array_equal(pyr[0], img)
    for lev in (1, 2, 3):
        b = 1 << lev
        for (y, x) in ((0, 0), (20, 36), (9, 17)):
            by, bx = (y // b) * b, (x // b) * b
            blk = img[by:by + b, bx:bx + b].astype(np.float64).mean(axis=(0, 1))
            assert np.allclose(pyr[lev, y, x], blk, rtol=0, atol=1e-6)


def test_foveated_frame_rings():
    fv = Foveator(64, 48, (8.0, 20.0), seed=2)
    fr, lev = fv.frame(30.25, 20.5)
    yy, xx = np.mgrid[0:48, 0:64]
    d2 = ((xx + 0.5) - 30.25) ** 2 + ((yy + 0.5) - 20.5) ** 2
    expect = (d2 > 64.0).astype(np.uint8) + (d2 > 400.0).astype(np.uint8)
    assert np.array_equal(lev.numpy(), expect)
    pyr = box_pyramid(fv.ground_truth.numpy(), 3)
    ref = np.take_along_axis(pyr.reshape(3, -1, 3), expect.reshape(1, -1, 1).astype(np.int64), 0)
    assert np.array_equal(fr.numpy().reshape(-1, 3), ref[0])


def test_foveator_ring_test_is_exact_on_dyadic_inputs():
    # the ring test uses float32 sub/mul/add only; with dyadic gaze and radius
    # every step is exact, so it must agree with exact rationals
    fv = Foveator(16, 16, (3.0,), seed=0)
    lev = fv.ring_map(7.75, 8.5).numpy()
    for y in range(16):
        for x in range(16):
            dx, dy = x + 0.5 - 7.75, y + 0.5 - 8.5
            assert lev[y, x] == (dx * dx + dy * dy > 9.0)
    assert torch.equal(fv.ring_map(7.75, 8.5), fv.ring_map(7.75, 8.5))
    # the boundary is inclusive: d2 == r2 stays inside (pixel (10, 8): dx = 2.75, dy = 0)
    fv2 = Foveator(16, 16, (2.75,), seed=0)
    assert fv2.ring_map(7.75, 8.5).numpy()[8, 10] == 0
    assert fv2.ring_map(7.75, 8.5).numpy()[8, 11] == 1


def test_block_sums_tree_and_counts():
    from synth import block_counts, block_sums
    img = ground_truth(37, 21, seed=5)
    for lev in (1, 2, 3, 4):
        s = block_sums(img, lev)
        b = 1 << lev
        # the tree sum is within float32 rounding of the FP64 block sum
        for (i, j) in ((0, 0), (s.shape[0] - 1, s.shape[1] - 1), (1, 2)):
            ref = img[i * b:(i + 1) * b, j * b:(j + 1) * b].astype(np.float64).sum(axis=(0, 1))
            assert np.allclose(s[i, j], ref, rtol=lev * 2.0 ** -23, atol=0)
        n = block_counts(21, 37, lev)
        assert n.sum() == 21 * 37
    # level L+1 sums are the quad sums of level L sums, in the stated order
    s1, s2 = block_sums(img, 1), block_sums(img, 2)
    pad = np.zeros((2 * s2.shape[0], 2 * s2.shape[1], 3), np.float32)
    pad[:s1.shape[0], :s1.shape[1]] = s1
    quad = (pad[0::2, 0::2] + pad[0::2, 1::2]) + (pad[1::2, 0::2] + pad[1::2, 1::2])
    assert np.array_equal(quad, s2)


def test_gaze_paths():
    g = gaze_path(1920, 1080, 120, seed=0)
    assert g.shape == (120, 2) and g.dtype == np.float32
    assert np.all((g[:, 0] >= 0) & (g[:, 0] <= 1920) & (g[:, 1] >= 0) & (g[:, 1] <= 1080))
    assert np.array_equal(g, gaze_path(1920, 1080, 120, seed=0))
    # within a fixation the spread is the jitter; across saccades it is large
    fix = g[1:27]
    assert np.std(fix[:, 0]) < 15 and np.std(fix[:, 1]) < 15
    j = gaze_path(256, 256, 5000, seed=0, model="jitter", jitter_px=4.0)
    assert abs(np.std(j[:, 0]) - 4.0) < 0.3 and abs(np.mean(j[:, 1]) - 128.0) < 0.3


def test_workloads():
    assert workload("tiny").pixels == 65536
    assert workload("hd").pixels == 2073600
    assert workload("4k").pixels == 8294400
    mix = workload("mix16")
    assert len(mix.streams) == 16 and mix.pixels == 68917248
    assert [s.K for s in mix.streams[:4]] == [8, 4, 8, 4]
    assert all(s.color_fp16 for s in mix.streams)


def test_block_means_order_and_bilinear():
    from synth import bilinear_level, block_means
    img = ground_truth(37, 21, seed=3)
    for lev in (1, 2, 3):
        m = block_means(img, lev)
        b = 1 << lev
        assert m.shape == (-(-21 // b), -(-37 // b), 3)
        blk = img[b:2 * b, 0:b].astype(np.float64).mean(axis=(0, 1))
        assert np.allclose(m[1, 0], blk, atol=1e-6)
        bl = bilinear_level(m, lev, 21, 37)
        # convex weights: the reconstruction stays within the range of the means
        assert bl.min() >= m.min() - 1e-6 and bl.max() <= m.max() + 1e-6
    # a linear ramp is reproduced exactly by block means + bilinear filtering
    # wherever no clamp applies (closed form: the mean of a block is the ramp
    # at the block centre, and bilinear interpolation of a linear function is
    # that function)
    w, h = 64, 32
    ramp = np.zeros((h, w, 3), np.float32)
    ramp[:, :, 0] = (np.arange(w) / 128.0)[None, :]
    ramp[:, :, 1] = (np.arange(h) / 64.0)[:, None]
    for lev in (1, 2, 3):
        b = 1 << lev
        bl = bilinear_level(block_means(ramp, lev), lev, h, w)
        inner = slice(b, -b)
        assert np.allclose(bl[inner, inner], ramp[inner, inner], atol=1e-6)
        assert np.all(bl[:, :, 2] == 0.0)
    fv = Foveator(37, 21, (4.0, 9.0), seed=3, filter="bilinear")
    fr, lev = fv.frame(10.0, 10.0)
    assert fr.shape == (21, 37, 3) and np.all(fr.numpy() >= 0) and np.all(fr.numpy() <= 1)


def test_pan_scene_motion_and_depth_are_consistent():
    from synth import PanScene
    sc = PanScene(96, 64, seed=3, velocity=(3.0, 1.0))
    f0, m0, d0 = sc.render(4)
    f1, m1, d1 = sc.render(5)
    f0, f1, m1, d0, d1 = (a.numpy() for a in (f0, f1, m1, d0, d1))
    assert f1.dtype == np.float32 and m1.shape == (64, 96, 2) and d1.shape == (64, 96)
    assert f1.min() >= 0 and f1.max() <= 1
    assert set(np.unique(d1)) <= set([10.0] + [np.float32(z) for z in sc.disk_z])
    # the background moves by exactly -velocity per frame: where it is seen in
    # both frames, a pixel shows what its motion vector points at
    bg = np.argwhere(d1 == 10.0)
    checked = 0
    for y, x in bg[::7]:
        py, px = int(y - m1[y, x, 1]), int(x - m1[y, x, 0])
        if 0 <= py < 64 and 0 <= px < 96 and d0[py, px] == 10.0:
            assert np.array_equal(f1[y, x], f0[py, px])
            checked += 1
    assert checked > 50
    # nearer disks move faster (parallax)
    assert np.abs(m1[d1 < 10.0]).max() > 3.0
    assert np.array_equal(sc.render(5)[0].numpy(), f1)  # deterministic


def test_pan_workload():
    s = workload("4k_pan").streams[0]
    assert s.pan_velocity == (3.25, 0.75) and s.pixels == 8294400
