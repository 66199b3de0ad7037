"""Batched persistent launch: every stream's planes and output are
bit-identical to pushing it alone (and to the oracle), for any launch shape."""
import numpy as np
import pytest
import torch

import paper_2510_03964_gb300 as wrs
from parity import assert_bits_equal, compare_states
from synth import Foveator, gaze_path, workload
import oracle

pytestmark = pytest.mark.gpu

MIX = [  # width, height, K, fp16, r_f
    (96, 40, 4, False, 10.0), (128, 32, 8, True, 12.0), (64, 16, 3, False, 6.0),
    (200, 8, 8, False, 20.0), (36, 20, 1, True, 5.0), (256, 12, 16, True, 30.0),
    (48, 24, 2, False, 7.0),
]


def _streams(dev, specs, seed0=1):
    out = []
    for i, (w, h, K, f16, rf) in enumerate(specs):
        out.append(wrs.Stream(w, h, K, rf, seed=seed0 + i, stream_id=i, color_fp16=f16, device=dev))
    return out


def _frames(specs, frames, seed0=1, dev="cuda"):
    per = []
    for i, (w, h, K, f16, rf) in enumerate(specs):
        fv = Foveator(w, h, (rf, 2.5 * rf), seed=seed0 + i)
        gz = gaze_path(w, h, frames, seed=seed0 + i, model="jitter", jitter_px=w / 4)
        per.append([(fv.frame(*gz[t])[0].to(dev).contiguous(), gz[t]) for t in range(frames)])
    return per


@pytest.mark.parametrize("launch", [(1, 0, 0, True), (1, 2, 1, True), (2, 0, 0, True),
                                    (4, 1, 0, False), (1, 3, 2, False), (2, 1, 1, True)])
def test_batch_equals_individual_pushes(launch):
    dev = torch.device("cuda")
    frames = 19  # more frames than the ring of replacement codes holds
    data = _frames(MIX, frames)
    solo = _streams(dev, MIX)
    mixed = _streams(dev, MIX)
    b = wrs.Batch(16)
    b.set_launch(*launch)
    outs_solo = [torch.empty((h, w, 3), device=dev) for (w, h, *_r) in MIX]
    outs_mix = [torch.empty((h, w, 3), device=dev) for (w, h, *_r) in MIX]
    for t in range(frames):
        for i, s in enumerate(solo):
            fr, g = data[i][t]
            s.push_frame(fr, g, out=outs_solo[i])
        fr = [data[i][t][0] for i in range(len(MIX))]
        gz = [data[i][t][1] for i in range(len(MIX))]
        try:
            b.push(mixed, fr, gz, outs=outs_mix)
        except wrs.WrsError as e:
            # a launch shape whose stages do not fit: nothing may have advanced
            assert "shared memory" in str(e) and t == 0
            assert all(x.frame_index == 0 for x in mixed)
            pytest.skip("these stages do not fit in shared memory")
    torch.cuda.synchronize()
    for i in range(len(MIX)):
        assert mixed[i].check_status() == 0 and solo[i].check_status() == 0
        assert mixed[i].frame_index == solo[i].frame_index == frames
        assert mixed[i].replacements() == solo[i].replacements() > 0
        assert_bits_equal(mixed[i].export_raw(), solo[i].export_raw(), f"stream {i} state")
        assert_bits_equal(outs_mix[i].cpu().numpy(), outs_solo[i].cpu().numpy(), f"stream {i} out")
    b.close()


def test_batch_matches_oracle_and_partial_outputs():
    dev = torch.device("cuda")
    specs = MIX[:4]
    frames = 6
    data = _frames(specs, frames, seed0=20)
    st = _streams(dev, specs, seed0=20)
    orcs = [oracle.OracleStream(w, h, K, rf, seed=20 + i, stream_id=i) for i, (w, h, K, f16, rf) in enumerate(specs)]
    b = wrs.Batch(8)
    outs = [torch.empty((h, w, 3), device=dev) for (w, h, *_r) in specs]
    for t in range(frames):
        fr = [data[i][t][0] for i in range(len(specs))]
        gz = [data[i][t][1] for i in range(len(specs))]
        b.push(st, fr, gz, outs=[outs[0], None, outs[2], None])
        for i, o in enumerate(orcs):
            o.push_frame(fr[i].cpu().numpy(), gz[i])
    torch.cuda.synchronize()
    for i, (w, h, K, f16, rf) in enumerate(specs):
        compare_states(st[i].export_state(), orcs[i].state(), None, f16)
    b.close()


def test_batch_rejects_bad_input_without_advancing():
    dev = torch.device("cuda")
    st = _streams(dev, MIX[:2])
    data = _frames(MIX[:2], 1)
    b = wrs.Batch(2)
    fr = [data[0][0][0], data[1][0][0]]
    gz = [data[0][0][1], data[1][0][1]]
    with pytest.raises(wrs.WrsError):
        b.push([st[0], st[0]], [fr[0], fr[0]], gz)           # same stream twice
    with pytest.raises(wrs.WrsError):
        b.push(st + st[:1], fr + fr[:1], gz + gz[:1])         # more than max_streams
    odd = wrs.Stream(37, 5, 2, 3.0, device=dev)
    with pytest.raises(wrs.WrsError):
        b.push([odd], [torch.zeros((5, 37, 3), device=dev)], [(1.0, 1.0)])  # width % 4 != 0
    with pytest.raises(wrs.WrsError):
        b.push(st, fr, [gz[0], (float("inf"), 0.0)])
    assert st[0].frame_index == 0 and st[1].frame_index == 0
    b.push(st, fr, gz)
    torch.cuda.synchronize()
    assert st[0].frame_index == 1 and st[0].check_status() == 0
    b.close()


def test_mix16_workload_batch_equals_individual():
    """The 16-stream uneven-resolution workload at full size, two frames."""
    dev = torch.device("cuda")
    wl = workload("mix16")
    specs = [(s.width, s.height, s.K, s.color_fp16, s.r_f) for s in wl.streams]
    frames = 2
    fvs = [Foveator(s.width, s.height, s.radii, seed=s.seed, device=dev) for s in wl.streams]
    gzs = [gaze_path(s.width, s.height, frames, seed=s.seed) for s in wl.streams]
    solo = [wrs.Stream(s.width, s.height, s.K, s.r_f, seed=s.seed, stream_id=s.stream_id,
                       color_fp16=s.color_fp16, device=dev) for s in wl.streams]
    mixed = [wrs.Stream(s.width, s.height, s.K, s.r_f, seed=s.seed, stream_id=s.stream_id,
                        color_fp16=s.color_fp16, device=dev) for s in wl.streams]
    b = wrs.Batch(16)
    outs = [torch.empty((s.height, s.width, 3), device=dev) for s in wl.streams]
    for t in range(frames):
        fr = [fvs[i].frame(*gzs[i][t])[0] for i in range(16)]
        b.push(mixed, fr, [g[t] for g in gzs], outs=outs)
        for i in range(16):
            solo[i].push_frame(fr[i], gzs[i][t])  # no resolve: the state does not depend on it
    torch.cuda.synchronize()
    for i in range(16):
        assert np.array_equal(mixed[i].export_raw(), solo[i].export_raw()), f"stream {i}"
    b.close()


def test_batch_mixes_literal_and_key_streams():
    dev = torch.device("cuda")
    specs = [(96, 40, 1, False, 10.0), (64, 16, 4, True, 6.0), (128, 32, 1, True, 12.0)]
    rules = [1, 0, 1]
    frames = 6
    data = _frames(specs, frames, seed0=40)
    mk = lambda: [wrs.Stream(w, h, K, rf, seed=40 + i, stream_id=i, color_fp16=f16, device=dev,
                             update_rule=rules[i]) for i, (w, h, K, f16, rf) in enumerate(specs)]
    solo, mixed = mk(), mk()
    b = wrs.Batch(4)
    for t in range(frames):
        for i, x in enumerate(solo):
            x.push_frame(*data[i][t])
        b.push(mixed, [d[t][0] for d in data], [d[t][1] for d in data])
    torch.cuda.synchronize()
    for i in range(len(specs)):
        assert np.array_equal(mixed[i].export_raw(), solo[i].export_raw()), f"stream {i}"
        assert mixed[i].replacements() == solo[i].replacements()
    orc = oracle.OracleStream(96, 40, 1, 10.0, seed=40, stream_id=0, rule=1)
    for t in range(frames):
        orc.push_frame(data[0][t][0].cpu().numpy(), data[0][t][1])
    compare_states(mixed[0].export_state(), orc.state(), None, False)
    b.close()


def test_batch_full_temporal_bias_without_outputs():
    # Eq. (full-temporal-bias) reads the slots' colours even when no output is
    # written: batched pushes without outputs equal solo pushes and the oracle
    dev = torch.device("cuda")
    specs = MIX[:4]
    frames = 6
    data = _frames(specs, frames, seed0=30)
    solo = [wrs.Stream(w, h, K, rf, seed=30 + i, stream_id=i, color_fp16=f16, device=dev,
                       temporal_bias=2) for i, (w, h, K, f16, rf) in enumerate(specs)]
    mixed = [wrs.Stream(w, h, K, rf, seed=30 + i, stream_id=i, color_fp16=f16, device=dev,
                        temporal_bias=2) for i, (w, h, K, f16, rf) in enumerate(specs)]
    orc = oracle.OracleStream(*specs[0][:3], specs[0][4], seed=30, stream_id=0, temporal_bias=2,
                              color_fp16=specs[0][3])
    b = wrs.Batch(8)
    for t in range(frames):
        for i, s in enumerate(solo):
            s.push_frame(data[i][t][0], data[i][t][1])
        b.push(mixed, [data[i][t][0] for i in range(len(specs))], [data[i][t][1] for i in range(len(specs))])
        orc.push_frame(data[0][t][0].cpu().numpy(), data[0][t][1])
    torch.cuda.synchronize()
    for i in range(len(specs)):
        assert_bits_equal(mixed[i].export_raw(), solo[i].export_raw(), f"stream {i} state")
    compare_states(mixed[0].export_state(), orc.state(), None, specs[0][3])
    b.close()


FOV_MIX = [  # width, height, K, fp16, rule, radii
    (96, 40, 4, False, 0, (10.0, 25.0)), (128, 32, 8, True, 0, (12.0, 30.0, 60.0)),
    (64, 16, 3, False, 0, (6.0, 15.0)), (200, 8, 8, False, 0, (20.0, 50.0)),
    (36, 20, 1, True, 1, (5.0, 12.0)), (256, 12, 16, True, 0, (30.0, 75.0)),
]


@pytest.mark.parametrize("filt", ["box", "bilinear"])
@pytest.mark.parametrize("with_outs", [True, False])
def test_foveating_batch_equals_solo_foveated_pushes(filt, with_outs):
    # each stream's frame foveated on read inside the batched update: the same
    # reservoirs and outputs as wrs_push_foveated of the stream alone
    from synth import ground_truth
    dev = torch.device("cuda")
    frames = 18
    fovs, gazes, solo, mixed = [], [], [], []
    for i, (w, h, K, f16, rule, radii) in enumerate(FOV_MIX):
        img = torch.from_numpy(ground_truth(w, h, 30 + i)).to(dev)
        fovs.append(wrs.Foveation(img, radii, filter=filt))
        gazes.append(gaze_path(w, h, frames, seed=40 + i, model="jitter", jitter_px=w / 3))
        for lst in (solo, mixed):
            lst.append(wrs.Stream(w, h, K, radii[0], seed=7 + i, stream_id=i, color_fp16=f16,
                                  device=dev, update_rule=rule))
    outs_solo = [torch.empty((h, w, 3), device=dev) for (w, h, *_r) in FOV_MIX]
    outs_mix = [torch.empty((h, w, 3), device=dev) for (w, h, *_r) in FOV_MIX]
    b = wrs.Batch(16)
    for t in range(frames):
        for i, s in enumerate(solo):
            s.push_foveated(fovs[i], gazes[i][t], out=outs_solo[i] if with_outs else None)
        b.push_foveated(mixed, fovs, [g[t] for g in gazes], outs=outs_mix if with_outs else None)
    torch.cuda.synchronize()
    for i in range(len(FOV_MIX)):
        assert mixed[i].check_status() == 0
        assert mixed[i].frame_index == solo[i].frame_index == frames
        assert_bits_equal(mixed[i].export_raw(), solo[i].export_raw(), f"stream {i} state")
        if with_outs:
            assert_bits_equal(outs_mix[i].cpu().numpy(), outs_solo[i].cpu().numpy(), f"stream {i} out")
    b.close()


def test_foveating_batch_rejects_mixed_filters_and_bad_sources():
    from synth import ground_truth
    dev = torch.device("cuda")
    img = torch.from_numpy(ground_truth(64, 16, 1)).to(dev)
    a = wrs.Foveation(img, (6.0, 15.0), filter="box")
    c = wrs.Foveation(img, (6.0, 15.0), filter="bilinear")
    s1 = wrs.Stream(64, 16, 4, 6.0, seed=1, device=dev)
    s2 = wrs.Stream(64, 16, 4, 6.0, seed=2, device=dev)
    b = wrs.Batch(4)
    with pytest.raises(ValueError):
        b.push_foveated([s1, s2], [a, c], [(3.0, 4.0), (5.0, 6.0)])
    small = wrs.Foveation(torch.from_numpy(ground_truth(32, 16, 1)).to(dev), (6.0, 15.0))
    with pytest.raises(ValueError):
        b.push_foveated([s1], [small], [(3.0, 4.0)])
    assert s1.frame_index == s2.frame_index == 0
    b.close()
