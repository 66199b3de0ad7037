"""Helpers for the GPU-vs-oracle parity tests: run one seeded stream through
both sides on identical inputs and compare.

Bars (from the method's fixed FP32 key sequence): every reservoir plane (keys,
sample indices, slot weights, W, P, slot colours) bit-exact; resolved colour
within |gpu - ref| <= 1e-5 |ref| + 1e-7 of the oracle's FP64 resolve for FP32
colour storage. FP16 storage: slot colours bit-exact with the oracle's colours
rounded to half (IEEE nearest-even), resolve within the same tolerance of the
FP64 resolve of those rounded colours, and within 2^-11 relative + 1e-7 of the
FP64 resolve of the unrounded colours.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
import paper_2510_03964_gb300 as wrs
from synth import Foveator, gaze_path

RTOL, ATOL = 1e-5, 1e-7
RTOL_F16 = 2.0 ** -11


def assert_bits_equal(a, b, what):
    a = np.ascontiguousarray(a)
    b = np.ascontiguousarray(b)
    assert a.shape == b.shape, f"{what}: shape {a.shape} vs {b.shape}"
    if a.dtype.itemsize == 4:
        a, b = a.view(np.uint32), b.view(np.uint32)
    elif a.dtype.itemsize == 2:
        a, b = a.view(np.uint16), b.view(np.uint16)
    bad = np.flatnonzero(a != b)
    assert bad.size == 0, f"{what}: {bad.size} entries differ, first at flat index {bad[:5]}"


def compare_states(g: dict, o: dict, pix, color_fp16: bool):
    """g: GPU planes (SoA over all pixels); o: oracle state (pixel-major over pix)."""
    pix = np.arange(g["W"].shape[0]) if pix is None else np.asarray(pix)
    assert_bits_equal(g["W"][pix], o["W"], "W")
    assert_bits_equal(g["P"][pix], o["P"], "P")
    assert_bits_equal(g["idx"][:, pix].T, o["idx"], "idx")
    assert_bits_equal(g["key"][:, pix].T, o["key"], "key")
    assert_bits_equal(g["wt"][:, pix].T, o["wt"], "wt")
    col = np.transpose(g["col"][:, :, pix], (2, 1, 0))  # [n][K][3]
    ref = o["rgb"].astype(np.float16) if color_fp16 else o["rgb"]
    assert_bits_equal(col, ref, "slot colours")


def resolve_reference(o: dict, color_fp16: bool) -> np.ndarray:
    """FP64 weighted mean of the oracle's slots with colours as stored on the GPU."""
    occ = o["idx"] != oracle.EMPTY
    w = np.where(occ, o["wt"].astype(np.float64), 0.0)
    c = o["rgb"].astype(np.float16).astype(np.float64) if color_fp16 else o["rgb"].astype(np.float64)
    den = w.sum(axis=1)
    num = (w[:, :, None] * c).sum(axis=1)
    return np.where(den[:, None] > 0, num / np.where(den > 0, den, 1.0)[:, None], 0.0)


def check_resolve(got: np.ndarray, o_stream, o_state: dict, color_fp16: bool, what="resolve"):
    got = got.reshape(-1, 3).astype(np.float64)
    if not color_fp16:
        ref = o_stream.resolve()
        err = np.abs(got - ref) - (RTOL * np.abs(ref) + ATOL)
        assert np.all(err <= 0), f"{what}: worst excess {err.max():.3g}"
        return 0.0
    ref16 = resolve_reference(o_state, True)
    err = np.abs(got - ref16) - (RTOL * np.abs(ref16) + ATOL)
    assert np.all(err <= 0), f"{what} (fp16 slots): worst excess {err.max():.3g}"
    ref = o_stream.resolve()
    rel = np.abs(got - ref) - (RTOL_F16 * np.abs(ref) + ATOL)
    assert np.all(rel <= 0), f"{what}: FP16 storage error above 2^-11: {rel.max():.3g}"
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-30)))


class PairedRun:
    """One stream on the GPU (libwrs) and in the oracle, fed identical frames."""

    def __init__(self, width, height, K, r_f, radii=None, frames=8, seed=0, stream_id=0,
                 gaze_model="jitter", jitter_px=4.0, color_fp16=False, temporal_bias=True,
                 deg_per_px=0.0, pixels=None, launch=None, gaze=None, scene_seed=None,
                 frame_device="cpu", pipeline=None, update_rule=0, switch_scene_at=None):
        self.width, self.height, self.K = width, height, K
        self.color_fp16 = color_fp16
        self.dev = torch.device("cuda")
        radii = radii or (r_f, 2.5 * r_f)
        self.fv = Foveator(width, height, radii, seed=seed if scene_seed is None else scene_seed,
                           device=frame_device)
        # a scene cut: from frame switch_scene_at on, frames come from another scene
        self.switch_at = switch_scene_at
        self.fv2 = None if switch_scene_at is None else Foveator(width, height, radii, seed=seed + 1000,
                                                                  device=frame_device)
        if gaze is None:
            gaze = gaze_path(width, height, frames, seed=seed, model=gaze_model, jitter_px=jitter_px)
        self.gaze = np.asarray(gaze, np.float32)
        self.pixels = None if pixels is None else np.asarray(pixels, np.int64)
        self.gpu = wrs.Stream(width, height, K, r_f, deg_per_px=deg_per_px, seed=seed,
                              stream_id=stream_id, color_fp16=color_fp16,
                              temporal_bias=temporal_bias, device=self.dev, update_rule=update_rule)
        if launch:
            self.gpu.set_launch(*launch)
        if pipeline is not None:
            self.gpu.set_pipeline(*pipeline)
        self.orc = oracle.OracleStream(width, height, K, r_f, deg_per_px=deg_per_px, seed=seed,
                                       stream_id=stream_id, temporal_bias=temporal_bias,
                                       pixels=self.pixels, nthreads=8, rule=update_rule,
                                       color_fp16=color_fp16)
        self.out = torch.empty((height, width, 3), dtype=torch.float32, device=self.dev)
        self._host_frame = None

    def step(self, t, fov_map=None, fused=True, pitch_pad=0):
        gx, gy = self.gaze[t]
        fv = self.fv2 if (self.switch_at is not None and t >= self.switch_at) else self.fv
        fr, _ = fv.frame(float(gx), float(gy))
        fm_d = None if fov_map is None else torch.as_tensor(fov_map).to(self.dev)
        if pitch_pad:
            padded = torch.zeros((self.height, 3 * self.width + pitch_pad), dtype=torch.float32)
            padded[:, : 3 * self.width] = fr.cpu().reshape(self.height, -1)
            self.gpu.push_frame(padded.to(self.dev), (gx, gy), fm_d, self.out if fused else None,
                                pitch=3 * self.width + pitch_pad)
        else:
            self.gpu.push_frame(fr.to(self.dev).contiguous(), (gx, gy), fm_d,
                                self.out if fused else None)
        if self.pixels is None:
            host = fr.cpu().numpy()
        else:
            if self._host_frame is None:
                self._host_frame = np.zeros((self.height, self.width, 3), np.float32)
            flat = fr.reshape(-1, 3)
            idx = torch.as_tensor(self.pixels, device=flat.device)
            self._host_frame.reshape(-1, 3)[self.pixels] = flat.index_select(0, idx).cpu().numpy()
            host = self._host_frame
        self.orc.push_frame(host, (gx, gy), None if fov_map is None else np.asarray(fov_map))

    def run(self, frames=None, **kw):
        n = len(self.gaze) if frames is None else frames
        for t in range(n):
            self.step(t, **kw)
        torch.cuda.synchronize()

    def compare(self, check_out=True):
        # WRS_OK: no device-side wait gave up and (in the checked build) no
        # index or copy range fell outside its buffer
        assert self.gpu.check_status() == 0, wrs.load().wrs_last_error().decode()
        g = self.gpu.export_state()
        o = self.orc.state()
        compare_states(g, o, self.pixels, self.color_fp16)
        err = None
        if check_out:
            got = self.out.cpu().numpy().reshape(-1, 3)
            if self.pixels is not None:
                got = got[self.pixels]
            err = check_resolve(got, self.orc, o, self.color_fp16)
        return g, o, err
