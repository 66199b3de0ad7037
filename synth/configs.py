"""The workload shapes: one tiny stream, one HD stream, one 4K stream, a
16-stream uneven-resolution mix and a 64-viewer serving mix.

Sizes follow the paper's display setting (4K at up to 120 Hz, Sec. 5.1) and
the per-eye resolutions of current headsets. Every stream carries its own
seed; the Philox seed of the method and the scene/gaze seed are the same
number, so a stream is reproducible from its spec alone.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace


@dataclass(frozen=True)
class StreamSpec:
    width: int
    height: int
    K: int
    radii: tuple          # ring radii in px; radii[0] is the foveal radius r_f
    seed: int
    stream_id: int = 0
    frames: int = 8
    gaze_model: str = "saccades"
    jitter_px: float = 6.0
    color_fp16: bool = False
    temporal_bias: int = 1     # 0 none, 1 Eq. (temporal-bias), 2 Eq. (full-temporal-bias)
    update_rule: int = 0   # 0: key race over K slots, 1: literal n = 1 rule (K = 1)
    pan_velocity: tuple | None = None   # camera pan in background pixels per frame (PanScene)

    @property
    def r_f(self) -> float:
        return float(self.radii[0])

    @property
    def pixels(self) -> int:
        return self.width * self.height


@dataclass(frozen=True)
class Workload:
    name: str
    description: str
    streams: tuple = field(default_factory=tuple)

    @property
    def pixels(self) -> int:
        return sum(s.pixels for s in self.streams)


# ring radii per resolution class (fovea, 2x ring, 4x ring[, 8x beyond])
_RINGS_4K = (200.0, 500.0, 1000.0)
_RINGS_VR = (200.0, 500.0, 1000.0)
_RINGS_1440 = (150.0, 375.0, 750.0)
_RINGS_HD = (120.0, 300.0)

_MIX_CLASSES = ((3840, 2160, _RINGS_4K), (2064, 2208, _RINGS_VR),
                (1440, 1600, _RINGS_1440), (1920, 1080, _RINGS_HD))


def _mix_streams(frames: int, count: int = 16):
    out = []
    for i in range(count):
        w, h, radii = _MIX_CLASSES[(i // 4) % 4] if count == 16 else _MIX_CLASSES[i % 4]
        out.append(StreamSpec(width=w, height=h, K=8 if i % 2 == 0 else 4, radii=radii,
                              seed=i + 1, stream_id=i, frames=frames, color_fp16=True))
    return tuple(out)


WORKLOADS = {
    "4k_pan": Workload(
        "4k_pan", "3840x2160 RGB FP32, 240 frames, K=8, rings as 4k, a camera panning 3.25 px/frame "
        "right and 0.75 px/frame down over a far grating background (depth 10) and 8 disks at depths "
        "U[2,6] (parallax up to 16 px/frame); per-pixel motion vectors and depth; temporal "
        "reprojection with a 5% relative depth test",
        (StreamSpec(3840, 2160, 8, _RINGS_4K, seed=0, frames=240, pan_velocity=(3.25, 0.75)),)),
    "tiny": Workload(
        "tiny", "256x256 RGB FP32, 8 frames, K=4, fovea 32 px, 2x to 80 px, 4x beyond, "
        "gaze = centre + N(0, 4^2) px, Philox seed 0",
        (StreamSpec(256, 256, 4, (32.0, 80.0), seed=0, frames=8, gaze_model="jitter", jitter_px=4.0),)),
    "hd": Workload(
        "hd", "1920x1080 RGB FP32, 120 frames, K=4, fovea 120 px, 2x to 300 px, 4x beyond, "
        "fixations 27 frames (300 ms at 90 Hz), jitter 6 px, saccade landing scatter 25 px",
        (StreamSpec(1920, 1080, 4, _RINGS_HD, seed=0, frames=120),)),
    "4k": Workload(
        "4k", "3840x2160 RGB, 240 frames, K=8, fovea 200 px, 2x to 500 px, 4x to 1000 px, 8x beyond, "
        "FP32 colour planes, same gaze model as hd",
        (StreamSpec(3840, 2160, 8, _RINGS_4K, seed=0, frames=240),)),
    "hd_k8": Workload(
        "hd_k8", "1920x1080 RGB FP32, 120 frames, K=8, fovea 120 px, rings as hd: the 4k slot "
        "layout at a quarter of the pixels (profiling case)",
        (StreamSpec(1920, 1080, 8, _RINGS_HD, seed=0, frames=120),)),
    "hd_k8_fp16": Workload(
        "hd_k8_fp16", "as hd_k8 with FP16 colour planes (profiling case)",
        (StreamSpec(1920, 1080, 8, _RINGS_HD, seed=0, frames=120, color_fp16=True),)),
    "4k_k1": Workload(
        "4k_k1", "as 4k with one slot (n = 1, the paper's reservoir), exponential-key race",
        (StreamSpec(3840, 2160, 1, _RINGS_4K, seed=0, frames=240),)),
    "4k_k1_literal": Workload(
        "4k_k1_literal", "as 4k_k1 with the literal n = 1 rule (rand * (R1 + R2) <= R1 keeps R1 "
        "after the temporal bias; no keys, no bias product)",
        (StreamSpec(3840, 2160, 1, _RINGS_4K, seed=0, frames=240, update_rule=1),)),
    "4k_bias2": Workload(
        "4k_bias2", "as 4k with the full temporal bias (Eq. full-temporal-bias): the history's "
        "weight also scales by 1 - |Delta L*|/100 against the new sample",
        (StreamSpec(3840, 2160, 8, _RINGS_4K, seed=0, frames=240, temporal_bias=2),)),
    "hd_pan": Workload(
        "hd_pan", "as 4k_pan at 1920x1080 with the hd rings and K=8 (profiling case)",
        (StreamSpec(1920, 1080, 8, _RINGS_HD, seed=0, frames=120, pan_velocity=(3.25, 0.75)),)),
    "4k_fp16": Workload(
        "4k_fp16", "as 4k with FP16 colour planes (keys, weights and accumulation FP32)",
        (StreamSpec(3840, 2160, 8, _RINGS_4K, seed=0, frames=240, color_fp16=True),)),
    "mix16": Workload(
        "mix16", "16 streams: 4x 3840x2160, 4x 2064x2208, 4x 1440x1600, 4x 1920x1080; "
        "K=8 for even stream index, K=4 for odd; seeds 1-16; FP16 colour",
        _mix_streams(240)),
}


def workload(name: str, **overrides) -> Workload:
    wl = WORKLOADS[name]
    if overrides:
        wl = replace(wl, streams=tuple(replace(s, **overrides) for s in wl.streams))
    return wl
