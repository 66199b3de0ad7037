"""Seeded gaze paths in pixel coordinates (float32 pairs, one per frame).

Two models stand in for the paper's eye-tracker recordings (Sec. 1 notes that
saccade landings scatter around their target and that fixations carry small
microsaccades):

* ``"jitter"``: a fixed centre plus isotropic Gaussian jitter every frame.
* ``"saccades"``: fixations of a fixed number of frames (300 ms at 90 Hz is
  27 frames) with per-frame Gaussian jitter around the fixation point; at
  the end of each fixation an instantaneous saccade to a uniformly random
  target, whose landing point scatters with a Gaussian around the target.

Gaze is clamped to the image rectangle [0, W] x [0, H].
"""
from __future__ import annotations

import numpy as np


def _normals(g: np.random.Generator, n: int) -> np.ndarray:
    # Box-Muller from plain uniforms, so the stream does not depend on the
    # numpy version's choice of normal sampler.
    u1 = 1.0 - g.random(n)  # (0, 1]
    u2 = g.random(n)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def gaze_path(width: int, height: int, frames: int, seed: int, model: str = "saccades",
              jitter_px: float = 6.0, fixation_frames: int = 27,
              landing_px: float = 25.0) -> np.ndarray:
    g = np.random.Generator(np.random.Philox(key=[seed & 0xFFFFFFFFFFFFFFFF, 2]))
    out = np.empty((frames, 2), dtype=np.float64)
    cx, cy = width / 2.0, height / 2.0
    if model == "jitter":
        n = _normals(g, 2 * frames).reshape(frames, 2)
        out[:, 0] = cx + jitter_px * n[:, 0]
        out[:, 1] = cy + jitter_px * n[:, 1]
    elif model == "saccades":
        fx, fy = cx, cy
        for t in range(frames):
            if t > 0 and t % fixation_frames == 0:
                tx, ty = g.random() * width, g.random() * height
                land = _normals(g, 2)
                fx = min(max(tx + landing_px * land[0], 0.0), float(width))
                fy = min(max(ty + landing_px * land[1], 0.0), float(height))
            j = _normals(g, 2)
            out[t, 0] = fx + jitter_px * j[0]
            out[t, 1] = fy + jitter_px * j[1]
    else:
        raise ValueError(f"unknown gaze model {model!r}")
    out[:, 0] = np.clip(out[:, 0], 0.0, float(width))
    out[:, 1] = np.clip(out[:, 1], 0.0, float(height))
    return out.astype(np.float32)
