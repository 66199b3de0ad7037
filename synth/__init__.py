"""Seeded synthetic inputs shared by the CPU oracle tests, the CUDA tests and bench.py.

This package holds no arithmetic of the reservoir method itself (no weights,
keys, bias or resolve): it only builds the frame streams the method consumes,
standing in for the paper's rendered scenes and eye-tracker scanpaths, which
are not available (the paper's Sponza / San Miguel / Fantasy Forest / Corridor
scenes and its Tobii recordings, Sec. 5).

* ``images``   procedural ground truth (gratings + hard-edged disks) and its
               aligned box-downsampled pyramid.
* ``foveate``  the foveation post-process: per-pixel ring level from the
               distance to the gaze, colour from that level's block mean
               (the paper simulates foveation as a mip-map post-process,
               Sec. 4.3 "Implementation").
* ``gaze``     gaze paths: jitter around a fixed centre, or fixations with
               jitter and saccades with scattered landings (Sec. 1).
* ``configs``  the five workload shapes (tiny, HD, 4K, 16-stream mix, serving).
"""
from .configs import WORKLOADS, Workload, StreamSpec, workload
from .images import bilinear_level, block_counts, block_means, block_sums, box_pyramid, ground_truth
from .foveate import Foveator, frame_pixels
from .gaze import gaze_path
from .scene import PanScene

__all__ = ["WORKLOADS", "Workload", "StreamSpec", "workload", "ground_truth",
           "box_pyramid", "block_means", "block_sums", "block_counts", "bilinear_level", "Foveator", "frame_pixels", "gaze_path", "PanScene"]
