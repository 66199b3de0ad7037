"""Autotuner for the launch shapes of the fused update + resolve.

For a stream configuration (or a batch of them) it times every feasible
candidate on scratch reservoirs of the same shapes, with CUDA events on the
launching stream, and keeps the fastest:

* single stream: the pipelined kernel's tile (256 x 1/2/4 pixels), number of
  shared-memory stages and CTAs per SM, and the plain kernel's block size and
  pixels per thread;
* batch: the batched kernel's tile, stages, CTAs per SM and graph/plain launch.

Results are cached per device name and shape signature in
``_build/autotune.json`` next to the library, so the sweep runs once.
Candidates that do not fit (shared memory, registers) are rejected by the
library itself and skipped here.
"""
from __future__ import annotations

import json
import os
import statistics
import threading

import torch

from . import build as _build
from ._lib import WrsError
from .wrs import Batch, Stream

CACHE = os.path.join(_build.OUT_DIR, "autotune.json")
_lock = threading.Lock()

PIPE_CANDIDATES = [(px, st, ctas) for px in (1, 2, 4) for st in (1, 2, 3, 4) for ctas in (0, 1, 2, 3)]
PLAIN_CANDIDATES = [(blk, px) for blk in (128, 256) for px in (1, 2, 4)]
BATCH_CANDIDATES = [(px, st, ctas, g) for px in (1, 2) for st in (0, 2, 3) for ctas in (0, 1, 2)
                    for g in (True,)]


def _key(kind: str, shapes) -> str:
    name = torch.cuda.get_device_name()
    return f"{name}|{kind}|" + ";".join(",".join(str(v) for v in s) for s in shapes)


def _load_cache() -> dict:
    try:
        return json.load(open(CACHE))
    except (OSError, ValueError):
        return {}


def _store(key: str, value: dict):
    with _lock:
        d = _load_cache()
        d[key] = value
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + f".{os.getpid()}.tmp"
        json.dump(d, open(tmp, "w"), indent=1)
        os.replace(tmp, CACHE)


def _time(fn, reps: int, stream) -> float:
    """Median milliseconds of fn() over reps launches, after two warm-up calls."""
    fn()
    fn()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    torch.cuda.synchronize()
    for a, b in ev:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in ev)


def _test_frame(w, h, dev, gen):
    return torch.rand((h, w, 3), device=dev, generator=gen)


def tune_stream(width, height, K, fovea_radius_px, color_fp16=False, device=None, reps=10,
                use_cache=True) -> dict:
    """Best launch shape for one stream shape: {"pipe": (px, stages, ctas)} or
    {"plain": (block, px)}, with the timing table."""
    shape = [(width, height, K, int(color_fp16))]
    key = _key("stream", shape)
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            return hit
    dev = torch.device("cuda") if device is None else torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(1234)
    stream = torch.cuda.Stream(device=dev)
    st = Stream(width, height, K, fovea_radius_px, color_fp16=color_fp16, device=dev, stream=stream)
    frame = _test_frame(width, height, dev, gen)
    out = torch.empty_like(frame)
    gaze = (width / 2.0, height / 2.0)
    table, cands = {}, {}

    def push():
        st.push_frame(frame, gaze, None, out, stream=stream)

    for cand in PIPE_CANDIDATES:
        try:
            st.set_pipeline(True, *cand)
            name = f"pipe {cand}"
            table[name] = _time(push, reps, stream)
            cands[name] = ("pipe", list(cand))
        except WrsError:
            continue
    for blk, px in PLAIN_CANDIDATES:
        st.set_pipeline(False)
        st.set_launch(blk, px)
        name = f"plain {(blk, px)}"
        table[name] = _time(push, reps, stream)
        cands[name] = ("plain", [blk, px])
    st.close()
    best = min(table, key=table.get)
    kind, tup = cands[best]
    res = {kind: tup, "ms": table[best], "table": table}
    if use_cache:
        _store(key, res)
    return res


def apply_stream(st: Stream, tuned: dict):
    if "pipe" in tuned:
        st.set_pipeline(True, *tuned["pipe"])
    else:
        st.set_pipeline(False)
        st.set_launch(*tuned["plain"])


def tune_batch(specs, device=None, reps=6, use_cache=True) -> dict:
    """Best batched launch for streams of the given (width, height, K, fp16,
    fovea radius) shapes: {"batch": (px, stages, ctas, use_graph)}."""
    shape = [(w, h, K, int(f16)) for (w, h, K, f16, _r) in specs]
    key = _key("batch", shape)
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            return hit
    dev = torch.device("cuda") if device is None else torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(4321)
    stream = torch.cuda.Stream(device=dev)
    streams = [Stream(w, h, K, r, seed=i + 1, stream_id=i, color_fp16=f16, device=dev, stream=stream)
               for i, (w, h, K, f16, r) in enumerate(specs)]
    frames = [_test_frame(w, h, dev, gen) for (w, h, *_x) in specs]
    outs = [torch.empty_like(f) for f in frames]
    gazes = [(w / 2.0, h / 2.0) for (w, h, *_x) in specs]
    b = Batch(len(specs))
    table, cands = {}, {}

    def push():
        b.push(streams, frames, gazes, outs=outs, stream=stream)

    for cand in BATCH_CANDIDATES:
        try:
            b.set_launch(*cand)
            name = str(tuple(cand))
            table[name] = _time(push, reps, stream)
            cands[name] = list(cand)
        except WrsError:
            continue
    b.close()
    for s in streams:
        s.close()
    best = min(table, key=table.get)
    res = {"batch": cands[best], "ms": table[best], "table": table}
    if use_cache:
        _store(key, res)
    return res
