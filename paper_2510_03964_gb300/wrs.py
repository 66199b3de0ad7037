"""Python face of libwrs: the same calls as include/wrs.h, with torch tensors
for device memory and torch CUDA streams. Every step of the reservoir update
and resolve runs in the library's CUDA kernels; this module only passes
pointers, sizes and stream handles.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from ._lib import (WRS_EMPTY_SLOT, WRS_FILTER_BILINEAR, WRS_FILTER_BOX, WrsConfig, WrsError,
                   WrsFovSource, WrsLayout, WrsMipLayout, check, load)


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _dev_ptr(t: torch.Tensor | None, dtype, name: str):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return t.data_ptr()


def make_config(width, height, K, fovea_radius_px, deg_per_px=0.0, seed=0, stream_id=0,
                color_fp16=False, temporal_bias=True, update_rule=0) -> WrsConfig:
    """update_rule: 0 = exponential-key race over K slots, 1 = the literal n = 1 rule (K = 1).
    temporal_bias: False/True (Eq. temporal-bias) or 2 (Eq. full-temporal-bias)."""
    return WrsConfig(int(width), int(height), int(K), float(fovea_radius_px), float(deg_per_px),
                     int(seed) & 0xFFFFFFFFFFFFFFFF, int(stream_id) & 0xFFFFFFFF,
                     1 if color_fp16 else 0, int(temporal_bias), int(update_rule))


def state_bytes(cfg: WrsConfig) -> int:
    n = load().wrs_state_bytes(C.byref(cfg))
    if n == 0:
        raise WrsError(1, load().wrs_last_error().decode())
    return int(n)


def state_layout(cfg: WrsConfig) -> WrsLayout:
    lay = WrsLayout()
    check(load().wrs_state_layout(C.byref(cfg), C.byref(lay)))
    return lay


class Stream:
    """One frame stream's reservoirs, resident in a caller-visible torch buffer.

    ``state`` may be passed in (uint8 CUDA tensor of at least
    ``state_bytes(cfg)`` bytes, 256-byte aligned) so that callers, such as the
    serving pool, control placement; otherwise one is allocated.
    """

    def __init__(self, width, height, K, fovea_radius_px, deg_per_px=0.0, seed=0, stream_id=0,
                 color_fp16=False, temporal_bias=True, device=None, stream=None,
                 state: torch.Tensor | None = None, update_rule: int = 0):
        self.cfg = make_config(width, height, K, fovea_radius_px, deg_per_px, seed, stream_id,
                               color_fp16, temporal_bias, update_rule)
        self.width, self.height, self.K = int(width), int(height), int(K)
        self.color_fp16 = bool(color_fp16)
        self.nbytes = state_bytes(self.cfg)
        self.layout = state_layout(self.cfg)
        if state is None:
            dev = torch.device("cuda") if device is None else torch.device(device)
            state = torch.empty(self.nbytes, dtype=torch.uint8, device=dev)
        elif state.numel() < self.nbytes:
            raise ValueError("state buffer too small")
        self.state = state
        self.spare = None
        self.device = state.device
        ctx = C.c_void_p()
        with torch.cuda.device(self.device):
            check(load().wrs_create(C.byref(self.cfg), state.data_ptr(), state.numel(),
                                    _stream_handle(stream), C.byref(ctx)))
        self._ctx = ctx

    # -- the four core calls -------------------------------------------------
    def push_frame(self, frame: torch.Tensor, gaze, fov_map: torch.Tensor | None = None,
                   out: torch.Tensor | None = None, stream=None, pitch: int | None = None):
        """frame: float32 CUDA [H][W][3] (or [H][pitch] with ``pitch``)."""
        if pitch is None:
            if tuple(frame.shape[-3:]) != (self.height, self.width, 3) or not frame.is_contiguous():
                raise ValueError("frame must be a contiguous [H][W][3] float32 tensor")
            pitch = 3 * self.width
        check(load().wrs_push_frame(self._ctx, _dev_ptr(frame, torch.float32, "frame"), int(pitch),
                                    float(gaze[0]), float(gaze[1]),
                                    _dev_ptr(fov_map, torch.uint8, "fov_map"),
                                    _dev_ptr(out, torch.float32, "out"), _stream_handle(stream)))
        return out

    def resolve(self, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.height, self.width, 3), dtype=torch.float32, device=self.device)
        check(load().wrs_resolve(self._ctx, _dev_ptr(out, torch.float32, "out"), _stream_handle(stream)))
        return out

    def close(self):
        if self._ctx:
            load().wrs_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- extras ----------------------------------------------------------------
    def set_reprojection_buffer(self, spare: torch.Tensor | None = "alloc", stream=None):
        """Attach a second state buffer (allocated when not given) so that
        push_frame_reproject can gather from the previous frame's reservoirs;
        None detaches it."""
        if isinstance(spare, str):
            spare = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        if spare is not None and spare.device != self.device:
            raise ValueError("the spare buffer must be on the stream's device")
        with torch.cuda.device(self.device):
            check(load().wrs_set_reprojection_buffer(
                self._ctx, None if spare is None else _dev_ptr(spare, torch.uint8, "spare"),
                0 if spare is None else spare.numel(), _stream_handle(stream)))
        self.spare = spare

    def push_frame_reproject(self, frame: torch.Tensor, gaze, motion: torch.Tensor | None = None,
                             depth: torch.Tensor | None = None, prev_depth: torch.Tensor | None = None,
                             depth_tol: float = 0.05, fov_map: torch.Tensor | None = None,
                             out: torch.Tensor | None = None, stream=None):
        """One frame with temporal reprojection: motion [H][W][2] float32
        (pixels moved since the previous frame), depth / prev_depth [H][W]
        float32 (view depth now and in the previous frame)."""
        if tuple(frame.shape) != (self.height, self.width, 3) or frame.stride(2) != 1 or frame.stride(1) != 3:
            raise ValueError("frame must be a [H][W][3] float32 tensor with packed pixels")
        for t, shape, name in ((motion, (self.height, self.width, 2), "motion"),
                               (depth, (self.height, self.width), "depth"),
                               (prev_depth, (self.height, self.width), "prev_depth"),
                               (fov_map, (self.height, self.width), "fov_map"),
                               (out, (self.height, self.width, 3), "out")):
            if t is not None and (tuple(t.shape) != shape or not t.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous tensor of shape {shape}")
        with torch.cuda.device(self.device):
            check(load().wrs_push_frame_reproject(
                self._ctx, _dev_ptr(frame, torch.float32, "frame"), int(frame.stride(0)),
                float(gaze[0]), float(gaze[1]), _dev_ptr(motion, torch.float32, "motion"),
                _dev_ptr(depth, torch.float32, "depth"), _dev_ptr(prev_depth, torch.float32, "prev_depth"),
                float(depth_tol), _dev_ptr(fov_map, torch.uint8, "fov_map"),
                _dev_ptr(out, torch.float32, "out"), _stream_handle(stream)))

    def push_foveated(self, foveation: "Foveation", gaze, fov_map: torch.Tensor | None = None,
                      out: torch.Tensor | None = None, stream=None):
        """Foveate this frame from ``foveation`` (image + mip buffer on the GPU)
        and push it in one pass: the same reservoirs and output as
        foveation.frame(gaze) followed by push_frame, without the frame in memory."""
        fv = foveation
        if (fv.height, fv.width) != (self.height, self.width):
            raise ValueError("the foveation source must match the stream's size")
        r = (C.c_float * len(fv.radii))(*fv.radii)
        iptr, ipitch = _image_args(fv.img, "img")
        with torch.cuda.device(self.device):
            check(load().wrs_push_foveated(
                self._ctx, iptr, ipitch, _dev_ptr(fv.mip, torch.uint8, "mip"), fv.mip.numel(),
                len(fv.radii), r, FILTERS[fv.filter] if isinstance(fv.filter, str) else int(fv.filter),
                float(gaze[0]), float(gaze[1]), _dev_ptr(fov_map, torch.uint8, "fov_map"),
                _dev_ptr(out, torch.float32, "out"), _stream_handle(stream)))

    @property
    def frame_index(self) -> int:
        return int(load().wrs_frame_index(self._ctx))

    def set_launch(self, block_threads: int = 0, px_per_thread: int = 0):
        check(load().wrs_set_launch(self._ctx, int(block_threads), int(px_per_thread)))

    def get_launch(self):
        b, p = C.c_int(), C.c_int()
        check(load().wrs_get_launch(self._ctx, C.byref(b), C.byref(p)))
        return b.value, p.value

    def set_pipeline(self, enable: bool = True, px_per_thread: int = 0, stages: int = 0,
                     ctas_per_sm: int = 0):
        check(load().wrs_set_pipeline(self._ctx, 1 if enable else 0, int(px_per_thread), int(stages),
                                      int(ctas_per_sm)))

    def get_pipeline(self):
        """(enabled, pixels per thread, stages, CTAs per SM (0 = as many as fit))."""
        e, p, s, c = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        check(load().wrs_get_pipeline(self._ctx, C.byref(e), C.byref(p), C.byref(s), C.byref(c)))
        return bool(e.value), p.value, s.value, c.value

    def set_wait_limit(self, timeout_ns: int = 0, test_extra_tx: int = 0):
        check(load().wrs_set_wait_limit(self._ctx, int(timeout_ns), int(test_extra_tx)))

    def check_status(self, stream=None) -> int:
        """Waits for the stream; returns 0, or the status code a device-side wait recorded."""
        return int(load().wrs_check_status(self._ctx, _stream_handle(stream)))

    def replacements(self, stream=None) -> int:
        """Slot replacements since create (waits for the stream)."""
        v = C.c_uint64()
        check(load().wrs_get_stats(self._ctx, C.byref(v), _stream_handle(stream)))
        return int(v.value)

    def push_frame_host(self, h_frame: torch.Tensor, gaze, h_out: torch.Tensor, d_frame_stage,
                        d_out_stage, h_fov_map=None, d_fov_stage=None, stream=None):
        """Host frame in, host resolved frame out (copies inside the call)."""
        for t, n in ((h_frame, "h_frame"), (h_out, "h_out")):
            if t.is_cuda or not t.is_contiguous():
                raise ValueError(f"{n} must be a contiguous host tensor")
        check(load().wrs_push_frame_host(
            self._ctx, h_frame.data_ptr(), float(gaze[0]), float(gaze[1]),
            None if h_fov_map is None else h_fov_map.data_ptr(), h_out.data_ptr(),
            _dev_ptr(d_frame_stage, torch.float32, "d_frame_stage"),
            _dev_ptr(d_fov_stage, torch.uint8, "d_fov_stage"),
            _dev_ptr(d_out_stage, torch.float32, "d_out_stage"), _stream_handle(stream)))

    def push_frame_host_noalloc(self, h_frame: torch.Tensor, gaze, h_out: torch.Tensor,
                                h_fov_map=None, stream=None):
        """Host frame in, host resolved frame out, staged in the library's own
        device array (wrs_push_frame_host_noalloc): no device buffers needed."""
        for t, n in ((h_frame, "h_frame"), (h_out, "h_out")):
            if t.is_cuda or not t.is_contiguous():
                raise ValueError(f"{n} must be a contiguous host tensor")
        with torch.cuda.device(self.device):
            check(load().wrs_push_frame_host_noalloc(
                self._ctx, h_frame.data_ptr(), float(gaze[0]), float(gaze[1]),
                None if h_fov_map is None else h_fov_map.data_ptr(), h_out.data_ptr(),
                _stream_handle(stream)))

    def export_raw(self, stream=None) -> np.ndarray:
        buf = np.empty(self.nbytes, dtype=np.uint8)
        check(load().wrs_export_state(self._ctx, buf.ctypes.data, buf.nbytes, _stream_handle(stream)))
        return buf

    def import_raw(self, buf: np.ndarray, frame_index: int, stream=None):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        check(load().wrs_import_state(self._ctx, buf.ctypes.data, buf.nbytes, int(frame_index),
                                      _stream_handle(stream)))

    def export_state(self, stream=None) -> dict:
        """State planes as numpy arrays: W [HW], P [HW], key/idx/wt [K][HW], col [3][K][HW]."""
        return unpack_state(self.export_raw(stream), self.layout, self.K, self.width * self.height,
                            self.color_fp16)


def unpack_state(buf: np.ndarray, lay: WrsLayout, K: int, hw: int, color_fp16: bool) -> dict:
    pl = lay.plane_px

    def plane(off, dtype, n):
        return np.frombuffer(buf, dtype=dtype, count=n * pl, offset=off).reshape(n, pl)[:, :hw]

    out = {
        "W": plane(lay.W_off, np.float32, 1)[0].copy(),
        "P": plane(lay.P_off, np.float32, 1)[0].copy(),
        "key": plane(lay.key_off, np.float32, K).copy(),
        "idx": plane(lay.idx_off, np.uint32, K).copy(),
    }
    if color_fp16:
        # the weight's low 16 bits in their own plane, its high 16 bits in the
        # record's fourth half word
        lo = plane(lay.wt_off, np.uint16, K).astype(np.uint32)
        rec = np.frombuffer(buf, dtype=np.uint16, count=K * pl * 4, offset=lay.col_off)
        rec = rec.reshape(K, pl, 4)[:, :hw]
        out["wt"] = ((rec[:, :, 3].astype(np.uint32) << 16) | lo).view(np.float32)
        out["col"] = np.ascontiguousarray(np.transpose(rec[:, :, :3].view(np.float16), (2, 0, 1)))
    else:
        rec = np.frombuffer(buf, dtype=np.float32, count=K * pl * 4, offset=lay.col_off)
        rec = rec.reshape(K, pl, 4)[:, :hw]
        out["wt"] = rec[:, :, 0].copy()
        out["col"] = np.ascontiguousarray(np.transpose(rec[:, :, 1:], (2, 0, 1)))
    return out


__all__ = ["Stream", "make_config", "state_bytes", "state_layout", "unpack_state", "WrsError",
           "WRS_EMPTY_SLOT"]


class Batch:
    """One persistent launch (a CUDA-graph kernel node) that pushes a frame into
    each of up to ``max_streams`` streams of any size, K and colour precision."""

    def __init__(self, max_streams: int = 64):
        b = C.c_void_p()
        check(load().wrs_batch_create(int(max_streams), C.byref(b)))
        self._b = b
        self.max_streams = int(max_streams)

    def set_launch(self, px_per_thread: int = 1, stages: int = 0, ctas_per_sm: int = 0,
                   use_graph: bool = True):
        check(load().wrs_batch_set_launch(self._b, int(px_per_thread), int(stages), int(ctas_per_sm),
                                          1 if use_graph else 0))

    def get_launch(self):
        p, s, c, g = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        check(load().wrs_batch_get_launch(self._b, C.byref(p), C.byref(s), C.byref(c), C.byref(g)))
        return p.value, s.value, c.value, bool(g.value)

    def push(self, streams, frames, gazes, fov_maps=None, outs=None, stream=None):
        n = len(streams)
        if not (len(frames) == n and len(gazes) == n):
            raise ValueError("streams, frames and gazes must have the same length")
        ctxs = (C.c_void_p * n)(*[s._ctx.value for s in streams])
        fr = (C.c_void_p * n)(*[_dev_ptr(f, torch.float32, "frame") for f in frames])
        gz = (C.c_float * (2 * n))(*[float(v) for g in gazes for v in (g[0], g[1])])
        fm = None if fov_maps is None else (C.c_void_p * n)(
            *[_dev_ptr(m, torch.uint8, "fov_map") for m in fov_maps])
        ot = None if outs is None else (C.c_void_p * n)(*[_dev_ptr(o, torch.float32, "out") for o in outs])
        for f, s in zip(frames, streams):
            if tuple(f.shape[-3:]) != (s.height, s.width, 3) or not f.is_contiguous():
                raise ValueError("frames must be contiguous [H][W][3] float32 tensors")
        check(load().wrs_push_batch(self._b, n, ctxs, fr, gz, fm, ot, _stream_handle(stream)))

    def push_foveated(self, streams, foveations, gazes, fov_maps=None, outs=None, stream=None):
        """One frame per stream, each foveated on read from its ``Foveation``
        (image + mip levels on the GPU; all with the same filter) inside the
        batched update (wrs_push_batch_foveated): the same reservoirs and
        outputs as Stream.push_foveated of each stream alone."""
        n = len(streams)
        if not (len(foveations) == n and len(gazes) == n):
            raise ValueError("streams, foveations and gazes must have the same length")
        filters = {FILTERS[f.filter] if isinstance(f.filter, str) else int(f.filter) for f in foveations}
        if len(filters) != 1:
            raise ValueError("every foveation source of a batch must use the same filter")
        srcs = (WrsFovSource * n)()
        for i, (fv, s) in enumerate(zip(foveations, streams)):
            if (fv.height, fv.width) != (s.height, s.width):
                raise ValueError("each foveation source must match its stream's size")
            iptr, ipitch = _image_args(fv.img, "img")
            srcs[i].d_img = iptr
            srcs[i].img_pitch_elems = ipitch
            srcs[i].d_mip = _dev_ptr(fv.mip, torch.uint8, "mip")
            srcs[i].mip_bytes = fv.mip.numel()
            srcs[i].nradii = len(fv.radii)
            for k, r in enumerate(fv.radii):
                srcs[i].radii[k] = float(r)
        ctxs = (C.c_void_p * n)(*[s._ctx.value for s in streams])
        gz = (C.c_float * (2 * n))(*[float(v) for g in gazes for v in (g[0], g[1])])
        fm = None if fov_maps is None else (C.c_void_p * n)(
            *[_dev_ptr(m, torch.uint8, "fov_map") for m in fov_maps])
        ot = None if outs is None else (C.c_void_p * n)(*[_dev_ptr(o, torch.float32, "out") for o in outs])
        check(load().wrs_push_batch_foveated(self._b, n, ctxs, srcs, filters.pop(), gz, fm, ot,
                                             _stream_handle(stream)))

    def close(self):
        if self._b:
            load().wrs_batch_destroy(self._b)
            self._b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ pipelined host frames

class HostPipeline:
    """Frames in host memory through one stream with the upload of the next
    frame, the update of this one and the download of the previous output
    overlapping (wrs_host_pipe_*). Host tensors should be pinned; the last three
    frames' buffers must stay untouched until finish()."""

    def __init__(self, stream: Stream, with_fov: bool = False):
        self.stream = stream
        lib = load()
        n = int(lib.wrs_host_pipe_stage_bytes(stream._ctx, 1 if with_fov else 0))
        self.stage = torch.empty(n, dtype=torch.uint8, device=stream.device)
        self._p = C.c_void_p()
        with torch.cuda.device(stream.device):
            check(lib.wrs_host_pipe_create(stream._ctx, self.stage.data_ptr(), n, 1 if with_fov else 0,
                                           C.byref(self._p)))
        self.hw = stream.width * stream.height

    def push(self, h_frame: torch.Tensor, gaze, h_out: torch.Tensor, h_fov: torch.Tensor | None = None):
        for t, n, name in ((h_frame, 3 * self.hw, "h_frame"), (h_out, 3 * self.hw, "h_out")):
            if t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or t.numel() != n:
                raise ValueError(f"{name} must be a contiguous host float32 tensor of {n} values")
        if h_fov is not None and (h_fov.is_cuda or h_fov.dtype != torch.uint8 or h_fov.numel() != self.hw):
            raise ValueError("h_fov must be a host uint8 tensor of width * height values")
        with torch.cuda.device(self.stream.device):
            check(load().wrs_host_pipe_push(self._p, h_frame.data_ptr(), float(gaze[0]), float(gaze[1]),
                                            None if h_fov is None else h_fov.data_ptr(), h_out.data_ptr()))

    def finish(self):
        with torch.cuda.device(self.stream.device):
            check(load().wrs_host_pipe_finish(self._p))

    def close(self):
        if self._p:
            with torch.cuda.device(self.stream.device):
                load().wrs_host_pipe_destroy(self._p)
            self._p = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ foveation post-process

FILTERS = {"box": WRS_FILTER_BOX, "bilinear": WRS_FILTER_BILINEAR}


def mip_layout(width: int, height: int, levels: int) -> WrsMipLayout:
    lay = WrsMipLayout()
    check(load().wrs_mip_layout_get(int(width), int(height), int(levels), C.byref(lay)))
    return lay


def _image_args(img: torch.Tensor, name: str):
    if img.dim() != 3 or img.shape[2] != 3 or img.stride(2) != 1 or img.stride(1) != 3:
        raise ValueError(f"{name} must be a [H][W][3] float32 tensor with packed pixels")
    return _dev_ptr(img, torch.float32, name), int(img.stride(0))


def mip_build(img: torch.Tensor, levels: int, out: torch.Tensor | None = None,
              stream=None) -> torch.Tensor:
    """Levels 1..levels-1 of the mip buffer of ``img`` ([H][W][3] float32 on
    the GPU) into ``out`` (uint8, allocated if None)."""
    h, w = int(img.shape[0]), int(img.shape[1])
    lay = mip_layout(w, h, levels)
    if out is None:
        out = torch.empty(max(int(lay.total_bytes), 256), dtype=torch.uint8, device=img.device)
    ptr, pitch = _image_args(img, "img")
    with torch.cuda.device(img.device):
        check(load().wrs_mip_build(ptr, pitch, w, h, int(levels), _dev_ptr(out, torch.uint8, "mip"),
                                   out.numel(), _stream_handle(stream)))
    return out


def mip_levels(mip: torch.Tensor, width: int, height: int, levels: int) -> list:
    """Views [height[L]][width[L]][4] float32 of levels 1..levels-1 of a mip buffer."""
    lay = mip_layout(width, height, levels)
    out = []
    for L in range(1, levels):
        n = lay.width[L] * lay.height[L] * 16
        out.append(mip[lay.offset[L]:lay.offset[L] + n].view(torch.float32)
                   .view(lay.height[L], lay.width[L], 4))
    return out


def foveate(img: torch.Tensor, mip: torch.Tensor, radii, gaze, filter="box",
            out: torch.Tensor | None = None, ring_map: torch.Tensor | None = None,
            want_ring_map: bool = True, stream=None):
    """(frame [H][W][3] float32, ring map [H][W] uint8 or None) of the
    foveation post-process for one gaze; ``mip`` from mip_build with at least
    len(radii) + 1 levels."""
    h, w = int(img.shape[0]), int(img.shape[1])
    if out is None:
        out = torch.empty((h, w, 3), dtype=torch.float32, device=img.device)
    if ring_map is None and want_ring_map:
        ring_map = torch.empty((h, w), dtype=torch.uint8, device=img.device)
    if ring_map is not None and (tuple(ring_map.shape) != (h, w) or not ring_map.is_contiguous()):
        raise ValueError("ring_map must be a contiguous [H][W] uint8 tensor")
    r = (C.c_float * len(radii))(*[float(v) for v in radii])
    iptr, ipitch = _image_args(img, "img")
    optr, opitch = _image_args(out, "out")
    f = FILTERS[filter] if isinstance(filter, str) else int(filter)
    with torch.cuda.device(img.device):
        check(load().wrs_foveate(iptr, ipitch, _dev_ptr(mip, torch.uint8, "mip"), mip.numel(), w, h,
                                 len(radii), r, float(gaze[0]), float(gaze[1]), f, optr, opitch,
                                 _dev_ptr(ring_map, torch.uint8, "ring_map"), _stream_handle(stream)))
    return out, ring_map


class Foveation:
    """A rendered full-resolution image and its mip buffer, resident on the
    GPU, producing foveated frames for any gaze (Sec. 4.3)."""

    def __init__(self, img: torch.Tensor, radii, filter="box", stream=None):
        self.img = img
        self.radii = tuple(float(r) for r in radii)
        self.levels = len(self.radii) + 1
        self.filter = filter
        self.height, self.width = int(img.shape[0]), int(img.shape[1])
        self.mip = mip_build(img, self.levels, stream=stream)

    def rebuild(self, stream=None):
        """Re-derive the mip levels after the image changed (a new rendered frame)."""
        mip_build(self.img, self.levels, out=self.mip, stream=stream)

    def frame(self, gaze, out=None, ring_map=None, want_ring_map=True, stream=None):
        return foveate(self.img, self.mip, self.radii, gaze, self.filter, out, ring_map,
                       want_ring_map, stream)
