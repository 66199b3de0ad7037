"""CPU oracle for foveated weighted reservoir sampling: ctypes wrapper over wrs_oracle.c.

TEST INFRASTRUCTURE ONLY. The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(``paper_2510_03964_gb300``) never does. The oracle shares no code with the
CUDA library; see wrs_oracle.h for what pins each function.

Parity unpinned: nothing. Each function is checked against an outside fact
(closed forms, libm, curand, brute-force sampling laws) in
tests/test_oracle_pins.py and tests/test_philox_curand.py.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wrs_oracle.c")
_HDR = os.path.join(_HERE, "wrs_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
# -std=c11 and -ffp-contract=off: no fused multiply-add anywhere (gcc would
# otherwise contract on aarch64); no fast-math: every operation is IEEE.
CFLAGS = ["-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-pthread", "-Wall"]

EMPTY = 0xFFFFFFFF
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (seconds). Returns its path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = force or not os.path.exists(_LIB) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB) for s in (_SRC, _HDR, __file__))
    if stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Config(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("K", C.c_int32),
                ("r_f", C.c_float), ("deg_per_px", C.c_float), ("seed", C.c_uint64),
                ("stream_id", C.c_uint32), ("temporal_bias", C.c_int32), ("rule", C.c_int32),
                ("color_fp16", C.c_int32)]


_P = C.c_void_p


def load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            sig = {
                "orc_exp": (C.c_float, [C.c_float]),
                "orc_log": (C.c_float, [C.c_float]),
                "orc_philox4x32_10": (None, [_P, _P, _P]),
                "orc_uniform": (C.c_float, [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int64]),
                "orc_density64": (C.c_double, [C.c_double]),
                "orc_density32": (C.c_float, [C.c_float]),
                "orc_weight32": (C.c_float, [C.POINTER(Config), C.c_int32, C.c_int32, C.c_float, C.c_float]),
                "orc_delta": (C.c_float, [C.POINTER(Config)]),
                "orc_pixel_step": (None, [C.c_int, C.c_int, C.c_float, C.c_float, C.c_uint32, _P, C.c_int,
                                          _P, _P, _P, _P, _P, _P]),
                "orc_resolve_pixel": (None, [C.c_int, _P, _P, _P, _P]),
                "orc_init_state": (None, [C.c_int, C.c_int64, _P, _P, _P, _P, _P, _P]),
                "orc_push_frame": (C.c_int, [C.POINTER(Config), C.c_uint32, _P, C.c_int64, C.c_float,
                                             C.c_float, _P, C.c_int64, _P, _P, _P, _P, _P, _P, _P, C.c_int]),
                "orc_resolve": (None, [C.c_int, C.c_int64, _P, _P, _P, _P, C.c_int]),
                "orc_run_streams": (None, [C.c_int, C.c_int, C.c_int64, C.c_int, _P, _P, _P, _P]),
                "orc_chao_literal": (None, [C.c_int, C.c_int64, C.c_int, _P, _P, _P]),
                "orc_exp_n": (None, [_P, _P, C.c_int64]),
                "orc_log_n": (None, [_P, _P, C.c_int64]),
                "orc_density32_n": (None, [_P, _P, C.c_int64]),
                "orc_density64_n": (None, [_P, _P, C.c_int64]),
                "orc_uniform_n": (None, [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int64, C.c_int64, _P]),
                "orc_weight32_grid": (None, [C.POINTER(Config), C.c_float, C.c_float, _P]),
                "orc_lightness": (C.c_float, [C.c_float, C.c_float, C.c_float]),
                "orc_lightness_n": (None, [_P, _P, C.c_int64]),
                "orc_push_frame_reproject": (C.c_int, [C.POINTER(Config), C.c_uint32, _P, C.c_int64,
                                                       C.c_float, C.c_float, _P, _P, _P, C.c_float, _P,
                                                       _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                                       C.c_int]),
                "orc_mip_means": (None, [_P, C.c_int64, C.c_int32, C.c_int32, C.c_int32, _P]),
                "orc_foveate": (C.c_int, [_P, C.c_int64, C.c_int32, C.c_int32, C.c_int32, _P,
                                          C.c_float, C.c_float, C.c_int32, _P, _P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data


def _f32(x):
    return np.ascontiguousarray(x, dtype=np.float32)


# ------------------------------------------------------------ element-wise

def exp32(x) -> np.ndarray:
    x = _f32(x)
    y = np.empty_like(x)
    load().orc_exp_n(_ptr(x), _ptr(y), x.size)
    return y


def log32(x) -> np.ndarray:
    x = _f32(x)
    y = np.empty_like(x)
    load().orc_log_n(_ptr(x), _ptr(y), x.size)
    return y


def density32(e) -> np.ndarray:
    e = _f32(e)
    y = np.empty_like(e)
    load().orc_density32_n(_ptr(e), _ptr(y), e.size)
    return y


def density64(e) -> np.ndarray:
    e = np.ascontiguousarray(e, dtype=np.float64)
    y = np.empty_like(e)
    load().orc_density64_n(_ptr(e), _ptr(y), e.size)
    return y


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty(4, dtype=np.uint32)
    load().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniforms(seed: int, stream_id: int, t: int, p0: int, n: int) -> np.ndarray:
    u = np.empty(n, dtype=np.float32)
    load().orc_uniform_n(seed, stream_id, t, p0, n, _ptr(u))
    return u


RULE_KEYS, RULE_LITERAL = 0, 1


BIAS_NONE, BIAS_TEMPORAL, BIAS_FULL = 0, 1, 2


def make_config(width, height, K, r_f, deg_per_px=0.0, seed=0, stream_id=0, temporal_bias=True,
                rule=RULE_KEYS, color_fp16=False):
    """temporal_bias: False/True (Eq. temporal-bias) or BIAS_FULL (Eq. full-temporal-bias)."""
    return Config(int(width), int(height), int(K), float(r_f), float(deg_per_px), int(seed),
                  int(stream_id), int(temporal_bias), int(rule), 1 if color_fp16 else 0)


def lightness(rgb) -> np.ndarray:
    rgb = np.ascontiguousarray(rgb, dtype=np.float32).reshape(-1, 3)
    out = np.empty(len(rgb), np.float32)
    load().orc_lightness_n(_ptr(rgb), _ptr(out), len(rgb))
    return out


def weight_grid(cfg: Config, gx: float, gy: float) -> np.ndarray:
    w = np.empty((cfg.height, cfg.width), dtype=np.float32)
    load().orc_weight32_grid(C.byref(cfg), gx, gy, _ptr(w))
    return w


def weight32(cfg: Config, x: int, y: int, gx: float, gy: float) -> float:
    return float(load().orc_weight32(C.byref(cfg), x, y, gx, gy))


def run_streams(K: int, bias: bool, w, u):
    """Independent single-pixel streams: w [n_items], u [n_trials][n_items] ->
    (final slot frame indices [n_trials][K], final W [n_trials])."""
    w = _f32(w)
    u = _f32(u)
    n_trials, n_items = u.shape
    assert w.shape == (n_items,)
    idx = np.empty((n_trials, K), dtype=np.uint32)
    W = np.empty(n_trials, dtype=np.float32)
    load().orc_run_streams(K, 1 if bias else 0, n_trials, n_items, _ptr(w), _ptr(u), _ptr(idx), _ptr(W))
    return idx, W


def chao_literal(bias: bool, w, u) -> np.ndarray:
    w = _f32(w)
    u = _f32(u)
    n_trials, n_items = u.shape
    idx = np.empty(n_trials, dtype=np.uint32)
    load().orc_chao_literal(1 if bias else 0, n_trials, n_items, _ptr(w), _ptr(u), _ptr(idx))
    return idx


# ------------------------------------------------------------ foveation

FILTER_BOX, FILTER_BILINEAR = 0, 1


def mip_means(img: np.ndarray, level: int) -> np.ndarray:
    """Level-`level` block means of an RGB float32 image [h][w][3] (or [h][pitch])."""
    img = _f32(img)
    h = img.shape[0]
    w = img.shape[1] if img.ndim == 3 else None
    if w is None:
        raise ValueError("pass the image as [h][w][3]")
    hb, wb = -(-h // (1 << level)), -(-w // (1 << level))
    out = np.empty((hb, wb, 3), np.float32)
    load().orc_mip_means(_ptr(img), 3 * w, w, h, level, _ptr(out))
    return out


def foveate(img: np.ndarray, radii, gx: float, gy: float, filter: int = FILTER_BOX):
    """(frame float32 [h][w][3], ring map uint8 [h][w]) of the foveation post-process."""
    img = _f32(img)
    h, w = img.shape[:2]
    r = _f32(list(radii))
    frame = np.empty((h, w, 3), np.float32)
    ring = np.empty((h, w), np.uint8)
    rc = load().orc_foveate(_ptr(img), 3 * w, w, h, len(r), _ptr(r), float(gx), float(gy),
                            int(filter), _ptr(frame), _ptr(ring))
    if rc != 0:
        raise ValueError("oracle rejected the foveation arguments")
    return frame, ring


# ------------------------------------------------------------ streams

class OracleStream:
    """One frame stream on the CPU; state is pixel-major (see wrs_oracle.h).

    ``pixels``: optional sorted row-major pixel indices to simulate (every
    pixel is an independent stream, so a sample of pixels evolves exactly as
    it would inside the full frame).
    """

    def __init__(self, width, height, K, r_f, deg_per_px=0.0, seed=0, stream_id=0,
                 temporal_bias=True, pixels=None, nthreads=1, rule=RULE_KEYS, color_fp16=False):
        self.cfg = make_config(width, height, K, r_f, deg_per_px, seed, stream_id, temporal_bias,
                               rule, color_fp16)
        self.K = int(K)
        self.pixels = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int64)
        n = width * height if self.pixels is None else len(self.pixels)
        self.n = n
        self.nthreads = nthreads
        self.W = np.empty(n, np.float32)
        self.P = np.empty(n, np.float32)
        self.key = np.empty((n, K), np.float32)
        self.idx = np.empty((n, K), np.uint32)
        self.wt = np.empty((n, K), np.float32)
        self.rgb = np.empty((n, K, 3), np.float32)
        load().orc_init_state(K, n, _ptr(self.W), _ptr(self.P), _ptr(self.key), _ptr(self.idx),
                              _ptr(self.wt), _ptr(self.rgb))
        self.t = 0

    def push_frame(self, frame: np.ndarray, gaze, fov_map: np.ndarray | None = None,
                   pitch: int | None = None):
        frame = np.ascontiguousarray(frame, dtype=np.float32)
        if pitch is None:
            pitch = 3 * self.cfg.width
        fm = None if fov_map is None else np.ascontiguousarray(fov_map, dtype=np.uint8)
        rc = load().orc_push_frame(C.byref(self.cfg), self.t, _ptr(frame), pitch, float(gaze[0]),
                                   float(gaze[1]), _ptr(fm), self.n, _ptr(self.pixels),
                                   _ptr(self.W), _ptr(self.P), _ptr(self.key), _ptr(self.idx),
                                   _ptr(self.wt), _ptr(self.rgb), self.nthreads)
        if rc != 0:
            raise ValueError("oracle rejected the frame arguments")
        self.t += 1

    def push_frame_reproject(self, frame: np.ndarray, gaze, motion: np.ndarray | None = None,
                             depth: np.ndarray | None = None, prev_depth: np.ndarray | None = None,
                             depth_tol: float = 0.05, fov_map: np.ndarray | None = None):
        """One frame with temporal reprojection (see orc_push_frame_reproject);
        the stream must hold every pixel."""
        if self.pixels is not None:
            raise ValueError("reprojection gathers from the whole previous frame: no pixel sample")
        frame = np.ascontiguousarray(frame, dtype=np.float32)
        mv = None if motion is None else np.ascontiguousarray(motion, dtype=np.float32)
        d = None if depth is None else _f32(depth)
        dp = None if prev_depth is None else _f32(prev_depth)
        fm = None if fov_map is None else np.ascontiguousarray(fov_map, dtype=np.uint8)
        nxt = {k: np.empty_like(v) for k, v in
               (("W", self.W), ("P", self.P), ("key", self.key), ("idx", self.idx),
                ("wt", self.wt), ("rgb", self.rgb))}
        rc = load().orc_push_frame_reproject(
            C.byref(self.cfg), self.t, _ptr(frame), 3 * self.cfg.width, float(gaze[0]),
            float(gaze[1]), _ptr(mv), _ptr(d), _ptr(dp), float(depth_tol), _ptr(fm),
            _ptr(self.W), _ptr(self.P), _ptr(self.key), _ptr(self.idx), _ptr(self.wt),
            _ptr(self.rgb), _ptr(nxt["W"]), _ptr(nxt["P"]), _ptr(nxt["key"]), _ptr(nxt["idx"]),
            _ptr(nxt["wt"]), _ptr(nxt["rgb"]), self.nthreads)
        if rc != 0:
            raise ValueError("oracle rejected the frame arguments")
        self.W, self.P, self.key, self.idx = nxt["W"], nxt["P"], nxt["key"], nxt["idx"]
        self.wt, self.rgb = nxt["wt"], nxt["rgb"]
        self.t += 1

    def resolve(self) -> np.ndarray:
        out = np.empty((self.n, 3), np.float64)
        load().orc_resolve(self.K, self.n, _ptr(self.idx), _ptr(self.wt), _ptr(self.rgb), _ptr(out),
                           self.nthreads)
        return out

    def state(self) -> dict:
        return {"W": self.W.copy(), "P": self.P.copy(), "key": self.key.copy(), "idx": self.idx.copy(),
                "wt": self.wt.copy(), "rgb": self.rgb.copy()}
