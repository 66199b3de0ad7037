"""The C-ABI library loads and exports what include/wrs.h declares; host-side
argument checks reject bad input before any CUDA call (no GPU needed)."""
import ctypes as C

import pytest

import paper_2510_03964_gb300 as pkg
from paper_2510_03964_gb300 import _lib


@pytest.fixture(scope="module")
def lib():
    return pkg.load()


def test_every_declared_function_is_exported(lib):
    names = pkg.header_functions()
    assert {"wrs_create", "wrs_push_frame", "wrs_resolve", "wrs_destroy"} <= set(names)
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/wrs.h but not exported"
    # the binding declares exactly the header's functions
    assert set(_lib.SIGNATURES) >= set(names)


def test_header_constants_match_binding():
    text = open(_lib.HEADER).read()
    assert "#define WRS_MAX_K 16" in text
    assert "#define WRS_EMPTY_SLOT 0xFFFFFFFFu" in text
    for i, n in enumerate(["WRS_OK", "WRS_ERR_ARG", "WRS_ERR_CUDA", "WRS_ERR_BUDGET",
                           "WRS_ERR_TIMEOUT", "WRS_ERR_STATE"]):
        assert f"#define {n} {i}" in text


def test_state_bytes_and_layout(lib):
    cfg = pkg.make_config(3840, 2160, 8, 200.0)
    n = pkg.state_bytes(cfg)
    lay = pkg.state_layout(cfg)
    hw = 3840 * 2160
    pl = lay.plane_px
    assert pl % 64 == 0 and pl >= hw
    # FP32 colour: W, P, key[8], idx[8] float planes + 8 float4 {w, r, g, b} record planes,
    # then the ring of 16 one-byte replacement-code planes
    assert lay.map_frames == 16 and lay.map_off == 256 + pl * 4 * (2 + 2 * 8) + pl * 16 * 8
    assert n == lay.total_bytes == lay.map_off + 16 * pl
    assert lay.status_off == 0 and lay.wt_off == -1 and lay.plane_bytes_col == 16 * pl
    for off in (lay.W_off, lay.P_off, lay.key_off, lay.idx_off, lay.col_off, lay.map_off):
        assert off % 256 == 0
    cfg16 = pkg.make_config(3840, 2160, 8, 200.0, color_fp16=True)
    lay16 = pkg.state_layout(cfg16)
    # FP16 colour: W, P, key[8], idx[8] float planes, 8 uint16 planes of the
    # weights' low halves, 8 records {r, g, b, w_hi} of 4 halves
    assert pkg.state_bytes(cfg16) == 256 + pl * (4 * (2 + 2 * 8) + 2 * 8 + 8 * 8) + 16 * pl
    assert lay16.wt_off > 0 and lay16.plane_bytes_col == 8 * pl and lay16.plane_bytes_wt == 2 * pl
    assert lay16.col_off % 256 == 0 and lay.plane_bytes_wt == 0
    # odd K: the weight planes end off a 256-byte boundary and the records start on the next
    lay3 = pkg.state_layout(pkg.make_config(8, 8, 3, 2.0, color_fp16=True))
    assert lay3.col_off == (lay3.wt_off + 3 * 2 * lay3.plane_px + 255) // 256 * 256
    # one or two slots: the sample indices are written directly, no code ring
    lay1 = pkg.state_layout(pkg.make_config(64, 8, 1, 4.0))
    assert lay1.map_frames == 0 and lay1.total_bytes == lay1.map_off
    assert pkg.state_layout(pkg.make_config(64, 8, 3, 4.0)).map_frames == 16
    # ragged size: planes padded to 64 entries
    lay2 = pkg.state_layout(pkg.make_config(37, 23, 3, 5.0))
    assert lay2.plane_px == 896


@pytest.mark.parametrize("bad", [dict(width=0), dict(height=-1), dict(K=0), dict(K=17),
                                 dict(fovea_radius_px=0.0), dict(fovea_radius_px=float("inf")),
                                 dict(deg_per_px=float("nan")), dict(width=1 << 16, height=1 << 15),
                                 dict(update_rule=2), dict(update_rule=1, K=2)])
def test_invalid_configs_rejected(lib, bad):
    args = dict(width=64, height=64, K=4, fovea_radius_px=8.0)
    args.update(bad)
    cfg = pkg.make_config(**args)
    assert lib.wrs_state_bytes(C.byref(cfg)) == 0
    assert lib.wrs_last_error().decode() != ""
    ctx = C.c_void_p()
    rc = lib.wrs_create(C.byref(cfg), C.c_void_p(256), 1 << 30, None, C.byref(ctx))
    assert rc == _lib.WRS_ERR_ARG and not ctx.value


def test_create_checks_buffer_before_cuda(lib):
    cfg = pkg.make_config(64, 64, 4, 8.0)
    ctx = C.c_void_p()
    assert lib.wrs_create(C.byref(cfg), None, 1 << 20, None, C.byref(ctx)) == _lib.WRS_ERR_ARG
    assert lib.wrs_create(C.byref(cfg), C.c_void_p(256 + 16), 1 << 20, None, C.byref(ctx)) == _lib.WRS_ERR_ARG
    assert "aligned" in lib.wrs_last_error().decode()
    need = lib.wrs_state_bytes(C.byref(cfg))
    assert lib.wrs_create(C.byref(cfg), C.c_void_p(256), need - 1, None, C.byref(ctx)) == _lib.WRS_ERR_BUDGET


def test_null_context_calls_fail_cleanly(lib):
    assert lib.wrs_push_frame(None, None, 0, 0.0, 0.0, None, None, None) == _lib.WRS_ERR_ARG
    assert lib.wrs_resolve(None, None, None) == _lib.WRS_ERR_ARG
    assert lib.wrs_destroy(None) == _lib.WRS_OK
    assert lib.wrs_frame_index(None) == 0
    assert lib.wrs_set_launch(None, 128, 4) == _lib.WRS_ERR_ARG


def test_mip_layout(lib):
    lay = pkg.mip_layout(3840, 2160, 4)
    assert lay.levels == 4 and lay.offset[0] == -1
    assert [lay.width[L] for L in range(4)] == [3840, 1920, 960, 480]
    assert [lay.height[L] for L in range(4)] == [2160, 1080, 540, 270]
    off = 0
    for L in range(1, 4):
        assert lay.offset[L] == off and off % 256 == 0
        off += -(-lay.width[L] * lay.height[L] * 16 // 256) * 256
    assert lay.total_bytes == off
    # ragged sizes round up; levels of a deeper layout sit at the same offsets
    lay6 = pkg.mip_layout(37, 21, 6)
    assert [lay6.width[L] for L in range(6)] == [37, 19, 10, 5, 3, 2]
    assert [lay6.height[L] for L in range(6)] == [21, 11, 6, 3, 2, 1]
    lay3 = pkg.mip_layout(37, 21, 3)
    assert list(lay3.offset)[:3] == list(lay6.offset)[:3]
    assert pkg.mip_layout(5, 5, 1).total_bytes == 0
    for bad in ((0, 5, 2), (5, 5, 0), (5, 5, 7), (1 << 16, 1 << 15, 2)):
        with pytest.raises(pkg.WrsError):
            pkg.mip_layout(*bad)


def test_foveate_host_checks_before_any_cuda_call(lib):
    # every failure below is decided on the host from the arguments alone;
    # the pointers are never dereferenced
    fake = C.c_void_p(1 << 20)
    r = (C.c_float * 2)(2.0, 1.0)
    assert lib.wrs_foveate(fake, 48, fake, 4096, 16, 8, 2, r, 8.0, 4.0, 0, fake, 48, None,
                           None) == _lib.WRS_ERR_ARG
    assert b"ascending" in lib.wrs_last_error()
    r = (C.c_float * 1)(2.0)
    assert lib.wrs_foveate(fake, 48, fake, 4096, 16, 8, 1, r, 8.0, 4.0, 2, fake, 48, None,
                           None) == _lib.WRS_ERR_ARG
    assert lib.wrs_foveate(fake, 47, fake, 4096, 16, 8, 1, r, 8.0, 4.0, 0, fake, 48, None,
                           None) == _lib.WRS_ERR_ARG
    assert lib.wrs_foveate(fake, 48, fake, 16, 16, 8, 1, r, 8.0, 4.0, 0, fake, 48, None,
                           None) == _lib.WRS_ERR_BUDGET
    assert lib.wrs_foveate(fake, 48, fake, 4096, 16, 8, 0, r, 8.0, 4.0, 0, fake, 48, None,
                           None) == _lib.WRS_ERR_ARG
    assert lib.wrs_mip_build(fake, 48, 16, 8, 3, fake, 16, None) == _lib.WRS_ERR_BUDGET
    assert lib.wrs_mip_build(None, 48, 16, 8, 3, fake, 4096, None) == _lib.WRS_ERR_ARG
    assert lib.wrs_mip_build(fake, 48, 16, 8, 3, C.c_void_p((1 << 20) + 16), 4096,
                             None) == _lib.WRS_ERR_ARG


def test_host_paths_check_arguments_before_any_cuda_call(lib):
    assert lib.wrs_host_pipe_stage_bytes(None, 0) == 0
    out = C.c_void_p()
    assert lib.wrs_host_pipe_create(None, C.c_void_p(1 << 20), 1 << 20, 0, C.byref(out)) == _lib.WRS_ERR_ARG
    assert lib.wrs_host_pipe_push(None, None, 0.0, 0.0, None, None) == _lib.WRS_ERR_ARG
    assert lib.wrs_host_pipe_finish(None) == _lib.WRS_ERR_ARG
    assert lib.wrs_host_pipe_destroy(None) == _lib.WRS_OK
    assert lib.wrs_push_frame_host_noalloc(None, None, 0.0, 0.0, None, None, None) == _lib.WRS_ERR_ARG
    assert b"context" in lib.wrs_last_error()
    text = open(_lib.HEADER).read()
    assert "#define WRS_NOALLOC_MAX_PIXELS 8294400" in text
