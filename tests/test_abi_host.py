"""Host-side checks of the C ABI that need no GPU.

The shared library must load and export every entry point include/decolor.h
declares; the ctypes mirrors must match the C struct sizes; argument validation and
workspace sizing run entirely on the host, so they are exercised here (no kernel is
launched by any of these calls: every call below fails validation or only sizes).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "decolor.h")


@pytest.fixture(scope="module")
def abi():
    from paper_2108_13656_gb300 import _abi, build_lib
    build_lib.build()
    _abi.load()
    return _abi


def _declared_symbols():
    text = open(HEADER).read()
    return re.findall(r"DC_API\s+[\w\s\*]+?\b(dc_\w+)\s*\(", text)


def test_header_declares_the_three_calls():
    syms = _declared_symbols()
    for name in ("dc_decolorize", "dc_decolorize_tonemap_global", "dc_decolorize_tonemap_local",
                 "dc_workspace_bytes", "dc_query_status", "dc_status_string"):
        assert name in syms


def test_library_exports_every_declared_symbol(abi):
    lib = abi.load()
    syms = _declared_symbols()
    assert len(syms) >= 10
    for name in syms:
        assert hasattr(lib, name), name
        assert name in abi._SIGS, "binding lacks " + name
    assert lib.dc_version() == 200


def test_struct_sizes(abi):
    assert ctypes.sizeof(abi.dc_image_in) == 32
    assert ctypes.sizeof(abi.dc_image_out) == 24
    assert ctypes.sizeof(abi.dc_decolor_params) == 16
    assert ctypes.sizeof(abi.dc_video_state) == 1056
    assert ctypes.sizeof(abi.dc_global_params) == 16
    assert ctypes.sizeof(abi.dc_local_params) == 24
    assert ctypes.sizeof(abi.dc_tuning) == 16
    assert abi.STATS_BYTES == 1056


def _img(w, h, dt=0, stride=None, ptr=1 << 20):
    esz = {0: 1, 1: 2, 2: 4}.get(dt, 1)
    d = None
    from paper_2108_13656_gb300 import _abi
    d = _abi.dc_image_in()
    d.data = ptr
    d.width, d.height = w, h
    d.stride_bytes = stride if stride is not None else 3 * w * esz
    d.dtype = dt
    d.reserved = 0
    return d


def test_workspace_bytes_sizes(abi):
    lib = abi.load()
    ins = (abi.dc_image_in * 1)(_img(3840, 2160))
    g = lib.dc_workspace_min_bytes(abi.DC_OP_GLOBAL, ins, 1, None)
    assert 256 < g < 1 << 20
    # 8-bit input of this size: the optional f32 luminance plane on top
    assert lib.dc_workspace_bytes(abi.DC_OP_GLOBAL, ins, 1, None) >= g + 3840 * 2160 * 4
    lp = abi.local_params()
    loc = lib.dc_workspace_min_bytes(abi.DC_OP_LOCAL, ins, 1, ctypes.byref(lp))
    Hb, Wb = (2160 + 31) // 32, 3840 // 32
    assert loc >= g + Hb * Wb * 32 * 8 + Hb * Wb * 33 * 4
    assert lib.dc_workspace_bytes(abi.DC_OP_LOCAL, ins, 1, ctypes.byref(lp)) >= loc + 3840 * 2160 * 4
    assert lib.dc_workspace_bytes(abi.DC_OP_LOCAL, ins, 1, None) == 0
    assert lib.dc_workspace_min_bytes(abi.DC_OP_LOCAL, ins, 1, None) == 0
    # decolorize never keeps a plane; HDR input keeps it in its f32 output
    assert lib.dc_workspace_bytes(abi.DC_OP_DECOLORIZE, ins, 1, None) == \
        lib.dc_workspace_min_bytes(abi.DC_OP_DECOLORIZE, ins, 1, None)
    hdr = (abi.dc_image_in * 1)(_img(3840, 2160, dt=abi.DC_F32))
    assert lib.dc_workspace_bytes(abi.DC_OP_GLOBAL, hdr, 1, None) == lib.dc_workspace_min_bytes(abi.DC_OP_GLOBAL, hdr, 1, None)
    # the 8-bit plane is asked for whatever the size (optional: the minimum omits it)
    big = (abi.dc_image_in * 1)(_img(4096, 3200))
    assert lib.dc_workspace_bytes(abi.DC_OP_GLOBAL, big, 1, None) >= \
        lib.dc_workspace_min_bytes(abi.DC_OP_GLOBAL, big, 1, None) + 4096 * 3200 * 4
    assert lib.dc_workspace_bytes(7, ins, 1, None) == 0
    many = (abi.dc_image_in * 300)(*[_img(64 + i, 32) for i in range(300)])
    assert lib.dc_workspace_bytes(abi.DC_OP_GLOBAL, many, 300, None) > 0


@pytest.mark.parametrize("bad", [
    dict(width=0), dict(height=0), dict(dtype=9), dict(stride=10), dict(ptr=0),
])
def test_invalid_inputs_rejected(abi, bad):
    lib = abi.load()
    d = _img(16, 4, dt=bad.get("dtype", 0), stride=bad.get("stride"), ptr=bad.get("ptr", 1 << 20))
    if "width" in bad:
        d.width = bad["width"]
    if "height" in bad:
        d.height = bad["height"]
    ins = (abi.dc_image_in * 1)(d)
    assert lib.dc_workspace_bytes(abi.DC_OP_DECOLORIZE, ins, 1, None) == 0
    out = (abi.dc_image_out * 1)(abi.dc_image_out(1 << 22, 16, 0, 0))
    p = abi.dc_decolor_params(0.55, 0.8)
    rc = lib.dc_decolorize(ins, out, 1, ctypes.byref(p), ctypes.c_void_p(1 << 12), 1 << 20, None)
    assert rc in (abi.DC_ERR_INVALID_ARG, abi.DC_ERR_UNSUPPORTED_DTYPE)


def test_invalid_params_and_workspace(abi):
    lib = abi.load()
    ins = (abi.dc_image_in * 1)(_img(16, 4))
    out = (abi.dc_image_out * 1)(abi.dc_image_out(1 << 22, 16, 0, 0))
    p = abi.dc_decolor_params(1.5, 0.8)
    assert lib.dc_decolorize(ins, out, 1, ctypes.byref(p), ctypes.c_void_p(1 << 12), 1 << 20, None) == abi.DC_ERR_INVALID_ARG
    p = abi.dc_decolor_params(0.55, 0.8)
    # workspace: NULL, misaligned, too small
    assert lib.dc_decolorize(ins, out, 1, ctypes.byref(p), None, 1 << 20, None) == abi.DC_ERR_WORKSPACE
    assert lib.dc_decolorize(ins, out, 1, ctypes.byref(p), ctypes.c_void_p((1 << 12) + 8), 1 << 20, None) == abi.DC_ERR_WORKSPACE
    assert lib.dc_decolorize(ins, out, 1, ctypes.byref(p), ctypes.c_void_p(1 << 12), 16, None) == abi.DC_ERR_WORKSPACE
    g = abi.dc_global_params(5, 1.0, 1e-4, 0)
    assert lib.dc_decolorize_tonemap_global(ins, out, 1, ctypes.byref(p), ctypes.byref(g), None,
                                            ctypes.c_void_p(1 << 12), 1 << 20, None) == abi.DC_ERR_INVALID_ARG
    g = abi.dc_global_params(0, 1.0, 0.0, 0)
    assert lib.dc_decolorize_tonemap_global(ins, out, 1, ctypes.byref(p), ctypes.byref(g), None,
                                            ctypes.c_void_p(1 << 12), 1 << 20, None) == abi.DC_ERR_INVALID_ARG
    for lp in [abi.local_params(block_s=0), abi.local_params(bins=33), abi.local_params(radius_blocks=17),
               abi.local_params(alpha=2.0)]:
        assert lib.dc_decolorize_tonemap_local(ins, out, 1, ctypes.byref(p), ctypes.byref(lp),
                                               ctypes.c_void_p(1 << 12), 1 << 20, None) == abi.DC_ERR_INVALID_ARG
    # overlapping input and output
    ov = (abi.dc_image_out * 1)(abi.dc_image_out(1 << 20, 16, 0, 0))
    assert lib.dc_decolorize(ins, ov, 1, ctypes.byref(p), ctypes.c_void_p(1 << 12), 1 << 20, None) == abi.DC_ERR_INVALID_ARG
    # batch limits
    assert lib.dc_decolorize(ins, out, 0, ctypes.byref(p), ctypes.c_void_p(1 << 12), 1 << 20, None) == abi.DC_ERR_INVALID_ARG
    assert lib.dc_decolorize(ins, out, 5000, ctypes.byref(p), ctypes.c_void_p(1 << 12), 1 << 20, None) == abi.DC_ERR_TOO_MANY


def test_tuning_table_validation(abi):
    orig = abi.get_tuning(abi.DC_OP_GLOBAL, abi.DC_U8)
    with pytest.raises(abi.DcError):
        abi.set_tuning(abi.DC_OP_GLOBAL, abi.DC_U8, 256, 1, 20)  # not a multiple of 16
    with pytest.raises(abi.DcError):
        abi.set_tuning(abi.DC_OP_GLOBAL, abi.DC_U8, 100, 1, 4096)
    abi.set_tuning(abi.DC_OP_GLOBAL, abi.DC_U8, 256, 2, 8192, 4)
    assert abi.get_tuning(abi.DC_OP_GLOBAL, abi.DC_U8) == (256, 2, 8192, 4)
    abi.set_tuning(abi.DC_OP_GLOBAL, abi.DC_U8, *orig)


def test_status_strings(abi):
    assert abi.status_string(abi.DC_ERR_TIMEOUT).startswith("device-side")
    assert abi.status_string(0) == "ok"


def _lcm16(s):
    import math
    return s // math.gcd(s, 16) * 16


def _tiles(sizes, s, w):
    return sum(((h + s - 1) // s) * ((wd + w - 1) // w) for h, wd in sizes)


@pytest.mark.parametrize("s", [1, 8, 16, 24, 32, 64])
@pytest.mark.parametrize("sizes", [[(2160, 3840)], [(4320, 7680)], [(1440, 2560)], [(97, 333)], [(64, 64)],
                                   [(2160, 3840), (480, 640), (1080, 1920)]])
def test_automatic_local_tile_width_is_a_valid_tiling(abi, s, sizes):
    # automatic width (the default): a multiple of lcm(s, 16), at most 1024 pixels,
    # and the busiest CTA of the persistent grid (CTA c takes tiles c, c + grid, ...)
    # covers hardly more pixels than with the 512-pixel tiling
    w = abi.local_tile_cols(sizes, block_s=s, in_dtype=abi.DC_U8, n_sm=152)
    assert w % _lcm16(s) == 0 and 0 < w <= 1024
    slots = 152 * 4

    def busiest(w_):
        px = [min(s, h - r0) * min(w_, wd - c * w_) for h, wd in sizes
              for r0 in range(0, h, s) for c in range(-(-wd // w_))]
        grid = min(len(px), slots)
        load = [0] * grid
        for t, p in enumerate(px):
            load[t % grid] += p
        return max(load)

    l = _lcm16(s)
    m = max(1, 512 // l)
    while m > 1 and (l * m // s > 32 or l * m > 1024):  # at most 32 blocks per tile
        m -= 1
    w512 = l * m
    assert busiest(w) <= 1.1 * busiest(w512)


def test_automatic_local_tile_width_fills_the_grid(abi):
    # 2560x1440, 32-pixel blocks: 512-pixel tiles give 225 tiles for 608 resident
    # CTAs; the balanced width uses most of them in one round
    w = abi.local_tile_cols([(1440, 2560)], block_s=32, n_sm=152)
    t = _tiles([(1440, 2560)], 32, w)
    assert 450 <= t <= 608
    # 3840x2160: one round of equal tiles (15 of the 120 block columns each)
    assert abi.local_tile_cols([(2160, 3840)], block_s=32, n_sm=152) == 480


def test_tuned_local_tile_width_is_kept(abi):
    orig = abi.get_tuning(abi.DC_OP_LOCAL, abi.DC_F32)
    try:
        abi.set_tuning(abi.DC_OP_LOCAL, abi.DC_F32, 256, 32, 512, 0)
        assert abi.local_tile_cols([(2160, 3840)], block_s=32, in_dtype=abi.DC_F32) == 512
        assert abi.local_tile_cols([(2160, 3840)], block_s=24, in_dtype=abi.DC_F32) == 480  # multiple of 48
    finally:
        abi.set_tuning(abi.DC_OP_LOCAL, abi.DC_F32, *orig)
    with pytest.raises(abi.DcError):
        abi.local_tile_cols([(0, 10)])
    with pytest.raises(abi.DcError):
        abi.local_tile_cols([(10, 10)], block_s=65)


def test_host_pipeline_rejects_zero_depth():
    from paper_2108_13656_gb300.pipeline import HostPipeline
    with pytest.raises(ValueError):
        HostPipeline({}, {}, [], depth=0)


def test_call_streams_rejects_zero_streams():
    from paper_2108_13656_gb300.pipeline import CallStreams
    with pytest.raises(ValueError):
        CallStreams(0)


def test_call_streams_workspace_ownership_without_a_device():
    # run() checks the workspace before it touches a stream: a fake call whose
    # workspace address is taken by another side stream is refused until a join
    # (emulated by clearing the table) releases it
    from paper_2108_13656_gb300.pipeline import CallStreams
    cs = CallStreams.__new__(CallStreams)
    cs.streams = ["s0", "s1"]
    cs._owner = {}
    seen = []

    class Fake:
        ws_ptr = 0x1000

        def __call__(self, stream):
            seen.append(stream)

    cs.run(0, Fake())
    cs.run(0, Fake())
    with pytest.raises(ValueError):
        cs.run(1, Fake())
    cs._owner = {}
    cs.run(1, Fake())
    assert seen == ["s0", "s0", "s1"]


def test_new_fields_validated(abi):
    lib = abi.load()
    ins = (abi.dc_image_in * 1)(_img(16, 4))
    out = (abi.dc_image_out * 1)(abi.dc_image_out(1 << 22, 16, 0, 0))
    ws = ctypes.c_void_p(1 << 12)
    g = abi.dc_global_params(0, 1.0, 1e-4, 0)
    for bad in (abi.dc_decolor_params(0.55, 0.8, 4, 1.0), abi.dc_decolor_params(0.55, 0.8, -1, 1.0),
                abi.dc_decolor_params(0.55, 0.8, 0, -0.5), abi.dc_decolor_params(0.55, 0.8, 0, 9.0),
                abi.dc_decolor_params(0.55, 0.8, 0, float("nan"))):
        assert lib.dc_decolorize_tonemap_global(ins, out, 1, ctypes.byref(bad), ctypes.byref(g), None, ws,
                                                1 << 20, None) == abi.DC_ERR_INVALID_ARG
    p = abi.dc_decolor_params(0.55, 0.8, 0, 1.0)
    # 3-channel outputs: only for the tone-mapping calls, and with room for 3 samples a pixel
    col = (abi.dc_image_out * 1)(abi.dc_image_out(1 << 22, 48, 0, 3))
    assert lib.dc_decolorize(ins, col, 1, ctypes.byref(p), ws, 1 << 20, None) == abi.DC_ERR_INVALID_ARG
    narrow = (abi.dc_image_out * 1)(abi.dc_image_out(1 << 22, 47, 0, 3))
    assert lib.dc_decolorize_tonemap_global(ins, narrow, 1, ctypes.byref(p), ctypes.byref(g), None, ws, 1 << 20,
                                            None) == abi.DC_ERR_INVALID_ARG
    two = (abi.dc_image_out * 1)(abi.dc_image_out(1 << 22, 48, 0, 2))
    assert lib.dc_decolorize_tonemap_global(ins, two, 1, ctypes.byref(p), ctypes.byref(g), None, ws, 1 << 20,
                                            None) == abi.DC_ERR_INVALID_ARG
    # a colour output that would overlap its input
    ovl = (abi.dc_image_out * 1)(abi.dc_image_out(0x100000 - 100, 48, 0, 3))
    ins2 = (abi.dc_image_in * 1)(_img(16, 4))
    assert lib.dc_decolorize_tonemap_global(ins2, ovl, 1, ctypes.byref(p), ctypes.byref(g), None, ws, 1 << 20,
                                            None) == abi.DC_ERR_INVALID_ARG


def test_video_arguments_validated(abi):
    lib = abi.load()
    ins = (abi.dc_image_in * 1)(_img(16, 4))
    out = (abi.dc_image_out * 1)(abi.dc_image_out(1 << 22, 16, 0, 0))
    ws = ctypes.c_void_p(1 << 12)
    p = abi.dc_decolor_params(0.55, 0.8, 0, 1.0)
    g = abi.dc_global_params(0, 1.0, 1e-4, 0)
    st = ctypes.c_void_p(1 << 24)
    call = lib.dc_decolorize_tonemap_video
    assert call(ins, out, 1, ctypes.byref(p), ctypes.byref(g), 1.0, 0, None, ws, 1 << 20, None) == abi.DC_ERR_INVALID_ARG
    assert call(ins, out, 1, ctypes.byref(p), ctypes.byref(g), 1.0, 2, st, ws, 1 << 20, None) == abi.DC_ERR_INVALID_ARG
    for lam in (0.0, -0.1, 1.5, float("nan")):
        assert call(ins, out, 1, ctypes.byref(p), ctypes.byref(g), lam, 0, st, ws, 1 << 20, None) == abi.DC_ERR_INVALID_ARG
    h = abi.dc_global_params(1, 1.0, 1e-4, 0)  # histogram equalisation: accepted (no GPU here: the launch fails)
    assert call(ins, out, 1, ctypes.byref(p), ctypes.byref(h), 1.0, 0, st, ws, 1 << 20, None) in (abi.DC_OK, abi.DC_ERR_CUDA)


def test_presets(abi):
    lib = abi.load()
    p, lp = abi.dc_decolor_params(), abi.dc_local_params()
    expect = {abi.DC_PRESET_PAPER: 0.8, abi.DC_PRESET_TM1: 0.55, abi.DC_PRESET_TM2: 0.95}
    for code, bk in expect.items():
        assert lib.dc_preset(code, ctypes.byref(p), ctypes.byref(lp)) == 0
        assert p.beta_r == pytest.approx(0.55) and p.beta_k == pytest.approx(bk)
        assert 0.5 < p.beta_k < 1 and p.luma == abi.DC_LUMA_OURS and p.color_s == 1.0
        assert (lp.block_s, lp.radius_blocks, lp.bins, lp.alpha) == (32, 2, 32, 1.0)
    assert lib.dc_preset(3, ctypes.byref(p), None) == abi.DC_ERR_INVALID_ARG
    assert lib.dc_preset(abi.DC_PRESET_TM1, None, None) == 0


def test_local_video_arguments_validated(abi):
    lib = abi.load()
    ins = (abi.dc_image_in * 1)(_img(100, 70))
    out = (abi.dc_image_out * 1)(abi.dc_image_out(1 << 24, 400, 2, 0))
    lp = abi.dc_local_params(32, 2, 32, 1.0, 1e-4, 0)
    # a 256-byte header and 3 x 4 blocks x 33 tables of 4 bytes, 256-aligned
    assert lib.dc_video_local_state_bytes(ins, 1, ctypes.byref(lp)) == 256 + ((3 * 4 * 33 * 4 + 255) // 256) * 256
    assert lib.dc_video_local_state_bytes(ins, 1, None) == 0
    p = abi.dc_decolor_params(0.55, 0.8, 0, 1.0)
    ws = ctypes.c_void_p(1 << 12)
    st = 1 << 26
    need = lib.dc_video_local_state_bytes(ins, 1, ctypes.byref(lp))
    call = lib.dc_decolorize_tonemap_local_video
    assert call(ins, out, 1, ctypes.byref(p), ctypes.byref(lp), 0, None, need, ws, 1 << 20, None) == abi.DC_ERR_INVALID_ARG
    assert call(ins, out, 1, ctypes.byref(p), ctypes.byref(lp), 0, ctypes.c_void_p(st + 16), need, ws, 1 << 20,
                None) == abi.DC_ERR_INVALID_ARG   # misaligned state
    assert call(ins, out, 1, ctypes.byref(p), ctypes.byref(lp), 0, ctypes.c_void_p(st), need - 1, ws, 1 << 20,
                None) == abi.DC_ERR_INVALID_ARG   # too small
    assert call(ins, out, 1, ctypes.byref(p), ctypes.byref(lp), 3, ctypes.c_void_p(st), need, ws, 1 << 20,
                None) == abi.DC_ERR_INVALID_ARG   # restart not 0 / 1
    # colour outputs are accepted (the launch itself fails here, with no GPU)
    col = (abi.dc_image_out * 1)(abi.dc_image_out(1 << 24, 1200, 2, 3))
    assert call(ins, col, 1, ctypes.byref(p), ctypes.byref(lp), 1, ctypes.c_void_p(st), need, ws, 1 << 20,
                None) in (abi.DC_OK, abi.DC_ERR_CUDA)
    narrow = (abi.dc_image_out * 1)(abi.dc_image_out(1 << 24, 1199, 2, 3))
    assert call(ins, narrow, 1, ctypes.byref(p), ctypes.byref(lp), 1, ctypes.c_void_p(st), need, ws, 1 << 20,
                None) == abi.DC_ERR_INVALID_ARG


def test_workspace_growth_rules_without_a_device():
    # the sizes a Workspace grows to, with a small host buffer standing in for device
    # memory: optional=False (the serving loop) grows only to a call's least need, so
    # the optional 8-bit plane is used only while it fits; the default grows to the
    # size the call asks for
    from paper_2108_13656_gb300 import _abi

    class FakeBuf:
        def __init__(self, n):
            self.n = n

        def numel(self):
            return self.n

        def data_ptr(self):
            return 1 << 20

    def make(optional):
        w = _abi.Workspace.__new__(_abi.Workspace)
        w.device, w.buf, w.fixed, w.optional = "cpu", None, False, optional
        w._set = lambda buf: setattr(w, "buf", FakeBuf(buf.numel()))
        return w

    K = 1 << 10
    w = make(optional=False)
    w.get(128 * K)                     # sized up front
    n0 = w.buf.numel()
    assert n0 >= 128 * K
    w.get(400 * K, 64 * K)             # asks for more, accepts less than it holds: no growth
    assert w.buf.numel() == n0
    w.get(400 * K, 200 * K)            # its least need is more: grows to that, not to what it asks
    assert 200 * K <= w.buf.numel() < 400 * K
    g = make(optional=True)
    g.get(128 * K)
    g.get(400 * K, 64 * K)
    assert g.buf.numel() >= 400 * K
