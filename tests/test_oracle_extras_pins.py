"""Pins of the oracle's comparison channels, colour reconstruction and frame-sequence
estimate against what the paper and the mathematics fix.

- Comparison channels (Sec. I quotes MATLAB's rgb2gray weights; Fig. GTMO and
  Sec. III-B-1 compare with V of HSV): hand-computed values, and the two statements
  of Sec. III-B-1 about them (V treats primaries and white alike; Y gives blue a very
  low luminance).
- Colour reconstruction (no formula in the paper; the reading is
  C_out = min(1, y (C/L)^s)): achromatic and black pixels, s = 0, closed forms for
  primaries, the clamp, and the fact that re-decolorizing the output with the same
  1-homogeneous channel gives back y.
- Frame sequences (no scheme in the paper; the reading is a carried log-mean
  m_t = (1 - lambda) m_{t-1} + lambda mu_t): the update in closed form, two-level
  achromatic sequences in closed form, and a still sequence equal to per-frame global
  tone mapping.
"""
import math

import numpy as np
import pytest

import oracle

SQ = math.sqrt


# ------------------------------------------------------------ channels ----
@pytest.mark.parametrize("rgb,y", [((1, 0, 0), 0.2989), ((0, 1, 0), 0.5870), ((0, 0, 1), 0.1140),
                                   ((0.2, 0.4, 0.6), 0.05978 + 0.2348 + 0.0684),
                                   ((0.5, 0.5, 0.5), 0.49995)])
def test_rgb2gray_weights(rgb, y):
    assert oracle.luma(*rgb, oracle.LUMA_Y) == pytest.approx(y, abs=1e-15)


@pytest.mark.parametrize("rgb,v", [((1, 0, 0), 1.0), ((0.2, 0.9, 0.4), 0.9), ((0.3, 0.3, 0.31), 0.31),
                                   ((0, 0, 0), 0.0), ((1, 1, 1), 1.0)])
def test_hsv_value(rgb, v):
    assert oracle.luma(*rgb, oracle.LUMA_V) == v


def test_channel_statements_of_the_global_tone_mapping_section():
    # V treats primary colours and white the same way
    assert oracle.luma(1, 0, 0, oracle.LUMA_V) == oracle.luma(0, 0, 1, oracle.LUMA_V) == oracle.luma(1, 1, 1, oracle.LUMA_V)
    # Y gives blue a very low luminance (the sky turns too dark); ours does not
    assert oracle.luma(0, 0, 1, oracle.LUMA_Y) < 0.2 < oracle.luma(0, 0, 1, oracle.LUMA_OURS)
    # Y weights red little (the red fish merges with its background); ours lifts warm colours
    assert oracle.luma(1, 0, 0, oracle.LUMA_Y) < oracle.luma(1, 0, 0, oracle.LUMA_OURS)


def test_decolorize_channel_on_an_image():
    img = np.array([[[255, 0, 0], [0, 255, 0]], [[0, 0, 255], [51, 102, 153]]], dtype=np.uint8)
    Y = oracle.decolorize(img, channel=oracle.LUMA_Y)
    np.testing.assert_allclose(Y, [[0.2989, 0.5870], [0.1140, 0.2 * 0.2989 + 0.4 * 0.5870 + 0.6 * 0.1140]],
                               rtol=0, atol=1e-15)
    V = oracle.decolorize(img, channel=oracle.LUMA_V)
    np.testing.assert_array_equal(V, [[1.0, 1.0], [1.0, 0.6]])
    ours = oracle.decolorize(img, channel=oracle.LUMA_OURS)
    np.testing.assert_array_equal(ours, oracle.decolorize(img))


def test_unknown_channel_rejected():
    with pytest.raises(ValueError):
        oracle.decolorize(np.zeros((2, 2, 3), np.uint8), channel=4)
    assert math.isnan(oracle.luma(1, 0, 0, 7))


# ------------------------------------------------------ colour reconstruction ----
def _rec(rgb, y, s, channel=oracle.LUMA_OURS):
    img = np.array([[rgb]], dtype=np.float32)
    L = oracle.decolorize(img, channel=channel)
    return oracle.color_reconstruct(img, L, np.array([[y]]), s)[0, 0]


@pytest.mark.parametrize("s", [0.0, 0.5, 1.0, 1.7])
def test_achromatic_pixel_keeps_gray(s):
    np.testing.assert_allclose(_rec((0.3, 0.3, 0.3), 0.62, s), [0.62] * 3, rtol=0, atol=1e-15)


def test_black_pixel_is_achromatic():
    np.testing.assert_array_equal(_rec((0.0, 0.0, 0.0), 0.4, 1.0), [0.4] * 3)
    np.testing.assert_array_equal(_rec((0.0, 0.0, 0.0), 0.4, 0.0), [0.4] * 3)


def test_zero_saturation_gives_gray_everywhere():
    np.testing.assert_array_equal(_rec((0.9, 0.1, 0.0), 0.3, 0.0), [0.3] * 3)  # 0^0 = 1 for the black channel


def test_pure_red_closed_form():
    L = SQ(0.8 * 0.55)  # pure red, Eq. 1-6
    np.testing.assert_allclose(_rec((1.0, 0.0, 0.0), 0.5, 1.0), [0.5 / L, 0.0, 0.0], rtol=1e-15, atol=0)
    np.testing.assert_allclose(_rec((1.0, 0.0, 0.0), 0.3, 2.0), [0.3 / L ** 2, 0.0, 0.0], rtol=1e-15, atol=0)
    np.testing.assert_allclose(_rec((1.0, 0.0, 0.0), 0.5, 0.5), [0.5 / SQ(L), 0.0, 0.0], rtol=1e-15, atol=0)


def test_clamp_at_one():
    # pure green decolorizes to sqrt(0.8/3) = 0.516, so y = 0.9 would need 1.74
    np.testing.assert_array_equal(_rec((0.0, 1.0, 0.0), 0.9, 1.0), [0.0, 1.0, 0.0])


def test_ratios_kept_at_unit_saturation():
    out = _rec((0.6, 0.3, 0.15), 0.35, 1.0)
    assert out[0] / out[1] == pytest.approx(2.0, rel=1e-14)
    assert out[1] / out[2] == pytest.approx(2.0, rel=1e-14)


@pytest.mark.parametrize("channel", [oracle.LUMA_OURS, oracle.LUMA_Y, oracle.LUMA_V])
def test_redecolorized_colour_output_is_y(channel):
    # every channel is 1-homogeneous, so L(y C / L(C)) = y wherever nothing clamps
    rng = np.random.default_rng(3)
    img = (rng.random((16, 16, 3)) * 255).astype(np.uint8)
    L = oracle.decolorize(img, channel=channel)
    cmax = img.max(axis=2) / 255.0
    y = rng.random(L.shape) * 0.9 * L / np.maximum(cmax, 1e-9)  # small enough that no channel clamps
    out = oracle.color_reconstruct(img, L, y, 1.0)
    assert out.max() < 1.0
    back = oracle.decolorize(out.astype(np.float32), channel=channel)
    ok = L > 0
    np.testing.assert_allclose(back[ok], y[ok], rtol=1e-6, atol=1e-7)  # f32 storage of out


def test_reconstruction_with_8bit_codes_uses_the_code_ratio():
    img = np.array([[[200, 100, 50]]], dtype=np.uint8)
    L = oracle.decolorize(img)
    out = oracle.color_reconstruct(img, L, np.array([[0.3]]), 1.0)[0, 0]
    np.testing.assert_allclose(out, [0.3 * 200 / 255 / L[0, 0], 0.3 * 100 / 255 / L[0, 0], 0.3 * 50 / 255 / L[0, 0]],
                               rtol=1e-15)


# --------------------------------------------------------- frame sequences ----
def test_mu_update_closed_form():
    assert oracle.video_mu_update(2.0, -1.0, 1.0) == -1.0
    assert oracle.video_mu_update(2.0, -1.0, 0.25) == 0.75 * 2.0 + 0.25 * -1.0
    assert oracle.video_mu_update(0.5, 0.5, 0.3) == pytest.approx(0.5, abs=1e-16)


def _gray_frame(code, H=4, W=6):
    return np.full((H, W, 3), code, dtype=np.uint8)


@pytest.mark.parametrize("lam", [1.0, 0.5, 0.1])
def test_two_level_sequence_closed_form(lam):
    d = 1e-4
    a, b = 40 / 255, 200 / 255  # achromatic frames: L is the gray value itself
    ys, ms = oracle.tonemap_video_global([_gray_frame(40), _gray_frame(200), _gray_frame(200)], lam=lam, delta=d)
    np.testing.assert_allclose(ys[0], 0.5, rtol=0, atol=1e-15)              # centred on its own log-mean
    np.testing.assert_allclose(ys[1], (b + d) / ((b + d) + (a + d)), rtol=1e-14)  # around frame 0's log-mean
    m1 = (1 - lam) * math.log(a + d) + lam * math.log(b + d)
    assert ms[0] == pytest.approx(math.log(a + d), rel=1e-15)
    assert ms[1] == pytest.approx(m1, rel=1e-14)
    np.testing.assert_allclose(ys[2], (b + d) / ((b + d) + math.exp(m1)), rtol=1e-13)


def test_still_sequence_equals_per_frame_global():
    from paper_2108_13656_gb300 import synth
    img = synth.s_ldr(48, 32, seed=9)
    y_ref, st = oracle.tonemap_global(img)
    ys, ms = oracle.tonemap_video_global([img] * 4, lam=0.3)
    for y, m in zip(ys, ms):
        np.testing.assert_allclose(y, y_ref, rtol=0, atol=1e-15)
        assert m == pytest.approx(st["mu"], rel=1e-14)


# ------------------------------------------------- local frame sequences ----
@pytest.mark.parametrize("kind", ["u8", "f32"])
def test_local_still_sequence_equals_per_frame(kind):
    from paper_2108_13656_gb300 import synth
    img = synth.s_ldr(70, 45, 3) if kind == "u8" else synth.s_hdr(70, 45, 3)
    ref = oracle.tonemap_local(img, block_s=16, bins=12)
    for y in oracle.tonemap_video_local([img] * 3, block_s=16, bins=12):
        np.testing.assert_array_equal(y, ref)


def test_local_sequence_through_a_constant_frame_closed_form():
    # frame 0 is a constant gray u0 = 100/255: every block histogram has its tent mass
    # split (1 - f, f) between bins j, j+1 (x0 = B u0 - 1/2 = j + f), so every block's
    # cumulative table is 0 up to bin j, rises by 1 - f over bin j and by f over bin
    # j+1; frame 1 (a gray ramp) is mapped through that single curve
    B, c0 = 8, 100
    u0 = c0 / 255
    x0 = B * u0 - 0.5
    j, f = int(math.floor(x0)), x0 - math.floor(x0)
    H, W = 24, 64
    ramp = np.tile(np.arange(W, dtype=np.float64)[None, :] * 4.0, (H, 1)).astype(np.uint8)
    frame1 = np.repeat(ramp[:, :, None], 3, axis=2)
    ys = oracle.tonemap_video_local([_gray_frame(c0, H, W), frame1], block_s=8, radius_blocks=1, bins=B)
    u = ramp.astype(np.float64) / 255
    x = B * u
    expect = np.where(x < j, 0.0, np.where(x < j + 1, (1 - f) * (x - j),
                      np.where(x < j + 2, (1 - f) + f * (x - j - 1), 1.0)))
    np.testing.assert_allclose(ys[1], expect, rtol=0, atol=1e-12)


def test_local_sequence_range_follows_one_frame_behind():
    # HDR frame 1 = frame 0 with one pixel far brighter: its coordinates are taken in
    # frame 0's log range and it is mapped through frame 0's tables, so every other
    # pixel gives exactly frame 0's output and the bright one clamps to u = 1, F = 1;
    # frame 2 (the same as frame 1) is taken in frame 1's own, wider range
    from paper_2108_13656_gb300 import synth
    f0 = synth.s_hdr(48, 32, 5)
    f1 = f0.copy()
    f1[7, 9] = f0.max() * 1e3
    ys = oracle.tonemap_video_local([f0, f1, f1], block_s=8, bins=16)
    other = np.ones(f0.shape[:2], bool)
    other[7, 9] = False
    np.testing.assert_array_equal(ys[1][other], ys[0][other])
    assert ys[1][7, 9] == 1.0
    assert np.abs(ys[2][other] - ys[1][other]).max() > 1e-3


# ------------------------------------------------------------ CIE L* ----
D = 6.0 / 29.0


@pytest.mark.parametrize("Y,lstar", [
    (1.0, 1.0),                       # reference white: L* = 100
    (0.0, 0.0),
    ((66.0 / 116.0) ** 3, 0.5),       # f(Y) = 66/116 on the cube-root branch: L* = 50
    (D ** 3, 0.08),                   # the branch point: f = 6/29 on both sides, L* = 8
    (D ** 3 / 2, 0.04),               # linear branch: f = 1/29 + 4/29 = 5/29, L* = 4
])
def test_lstar_closed_forms(Y, lstar):
    # achromatic linear samples: Rec. 709 luminance Y equals the sample (weights sum to 1)
    assert oracle.luma(Y, Y, Y, oracle.LUMA_LSTAR) == pytest.approx(lstar, abs=1e-12)


def test_lstar_of_srgb_red():
    # Y = 0.2126 for linear red: L* = 116 cbrt(0.2126) - 16
    assert oracle.luma(1, 0, 0, oracle.LUMA_LSTAR) == pytest.approx((116 * 0.2126 ** (1 / 3) - 16) / 100, abs=1e-14)


def test_lstar_decodes_8bit_srgb():
    img = np.array([[[255, 255, 255], [0, 0, 0], [10, 10, 10], [200, 200, 200]]], dtype=np.uint8)
    L = oracle.decolorize(img, channel=oracle.LUMA_LSTAR)[0]
    assert L[0] == pytest.approx(1.0, abs=1e-15) and L[1] == 0.0
    c = 10 / 255  # on the linear segment of the sRGB curve (c <= 0.04045): Y = c / 12.92 < (6/29)^3
    Y = c / 12.92
    assert L[2] == pytest.approx(116 * (Y / (3 * D * D)) / 100, rel=1e-12)
    Y = ((200 / 255 + 0.055) / 1.055) ** 2.4
    assert L[3] == pytest.approx((116 * Y ** (1 / 3) - 16) / 100, rel=1e-12)


def test_video_colour_of_a_still_sequence_is_the_colour_call():
    from paper_2108_13656_gb300 import synth
    img = synth.s_ldr(40, 24, seed=12)
    ys, _ = oracle.tonemap_video_global([img] * 3, lam=0.4)
    for c in oracle.video_color([img] * 3, ys, s=0.7):
        np.testing.assert_array_equal(c, oracle.tonemap_global_color(img, s=0.7))
    ysl = oracle.tonemap_video_local([img] * 2, block_s=8)
    for c in oracle.video_color([img] * 2, ysl):
        np.testing.assert_array_equal(c, oracle.tonemap_local_color(img, block_s=8))


@pytest.mark.parametrize("kind", ["u8", "f32"])
def test_histeq_still_sequence_equals_per_frame(kind):
    from paper_2108_13656_gb300 import synth
    img = synth.s_ldr(50, 30, 4) if kind == "u8" else synth.s_hdr(50, 30, 4)
    ref, _ = oracle.tonemap_global(img, mode=oracle.MODE_HISTEQ)
    for y in oracle.tonemap_video_histeq([img] * 3):
        np.testing.assert_array_equal(y, ref)


def test_histeq_sequence_through_a_two_level_frame_closed_form():
    # frame 0: half black (code 0), half white (code 255): its cumulative histogram is
    # 1/2 for every code below 255 and 1 at 255, so frame 1 (a gray ramp) maps to 1/2
    # everywhere except its white pixels
    H, W = 8, 64
    f0 = np.zeros((H, W, 3), np.uint8)
    f0[:, W // 2:] = 255
    ramp = np.tile((np.arange(W) * 255 // (W - 1)).astype(np.uint8)[None, :], (H, 1))
    f1 = np.repeat(ramp[:, :, None], 3, axis=2)
    ys = oracle.tonemap_video_histeq([f0, f1])
    expect = np.where(ramp == 255, 1.0, 0.5)
    np.testing.assert_allclose(ys[1], expect, rtol=0, atol=1e-15)


def test_histeq_sequence_range_follows_one_frame_behind():
    from paper_2108_13656_gb300 import synth
    f0 = synth.s_hdr(40, 24, 6)
    f1 = f0.copy()
    f1[3, 5] = f0.max() * 1e3  # beyond frame 0's range: clamps to u = 1
    ys = oracle.tonemap_video_histeq([f0, f1])
    other = np.ones(f0.shape[:2], bool)
    other[3, 5] = False
    np.testing.assert_array_equal(ys[1][other], ys[0][other])
    assert ys[1][3, 5] == 1.0
