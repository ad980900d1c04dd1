"""Pins for the oracle's tone-mapping passes (Sec. III-B).

The paper names the global curve only as a "centred sigmoid" (Sec. III-B-1) and the
local operator only as smoothed local-histogram equalisation built from local
cumulative histograms (Sec. III-B-2); the readings are in oracle/decolor_oracle.c.
These tests pin the oracle with closed forms (centre point, two-level images,
constant images), textbook histogram equalisation (rank counting with numpy),
symmetry, and a brute-force pure-Python evaluation of the local definition on tiny
images that sums window pixels directly instead of going through block histograms.
"""
import math

import numpy as np
import pytest


def _gray_u8(codes):
    codes = np.asarray(codes, dtype=np.uint8)
    return np.repeat(codes[..., None], 3, axis=-1)


def _gray_f32(vals):
    vals = np.asarray(vals, dtype=np.float32)
    return np.repeat(vals[..., None], 3, axis=-1)


# ----------------------------------------------------------------- sigmoid ----
def test_sigmoid_centre_and_two_levels(oracle_mod):
    delta = 1e-4
    a, b = 0.02, 3.0
    m = math.sqrt((a + delta) * (b + delta)) - delta
    img = _gray_f32([[a, b, m]])
    L = oracle_mod.decolorize(img)  # achromatic: L is the stored sample
    y, st = oracle_mod.tonemap_global_plane(L, ldr=False, mode=oracle_mod.MODE_SIGMOID, k=1.0, delta=delta)
    a32, b32, m32 = (float(np.float32(v)) for v in (a, b, m))
    mu = (math.log(a32 + delta) + math.log(b32 + delta) + math.log(m32 + delta)) / 3
    assert st["mu"] == pytest.approx(mu, rel=1e-15)
    # centre: ln(L + delta) = mu maps to exactly 1/2 (up to the f32 storage of m)
    assert y[0, 2] == pytest.approx(0.5, abs=1e-7)
    # k = 1: y = (L + delta) / (L + delta + e^mu)
    for i, v32 in enumerate([a32, b32]):
        assert y[0, i] == pytest.approx((v32 + delta) / (v32 + delta + math.exp(mu)), rel=1e-14)


def test_sigmoid_constant_image_is_half(oracle_mod):
    for c in [0, 17, 128, 255]:
        y, _ = oracle_mod.tonemap_global(_gray_u8(np.full((3, 5), c)))
        np.testing.assert_allclose(y, 0.5, atol=1e-15)


def test_sigmoid_monotone_and_gain_zero(oracle_mod, ):
    from paper_2108_13656_gb300 import synth
    img = synth.s_hdr(64, 48, seed=3)
    L = oracle_mod.decolorize(img)
    y, _ = oracle_mod.tonemap_global_plane(L, ldr=False)
    order = np.argsort(L, axis=None, kind="stable")
    assert np.all(np.diff(y.ravel()[order]) >= 0)
    assert np.all((y > 0) & (y < 1))
    y0, _ = oracle_mod.tonemap_global_plane(L, ldr=False, k=0.0)
    np.testing.assert_allclose(y0, 0.5, atol=0)


def test_sigmoid_scale_invariant_without_delta(oracle_mod):
    from paper_2108_13656_gb300 import synth
    img = synth.s_hdr(40, 30, seed=4).astype(np.float64)
    L = oracle_mod.decolorize(img.astype(np.float32))
    y1, _ = oracle_mod.tonemap_global_plane(L, ldr=False, delta=0.0)
    y2, _ = oracle_mod.tonemap_global_plane(L * 37.0, ldr=False, delta=0.0)
    np.testing.assert_allclose(y1, y2, rtol=0, atol=1e-13)


# ------------------------------------------------------------------ HISTEQ ----
def test_histeq_ldr_textbook_small(oracle_mod):
    img = _gray_u8([[0, 0, 128, 255]])
    y, st = oracle_mod.tonemap_global(img, mode=oracle_mod.MODE_HISTEQ)
    np.testing.assert_allclose(y, [[0.5, 0.5, 0.75, 1.0]], atol=1e-15)
    assert st["hist"][0] == 2 and st["hist"][128] == 1 and st["hist"][255] == 1
    assert int(st["hist"].sum()) == 4


def test_histeq_ldr_is_rank_cdf(oracle_mod):
    rng = np.random.default_rng(21)
    codes = rng.integers(0, 256, (37, 29))
    y, st = oracle_mod.tonemap_global(_gray_u8(codes), mode=oracle_mod.MODE_HISTEQ)
    flat = np.sort(codes.ravel())
    want = np.searchsorted(flat, codes, side="right") / codes.size
    np.testing.assert_allclose(y, want, atol=1e-15)
    np.testing.assert_array_equal(st["hist"], np.bincount(codes.ravel(), minlength=256))


def test_histeq_hdr_two_levels_and_uniform(oracle_mod):
    delta = 1e-4
    img = _gray_f32([[0.01, 5.0, 0.01, 5.0]])
    y, st = oracle_mod.tonemap_global(img, mode=oracle_mod.MODE_HISTEQ, delta=delta)
    np.testing.assert_allclose(y, [[0.0, 1.0, 0.0, 1.0]], atol=1e-15)
    assert st["hist"][0] == 2 and st["hist"][255] == 2
    # u evenly spread with four samples per bin: the piecewise-linear CDF is the identity
    n = 256 * 4
    t = (np.arange(n) + 0.5) / n
    lo, hi = math.log(0.5 + delta), math.log(4000 + delta)
    vals = np.exp(lo + (hi - lo) * t) - delta
    vals[0], vals[-1] = 0.5, 4000.0
    L = vals.reshape(1, -1)
    y, st = oracle_mod.tonemap_global_plane(L, ldr=False, mode=oracle_mod.MODE_HISTEQ, delta=delta)
    u = (np.log(L + delta) - lo) / (hi - lo)
    inner = slice(1, n - 1)
    np.testing.assert_allclose(y[0, inner], u[0, inner], atol=1e-12)


# ------------------------------------------------------------------- local ----
def _tent_f(c, bins):
    x = bins * c - 0.5
    return x - math.floor(x)


def test_local_constant_image_closed_form(oracle_mod):
    # Every block window holds one value c, split by the tent between bins j, j+1
    # with fraction f; the uniform-mass CDF gives (1-f) min(f+1/2, 1) + f max(f-1/2, 0).
    bins = 32
    for code in [3, 40, 77, 128, 200, 251]:
        img = _gray_u8(np.full((70, 90), code))
        y = oracle_mod.tonemap_local(img, block_s=16, radius_blocks=1, bins=bins)
        c = code / 255.0
        x = bins * c - 0.5
        if x <= 0:            # all mass in bin 0: F = bins * c
            want = bins * c
        elif x >= bins - 1:   # all mass in the top bin: F = bins * c - (bins - 1)
            want = bins * c - (bins - 1)
        else:
            f = _tent_f(c, bins)
            want = (1 - f) * min(f + 0.5, 1.0) + f * max(f - 0.5, 0.0)
            assert 7 / 16 - 1e-15 <= want <= 9 / 16 + 1e-15
        np.testing.assert_allclose(y, want, atol=1e-14)


def test_local_alpha_zero_is_identity(oracle_mod):
    from paper_2108_13656_gb300 import synth
    img = synth.s_ldr(50, 40, seed=5)
    L = oracle_mod.decolorize(img)
    y = oracle_mod.tonemap_local(img, block_s=8, radius_blocks=1, bins=16, alpha=0.0)
    np.testing.assert_allclose(y, L, atol=1e-15)


def _brute_local(u, s, R, bins, alpha):
    """Definition evaluated directly: window pixels summed one by one, per block."""
    H, W = len(u), len(u[0])
    Hb, Wb = -(-H // s), -(-W // s)

    def tent(v):
        x = bins * v - 0.5
        if x <= 0:
            return {0: 1.0}
        if x >= bins - 1:
            return {bins - 1: 1.0}
        j = math.floor(x)
        return {j: 1.0 - (x - j), j + 1: x - j}

    def curve(I, J, v):
        num = 0.0
        den = 0.0
        for py in range(H):
            for px in range(W):
                if abs(py // s - I) <= R and abs(px // s - J) <= R:
                    for j, w in tent(u[py][px]).items():
                        # mass w spread uniformly over [j/bins, (j+1)/bins)
                        num += w * min(max(bins * v - j, 0.0), 1.0)
                        den += w
        return num / den

    out = [[0.0] * W for _ in range(H)]
    for py in range(H):
        fy = (py + 0.5) / s - 0.5
        I0 = math.floor(fy)
        wy = fy - I0
        for px in range(W):
            fx = (px + 0.5) / s - 0.5
            J0 = math.floor(fx)
            wx = fx - J0
            acc = 0.0
            for dI, wI in ((0, 1 - wy), (1, wy)):
                for dJ, wJ in ((0, 1 - wx), (1, wx)):
                    I = min(max(I0 + dI, 0), Hb - 1)
                    J = min(max(J0 + dJ, 0), Wb - 1)
                    acc += wI * wJ * curve(I, J, u[py][px])
            out[py][px] = alpha * acc + (1 - alpha) * u[py][px]
    return np.array(out)


@pytest.mark.parametrize("H,W,s,R,bins", [(4, 4, 2, 0, 4), (4, 4, 2, 1, 4), (5, 7, 2, 1, 3), (6, 5, 3, 0, 5)])
def test_local_brute_force_tiny(oracle_mod, H, W, s, R, bins):
    rng = np.random.default_rng(100 + H * W + R)
    img = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    L = oracle_mod.decolorize(img)
    y = oracle_mod.tonemap_local(img, block_s=s, radius_blocks=R, bins=bins, alpha=0.9)
    want = _brute_local(L.tolist(), s, R, bins, 0.9)
    np.testing.assert_allclose(y, want, atol=1e-13)


def test_local_brute_force_tiny_hdr(oracle_mod):
    from paper_2108_13656_gb300 import synth
    img = synth.s_hdr(6, 5, seed=8)
    delta = 1e-4
    L = oracle_mod.decolorize(img)
    lg = np.log(L + delta)
    u = (lg - lg.min()) / (lg.max() - lg.min())
    y = oracle_mod.tonemap_local(img, block_s=2, radius_blocks=1, bins=4, delta=delta)
    np.testing.assert_allclose(y, _brute_local(u.tolist(), 2, 1, 4, 1.0), atol=1e-13)


def test_local_single_block_is_global_soft_equalisation(oracle_mod):
    # One block whose window is the whole image: the four interpolation corners are
    # the same block, so y = F(u) of the soft histogram of the whole image.
    rng = np.random.default_rng(31)
    img = rng.integers(0, 256, (9, 11, 3), dtype=np.uint8)
    L = oracle_mod.decolorize(img)
    bins = 8
    y = oracle_mod.tonemap_local(img, block_s=16, radius_blocks=0, bins=bins)
    # soft histogram via numpy's linear interpolation weights onto bin centres
    x = np.clip(bins * L.ravel() - 0.5, 0, bins - 1)
    j = np.minimum(np.floor(x).astype(int), bins - 2)
    f = x - j
    h = np.bincount(j, weights=1 - f, minlength=bins) + np.bincount(j + 1, weights=f, minlength=bins)
    edge = np.concatenate([[0.0], np.cumsum(h) / h.sum()])
    want = np.interp(bins * L, np.arange(bins + 1), edge)
    np.testing.assert_allclose(y, want, atol=1e-13)


def test_local_mirror_symmetry(oracle_mod):
    from paper_2108_13656_gb300 import synth
    img = synth.s_ldr(64, 48, seed=9)
    y = oracle_mod.tonemap_local(img, block_s=16, radius_blocks=1, bins=16)
    y_lr = oracle_mod.tonemap_local(img[:, ::-1].copy(), block_s=16, radius_blocks=1, bins=16)
    y_ud = oracle_mod.tonemap_local(img[::-1].copy(), block_s=16, radius_blocks=1, bins=16)
    np.testing.assert_allclose(y_lr, y[:, ::-1], atol=1e-13)
    np.testing.assert_allclose(y_ud, y[::-1], atol=1e-13)
    assert y.min() >= 0.0 and y.max() <= 1.0


# ------------------------------------------------------------ helper masks ----
def test_u8_boundary_mask(oracle_mod):
    y = np.array([0.5 / 255, 0.5 / 255 + 2e-5, 10.5 / 255 - 5e-6, 0.31])
    np.testing.assert_array_equal(oracle_mod.u8_boundary_mask(y), [True, False, True, False])
    np.testing.assert_array_equal(oracle_mod.gray_code(np.array([0.5 / 255 + 1e-9, 1.0, 0.0])), [1, 255, 0])
