"""Pins for the FP64 oracle that do not come from the oracle itself.

Eq. 1-6 and the parameter values are from Sec. II-B.  The checks below use
closed forms derived by hand (tests/golden/primaries.txt), exact invariants of the
equations (achromatic identity, 1-homogeneity, min <= L <= max over every 8-bit
triple), special cases that collapse the equations, the qualitative statements of
Sec. I (warm colours lighter than Y) and Sec. III-C (green maps dark), and the
decode of binary16 against numpy's conversion.
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_primaries():
    rows = []
    with open(os.path.join(GOLDEN, "primaries.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            lhs, rhs = line.split("|")
            rgb = [float(v) for v in lhs.split()]
            val = eval(rhs.strip(), {"sqrt": math.sqrt, "__builtins__": {}})
            rows.append((rgb, val))
    return rows


@pytest.mark.parametrize("rgb,expected", _golden_primaries())
def test_primaries_closed_form(oracle_mod, rgb, expected):
    got = oracle_mod.luminance(*rgb)
    assert got == pytest.approx(expected, rel=1e-14, abs=1e-15)


def test_paper_parameters(oracle_mod):
    # Sec. II-B fixes beta_R = 0.55 and beta_k = 0.8 and both in (0.5, 1).
    assert oracle_mod.BETA_R == 0.55 and oracle_mod.BETA_K == 0.8


@pytest.mark.parametrize("beta_R,beta_k", [(0.55, 0.8), (0.6, 0.9), (0.99, 0.51), (0.0, 1.0), (1.0, 0.0)])
def test_achromatic_identity(oracle_mod, beta_R, beta_k):
    # R = G = B = c: every intermediate of Eq. 1-5 is c, so Eq. 6 gives c.
    for c in [0.0, 1e-9, 0.1, 0.25, 1.0 / 3.0, 0.5, 0.999, 1.0, 7.5, 1e4]:
        assert oracle_mod.luminance(c, c, c, beta_R, beta_k) == pytest.approx(c, rel=1e-15, abs=0)


def test_pure_channels_any_beta(oracle_mod):
    rng = np.random.default_rng(11)
    for _ in range(200):
        bR, bk = rng.uniform(0, 1, 2)
        v = rng.uniform(0.0, 10.0)
        # pure blue: L_WARM = L_WHITE = L_COOL = v/sqrt(3) whatever the betas
        assert oracle_mod.luminance(0, 0, v, bR, bk) == pytest.approx(v / math.sqrt(3), rel=1e-14)
        # pure red: L_WARM = sqrt(beta_R) v, L_COOL = 0
        assert oracle_mod.luminance(v, 0, 0, bR, bk) == pytest.approx(v * math.sqrt(bR * bk), rel=1e-14, abs=1e-300)
        # pure green: r = 0 so L_WARM = L_WHITE, L_COOL = 0
        assert oracle_mod.luminance(0, v, 0, bR, bk) == pytest.approx(v * math.sqrt(bk / 3), rel=1e-14, abs=1e-300)


def test_special_case_betas(oracle_mod):
    rng = np.random.default_rng(12)
    for _ in range(500):
        R, G, B = rng.uniform(0, 1, 3)
        S = R + G + B
        Q = R * R + G * G + B * B
        # beta_R = beta_k = 1: L_GR = R and L = L_WARM = R^2/S + (G+B)/S sqrt(Q/3)
        want = (R * R + (G + B) * math.sqrt(Q / 3)) / S
        assert oracle_mod.luminance(R, G, B, 1.0, 1.0) == pytest.approx(want, rel=1e-13)
        # beta_k = 0: L = L_COOL = B (R+G)/S + B/S sqrt(Q/3) = B (R + G + sqrt(Q/3)) / S
        want = B * (R + G + math.sqrt(Q / 3)) / S
        assert oracle_mod.luminance(R, G, B, 0.3, 0.0) == pytest.approx(want, rel=1e-13)


def test_homogeneity(oracle_mod):
    rng = np.random.default_rng(13)
    for _ in range(500):
        R, G, B = rng.uniform(0, 1, 3)
        s = float(np.exp(rng.uniform(-20, 20)))
        base = oracle_mod.luminance(R, G, B)
        assert oracle_mod.luminance(s * R, s * G, s * B) == pytest.approx(s * base, rel=1e-14)


def test_black_pixel_is_continuous(oracle_mod):
    assert oracle_mod.luminance(0, 0, 0) == 0.0
    for e in [1e-3, 1e-9, 1e-150]:  # squares must stay normal doubles
        assert 0.0 < oracle_mod.luminance(e, 0.5 * e, 0.25 * e) <= e


def test_bounds_every_8bit_triple(oracle_mod):
    # min(R,G,B) <= L <= max(R,G,B) for every one of the 2^24 8-bit triples.
    v = np.arange(1 << 24, dtype=np.uint32)
    img = np.empty((4096, 4096, 3), dtype=np.uint8)
    img[..., 0] = (v >> 16).reshape(4096, 4096)
    img[..., 1] = ((v >> 8) & 255).reshape(4096, 4096)
    img[..., 2] = (v & 255).reshape(4096, 4096)
    L = oracle_mod.decolorize(img)
    lo = img.min(axis=2) / 255.0
    hi = img.max(axis=2) / 255.0
    assert np.all(L >= lo * (1 - 1e-15))
    assert np.all(L <= hi * (1 + 1e-15))
    assert L.min() == 0.0 and L.max() == 1.0


def test_not_monotone_per_channel(oracle_mod):
    # Sec. I assumption (ii): mixed colours are darker.  Adding a little blue to pure
    # red lowers L, so tests must never assert per-channel monotonicity.
    assert oracle_mod.luminance(1, 0, 0.1) < oracle_mod.luminance(1, 0, 0)


def test_green_maps_dark(oracle_mod):
    # Sec. III-C: pure green maps to a dark value, below pure blue and pure red.
    g = oracle_mod.luminance(0, 1, 0)
    b = oracle_mod.luminance(0, 0, 1)
    r = oracle_mod.luminance(1, 0, 0)
    assert g < b < r


def test_warm_lighter_than_ycbcr_y(oracle_mod):
    # Sec. I assumption (i): warm colours (mainly R) are lighter than Y.
    def y601(R, G, B):
        return 0.2989 * R + 0.5870 * G + 0.1140 * B
    for rgb in [(1, 0, 0), (1, 0.25, 0), (1, 0.5, 0), (0.8, 0.2, 0.1), (0.9, 0.4, 0.0)]:
        assert oracle_mod.luminance(*rgb) > y601(*rgb)


def test_decode_u8_scale(oracle_mod):
    rng = np.random.default_rng(14)
    img = rng.integers(0, 256, (5, 7, 3), dtype=np.uint8)
    L = oracle_mod.decolorize(img)
    for y in range(5):
        for x in range(7):
            R, G, B = (img[y, x] / 255.0).tolist()
            assert L[y, x] == oracle_mod.luminance(R, G, B)


def test_decode_binary16_every_pattern(oracle_mod):
    # Achromatic pixels return their own value, so the plane reproduces the oracle's
    # binary16 decode, which must equal numpy's conversion for every non-negative
    # finite pattern.
    pats = np.arange(0, 0x7C00, dtype=np.uint16)
    vals = pats.view(np.float16)
    img = np.repeat(vals[:, None], 3, axis=1).reshape(1, -1, 3)
    L = oracle_mod.decolorize(img)
    np.testing.assert_allclose(L[0], vals.astype(np.float64), rtol=4e-16, atol=0)


def test_negative_samples_read_as_black(oracle_mod):
    img = np.array([[[-1.0, 0.5, 0.25], [0.0, 0.5, 0.25]]], dtype=np.float32)
    L = oracle_mod.decolorize(img)
    assert L[0, 0] == L[0, 1]


def test_strided_rows(oracle_mod):
    rng = np.random.default_rng(15)
    big = rng.integers(0, 256, (9, 13, 3), dtype=np.uint8)
    view = big[:, 2:11, :]
    assert view.strides[0] == 39
    np.testing.assert_array_equal(oracle_mod.decolorize(view), oracle_mod.decolorize(view.copy()))
