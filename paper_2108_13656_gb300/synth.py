"""Seeded synthetic inputs shaped like the paper's workloads.

The paper evaluates on photographs (Cadik's set, color250, HDR scenes; Sec. II-C,
Sec. II-D, Sec. III-B) that are not available here.  These generators stand in
for them.  They hold none of the method's arithmetic: they only draw pixels.
Both the CUDA path and the CPU oracle read the arrays produced here, and nothing
here imports either of them.

Recipes
-------
Ragged batch (n, seed)
    Sizes drawn uniformly from RAGGED_SIZE_CHOICES (seeded); one S-LDR base image
    per distinct size (seed 1000 + the size's index); image i is its base
    cyclically shifted by a seeded (dy, dx), so that every image of the batch is a
    distinct buffer with distinct content at the same statistics.

S-LDR(W, H, seed)
    A smooth linear gradient per channel (random endpoints and direction),
    overlaid with 64 axis-aligned patches of uniform colour.  Patch colour is
    drawn in HSV with hue ~ U[0,1), saturation ~ U[0.2,1], value ~ U[0.1,1];
    patch sides are U[W/32, W/4] x U[H/32, H/4].  Values are quantised to
    8-bit sRGB codes (round(255 v)), interleaved RGB, shape (H, W, 3).

S-HDR(W, H, seed, decades, sigma)
    Linear HDR radiance.  ln Y is a standardised mix of a smooth field, a
    patch field (the same layout rule as S-LDR) and i.i.d. noise, scaled to
    N(0, sigma^2) and clipped to +-decades*ln(10)/2 so that Y spans exactly
    the stated number of decades.  Chromaticity (r, g, b >= 0, r+g+b = 1) is a
    smooth field in the background and Dirichlet(1,1,1) per patch; the pixel
    is 3*Y*(r, g, b).  float32, shape (H, W, 3).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "rng_for",
    "s_ldr",
    "s_hdr",
    "ragged_sizes",
    "ragged_batch_spec",
    "ragged_base",
    "shifted",
    "RAGGED_SIZE_CHOICES",
]

RAGGED_SIZE_CHOICES = ((320, 240), (640, 480), (1280, 720), (1920, 1080), (4096, 3072))


def rng_for(seed: int) -> np.random.Generator:
    """PCG64 generator for a seed (numpy's published bit generator)."""
    return np.random.Generator(np.random.PCG64(seed))


def _hsv_to_rgb(h: float, s: float, v: float) -> tuple[float, float, float]:
    """Standard hexcone HSV -> RGB (Smith 1978), used only to draw patch colours."""
    i = int(h * 6.0) % 6
    f = h * 6.0 - math.floor(h * 6.0)
    p = v * (1.0 - s)
    q = v * (1.0 - f * s)
    t = v * (1.0 - (1.0 - f) * s)
    return [(v, t, p), (q, v, p), (p, v, t), (p, q, v), (t, p, v), (v, p, q)][i]


def _patches(rng: np.random.Generator, width: int, height: int, n: int):
    """n axis-aligned rectangles (x0, y0, w, h) with sides U[W/32, W/4] x U[H/32, H/4]."""
    out = []
    for _ in range(n):
        w = int(round(rng.uniform(width / 32.0, width / 4.0)))
        h = int(round(rng.uniform(height / 32.0, height / 4.0)))
        w = max(1, min(w, width))
        h = max(1, min(h, height))
        x0 = int(rng.integers(0, width - w + 1))
        y0 = int(rng.integers(0, height - h + 1))
        out.append((x0, y0, w, h))
    return out


def s_ldr(width: int, height: int, seed: int, n_patches: int = 64) -> np.ndarray:
    """S-LDR: 8-bit interleaved RGB (H, W, 3) uint8; see the module docstring."""
    rng = rng_for(seed)
    lo = rng.uniform(0.0, 1.0, 3).astype(np.float32)
    hi = rng.uniform(0.0, 1.0, 3).astype(np.float32)
    theta = rng.uniform(0.0, 2.0 * math.pi)
    xs = ((np.arange(width, dtype=np.float32) + 0.5) / width) * np.float32(math.cos(theta))
    ys = ((np.arange(height, dtype=np.float32) + 0.5) / height) * np.float32(math.sin(theta))
    t = ys[:, None] + xs[None, :]
    t -= t.min()
    tmax = t.max()
    if tmax > 0:
        t /= tmax
    img = np.empty((height, width, 3), dtype=np.float32)
    for c in range(3):
        img[:, :, c] = lo[c] + (hi[c] - lo[c]) * t
    for (x0, y0, w, h) in _patches(rng, width, height, n_patches):
        hue = rng.uniform(0.0, 1.0)
        sat = rng.uniform(0.2, 1.0)
        val = rng.uniform(0.1, 1.0)
        img[y0:y0 + h, x0:x0 + w, :] = np.asarray(_hsv_to_rgb(hue, sat, val), dtype=np.float32)
    np.clip(img, 0.0, 1.0, out=img)
    img *= 255.0
    return np.rint(img).astype(np.uint8)


def _smooth_field(rng: np.random.Generator, width: int, height: int, terms: int = 6) -> np.ndarray:
    """Sum of a few random low-frequency plane waves, built from separable factors."""
    xs = (np.arange(width, dtype=np.float64) + 0.5) / width
    ys = (np.arange(height, dtype=np.float64) + 0.5) / height
    f = np.zeros((height, width), dtype=np.float32)
    for _ in range(terms):
        fx, fy = rng.uniform(-3.0, 3.0, 2)
        ph = rng.uniform(0.0, 2.0 * math.pi)
        a = 2.0 * math.pi * fx * xs + ph
        b = 2.0 * math.pi * fy * ys
        # cos(a + b) = cos a cos b - sin a sin b
        f += (np.cos(b)[:, None] * np.cos(a)[None, :]).astype(np.float32)
        f -= (np.sin(b)[:, None] * np.sin(a)[None, :]).astype(np.float32)
    return f


def _standardise(z: np.ndarray) -> np.ndarray:
    m = float(z.mean(dtype=np.float64))
    s = float(z.std(dtype=np.float64))
    z -= np.float32(m)
    if s > 0:
        z *= np.float32(1.0 / s)
    return z


def s_hdr(width: int, height: int, seed: int, decades: float = 5.0, sigma: float = 2.5,
          n_patches: int = 64) -> np.ndarray:
    """S-HDR: linear radiance, interleaved RGB (H, W, 3) float32; see the module docstring."""
    rng = rng_for(seed)
    smooth = _standardise(_smooth_field(rng, width, height))
    patch = np.zeros((height, width), dtype=np.float32)
    rects = _patches(rng, width, height, n_patches)
    chroma_p = []
    for (x0, y0, w, h) in rects:
        patch[y0:y0 + h, x0:x0 + w] = np.float32(rng.standard_normal() * 1.5)
        chroma_p.append(rng.dirichlet((1.0, 1.0, 1.0)).astype(np.float32))
    noise = rng.standard_normal((height, width), dtype=np.float32)
    z = smooth * np.float32(0.6) + patch * np.float32(0.6) + noise * np.float32(0.5)
    z = _standardise(z)
    half = decades * math.log(10.0) / 2.0
    z *= np.float32(sigma)
    np.clip(z, -half, half, out=z)
    y3 = np.exp(z) * np.float32(3.0)
    img = np.empty((height, width, 3), dtype=np.float32)
    csum = np.zeros((height, width), dtype=np.float32)
    for c in range(3):
        img[:, :, c] = np.float32(1.0) + np.float32(0.8) * np.tanh(_smooth_field(rng, width, height, terms=2))
        csum += img[:, :, c]
    for c in range(3):
        img[:, :, c] /= csum
    for (x0, y0, w, h), ch in zip(rects, chroma_p):
        img[y0:y0 + h, x0:x0 + w, :] = ch
    img *= y3[:, :, None]
    return img


def ragged_sizes(n: int, seed: int, choices=RAGGED_SIZE_CHOICES) -> list[tuple[int, int]]:
    """n (width, height) pairs drawn uniformly from `choices` with a seeded generator."""
    rng = rng_for(seed)
    idx = rng.integers(0, len(choices), n)
    return [tuple(choices[int(i)]) for i in idx]


def ragged_batch_spec(n: int, seed: int, choices=RAGGED_SIZE_CHOICES):
    """(sizes, shifts): n (width, height) pairs as ragged_sizes and a seeded cyclic
    shift (dy, dx) per image; the base image of size index k is s_ldr(W, H, 1000 + k)."""
    sizes = ragged_sizes(n, seed, choices)
    rng = rng_for(seed + 1)
    shifts = [(int(rng.integers(0, h)), int(rng.integers(0, w))) for (w, h) in sizes]
    return sizes, shifts


def ragged_base(size, choices=RAGGED_SIZE_CHOICES) -> np.ndarray:
    """The S-LDR base image of one size of the ragged batch."""
    k = [tuple(c) for c in choices].index(tuple(size))
    return s_ldr(size[0], size[1], 1000 + k)


def shifted(img: np.ndarray, dy: int, dx: int) -> np.ndarray:
    """Cyclic shift of an (H, W, C) image by dy rows and dx columns (np.roll)."""
    return np.roll(img, (dy, dx), axis=(0, 1))
