"""FP64 CPU oracle for the decolorization hot path (test infrastructure).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the product package never
does.  The arithmetic lives in ``decolor_oracle.c`` (plain IEEE double, built with
``-O2 -ffp-contract=off``, no fast-math); this module only marshals numpy arrays.
It shares no code with the CUDA library.

Functions follow the paper: Eq. 1-6 (Sec. II-B) for the luminance, the centred
sigmoid global curve (Sec. III-B-1) and smoothed local-histogram equalisation
(Sec. III-B-2).  The readings of what the paper leaves open are listed in the
header of ``decolor_oracle.c``.  Parity of the tone-mapping parameters is
unpinned by the paper (it prints none); the closed forms and invariants that pin
the operators live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "decolor_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

DT_U8, DT_F16, DT_F32 = 0, 1, 2
LUMA_OURS, LUMA_Y, LUMA_V, LUMA_LSTAR = 0, 1, 2, 3  # Eq. 1-6; rgb2gray Y of Sec. I; V of HSV (Fig. GTMO); CIE L*/100
BETA_R, BETA_K = 0.55, 0.8  # Sec. II-B: "(beta_R = 0.55; beta_k = 0.8)"
MODE_SIGMOID, MODE_HISTEQ = 0, 1

_dp = ctypes.POINTER(ctypes.c_double)
_up = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE double; no contraction, no fast-math)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + ".tmp%d" % os.getpid()
            subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                                   "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.oracle_luminance.restype = ctypes.c_double
        lib.oracle_luminance.argtypes = [ctypes.c_double] * 5
        lib.oracle_decolorize.restype = ctypes.c_int
        lib.oracle_decolorize.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                          ctypes.c_double, _dp]
        lib.oracle_log_stats.restype = None
        lib.oracle_log_stats.argtypes = [_dp, ctypes.c_int64, ctypes.c_double, _dp, _dp, _dp]
        lib.oracle_gray_hist.restype = None
        lib.oracle_gray_hist.argtypes = [_dp, ctypes.c_int64, _up]
        lib.oracle_log_hist.restype = None
        lib.oracle_log_hist.argtypes = [_dp, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, _up]
        lib.oracle_tone_sigmoid.restype = None
        lib.oracle_tone_sigmoid.argtypes = [_dp, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, _dp]
        lib.oracle_tone_histeq_ldr.restype = None
        lib.oracle_tone_histeq_ldr.argtypes = [_dp, ctypes.c_int64, _up, _dp]
        lib.oracle_tone_histeq_hdr.restype = None
        lib.oracle_tone_histeq_hdr.argtypes = [_dp, ctypes.c_int64, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, _up, _dp]
        lib.oracle_luma.restype = ctypes.c_double
        lib.oracle_luma.argtypes = [ctypes.c_double] * 3 + [ctypes.c_int32, ctypes.c_double, ctypes.c_double]
        lib.oracle_decolorize_luma.restype = ctypes.c_int
        lib.oracle_decolorize_luma.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                               ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double, _dp]
        lib.oracle_color_reconstruct.restype = ctypes.c_int
        lib.oracle_color_reconstruct.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                                 ctypes.c_int32, _dp, _dp, ctypes.c_double, _dp]
        lib.oracle_video_mu_update.restype = ctypes.c_double
        lib.oracle_video_mu_update.argtypes = [ctypes.c_double] * 3
        lib.oracle_local_tables.restype = ctypes.c_int
        lib.oracle_local_tables.argtypes = [_dp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int32, _dp]
        lib.oracle_local_apply.restype = ctypes.c_int
        lib.oracle_local_apply.argtypes = [_dp, _dp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_double, _dp]
        lib.oracle_local_coord.restype = None
        lib.oracle_local_coord.argtypes = [_dp, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, _dp]
        lib.oracle_tone_local.restype = ctypes.c_int
        lib.oracle_tone_local.argtypes = [_dp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, _dp]
        _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _uptr(a: np.ndarray):
    return a.ctypes.data_as(_up)


def dtype_code(a: np.ndarray) -> int:
    if a.dtype == np.uint8:
        return DT_U8
    if a.dtype == np.float16:
        return DT_F16
    if a.dtype == np.float32:
        return DT_F32
    raise TypeError("unsupported sample type %s" % a.dtype)


# ---------------------------------------------------------------- Eq. 1-6 ----
def luminance(R: float, G: float, B: float, beta_R: float = BETA_R, beta_k: float = BETA_K) -> float:
    """Eq. 1-6 for one pixel with channel values in linear units (8-bit codes / 255)."""
    return _load().oracle_luminance(float(R), float(G), float(B), float(beta_R), float(beta_k))


def luma(R: float, G: float, B: float, channel: int, beta_R: float = BETA_R, beta_k: float = BETA_K) -> float:
    """One pixel's luminance in the chosen channel (LUMA_OURS, LUMA_Y or LUMA_V)."""
    return _load().oracle_luma(float(R), float(G), float(B), int(channel), float(beta_R), float(beta_k))


def _interleaved(img: np.ndarray) -> np.ndarray:
    if img.ndim != 3 or img.shape[2] != 3:
        raise ValueError("expected (H, W, 3)")
    esz = img.dtype.itemsize
    if img.shape[0] > 0 and img.shape[1] > 0 and (img.strides[2] != esz or img.strides[1] != 3 * esz):
        img = np.ascontiguousarray(img)
    return img


def decolorize(img: np.ndarray, beta_R: float = BETA_R, beta_k: float = BETA_K, channel: int = LUMA_OURS) -> np.ndarray:
    """Eq. 1-6 (or the comparison channel `channel`) over an interleaved (H, W, 3) image
    (any row stride); returns float64 (H, W)."""
    img = _interleaved(img)
    H, W = img.shape[:2]
    out = np.empty((H, W), dtype=np.float64)
    if H == 0 or W == 0:
        return out
    if channel == LUMA_OURS:
        rc = _load().oracle_decolorize(ctypes.c_void_p(img.ctypes.data), W, H, img.strides[0],
                                       dtype_code(img), beta_R, beta_k, _dptr(out))
    else:
        rc = _load().oracle_decolorize_luma(ctypes.c_void_p(img.ctypes.data), W, H, img.strides[0],
                                            dtype_code(img), int(channel), beta_R, beta_k, _dptr(out))
    if rc != 0:
        raise ValueError("oracle decolorize failed (%d)" % rc)
    return out


def color_reconstruct(img: np.ndarray, L: np.ndarray, y: np.ndarray, s: float = 1.0) -> np.ndarray:
    """C_out = min(1, y (C_in / L)^s) per channel (black pixel: y); float64 (H, W, 3)."""
    img = _interleaved(img)
    H, W = img.shape[:2]
    L = np.ascontiguousarray(L, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    if L.shape != (H, W) or y.shape != (H, W):
        raise ValueError("L and y must be (H, W)")
    out = np.empty((H, W, 3), dtype=np.float64)
    if H == 0 or W == 0:
        return out
    rc = _load().oracle_color_reconstruct(ctypes.c_void_p(img.ctypes.data), W, H, img.strides[0], dtype_code(img),
                                          _dptr(L), _dptr(y), float(s), _dptr(out))
    if rc != 0:
        raise ValueError("oracle_color_reconstruct failed (%d)" % rc)
    return out


def video_mu_update(m_prev: float, mu_frame: float, lam: float) -> float:
    """m_t = (1 - lambda) m_{t-1} + lambda mu_t (the frame-sequence estimate)."""
    return _load().oracle_video_mu_update(float(m_prev), float(mu_frame), float(lam))


# ------------------------------------------------------- global statistics ----
def log_stats(L: np.ndarray, delta: float = 1e-4):
    """(mu, lmin, lmax) of ln(L + delta) over the plane."""
    L = np.ascontiguousarray(L, dtype=np.float64)
    mu, lo, hi = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _load().oracle_log_stats(_dptr(L), L.size, delta, ctypes.byref(mu), ctypes.byref(lo),
                             ctypes.byref(hi))
    return mu.value, lo.value, hi.value


def gray_hist(L: np.ndarray) -> np.ndarray:
    L = np.ascontiguousarray(L, dtype=np.float64)
    h = np.zeros(256, dtype=np.uint32)
    _load().oracle_gray_hist(_dptr(L), L.size, _uptr(h))
    return h


def log_hist(L: np.ndarray, delta: float, lmin: float, lmax: float) -> np.ndarray:
    L = np.ascontiguousarray(L, dtype=np.float64)
    h = np.zeros(256, dtype=np.uint32)
    _load().oracle_log_hist(_dptr(L), L.size, delta, lmin, lmax, _uptr(h))
    return h


def gray_code(L: np.ndarray) -> np.ndarray:
    """8-bit code floor(255 L + 1/2) clamped to [0, 255] (used for u8 output too)."""
    return np.clip(np.floor(255.0 * np.asarray(L, dtype=np.float64) + 0.5), 0, 255).astype(np.uint8)


# ------------------------------------------------------------ tone curves ----
def tonemap_global_plane(L: np.ndarray, ldr: bool, mode: int = MODE_SIGMOID, k: float = 1.0,
                         delta: float = 1e-4):
    """Global tone curve of a luminance plane; returns (y, stats dict)."""
    Lc = np.ascontiguousarray(L, dtype=np.float64)
    mu, lmin, lmax = log_stats(Lc, delta)
    y = np.empty_like(Lc)
    hist = np.zeros(256, dtype=np.uint32)
    lib = _load()
    if mode == MODE_SIGMOID:
        lib.oracle_tone_sigmoid(_dptr(Lc), Lc.size, k, delta, mu, _dptr(y))
        if ldr:
            hist = gray_hist(Lc)
    elif mode == MODE_HISTEQ:
        if ldr:
            hist = gray_hist(Lc)
            lib.oracle_tone_histeq_ldr(_dptr(Lc), Lc.size, _uptr(hist), _dptr(y))
        else:
            hist = log_hist(Lc, delta, lmin, lmax)
            lib.oracle_tone_histeq_hdr(_dptr(Lc), Lc.size, delta, lmin, lmax, _uptr(hist), _dptr(y))
    else:
        raise ValueError("unknown global mode %r" % mode)
    stats = {"mu": mu, "lmin": lmin, "lmax": lmax, "hist": hist, "n": Lc.size}
    return y.reshape(np.shape(L)), stats


def tonemap_local_plane(L: np.ndarray, ldr: bool, block_s: int = 32, radius_blocks: int = 2,
                        bins: int = 32, alpha: float = 1.0, delta: float = 1e-4) -> np.ndarray:
    """Smoothed local-histogram equalisation of a luminance plane (float64 (H, W))."""
    Lc = np.ascontiguousarray(L, dtype=np.float64)
    H, W = Lc.shape
    lmin = lmax = 0.0
    if not ldr:
        _, lmin, lmax = log_stats(Lc, delta)
    y = np.empty_like(Lc)
    rc = _load().oracle_tone_local(_dptr(Lc), W, H, 1 if ldr else 0, block_s, radius_blocks, bins,
                                   alpha, delta, lmin, lmax, _dptr(y))
    if rc != 0:
        raise ValueError("oracle_tone_local failed (%d)" % rc)
    return y


def tonemap_global(img: np.ndarray, mode: int = MODE_SIGMOID, k: float = 1.0, delta: float = 1e-4,
                   beta_R: float = BETA_R, beta_k: float = BETA_K, channel: int = LUMA_OURS):
    """Decolorize then apply the global curve; LDR iff 8-bit input. Returns (y, stats)."""
    L = decolorize(img, beta_R, beta_k, channel)
    return tonemap_global_plane(L, img.dtype == np.uint8, mode, k, delta)


def tonemap_local(img: np.ndarray, block_s: int = 32, radius_blocks: int = 2, bins: int = 32,
                  alpha: float = 1.0, delta: float = 1e-4, beta_R: float = BETA_R,
                  beta_k: float = BETA_K, channel: int = LUMA_OURS) -> np.ndarray:
    """Decolorize then apply the local operator; LDR iff 8-bit input."""
    L = decolorize(img, beta_R, beta_k, channel)
    return tonemap_local_plane(L, img.dtype == np.uint8, block_s, radius_blocks, bins, alpha, delta)


def tonemap_global_color(img: np.ndarray, s: float = 1.0, channel: int = LUMA_OURS, **kw) -> np.ndarray:
    """Global tone mapping of the chosen luminance, then colour reconstruction: (H, W, 3)."""
    beta_R, beta_k = kw.pop("beta_R", BETA_R), kw.pop("beta_k", BETA_K)
    L = decolorize(img, beta_R, beta_k, channel)
    y, _ = tonemap_global_plane(L, img.dtype == np.uint8, **kw)
    return color_reconstruct(img, L, y, s)


def tonemap_local_color(img: np.ndarray, s: float = 1.0, channel: int = LUMA_OURS, **kw) -> np.ndarray:
    """Local tone mapping of the chosen luminance, then colour reconstruction: (H, W, 3)."""
    beta_R, beta_k = kw.pop("beta_R", BETA_R), kw.pop("beta_k", BETA_K)
    L = decolorize(img, beta_R, beta_k, channel)
    y = tonemap_local_plane(L, img.dtype == np.uint8, **kw)
    return color_reconstruct(img, L, y, s)


def tonemap_video_global(frames, lam: float = 1.0, k: float = 1.0, delta: float = 1e-4, beta_R: float = BETA_R,
                         beta_k: float = BETA_K, channel: int = LUMA_OURS):
    """A frame sequence through the centred sigmoid with the carried log-mean estimate:
    frame 0 around its own log-mean mu_0 (m_0 = mu_0); frame t >= 1 around m_{t-1},
    then m_t = (1 - lambda) m_{t-1} + lambda mu_t.  Returns ([y_t], [m_t])."""
    ys, ms = [], []
    m = None
    lib = _load()
    for img in frames:
        L = np.ascontiguousarray(decolorize(img, beta_R, beta_k, channel))
        mu, _, _ = log_stats(L, delta)
        centre = mu if m is None else m
        y = np.empty_like(L)
        lib.oracle_tone_sigmoid(_dptr(L), L.size, k, delta, centre, _dptr(y))
        m = mu if m is None else video_mu_update(m, mu, lam)
        ys.append(y)
        ms.append(m)
    return ys, ms


def u8_boundary_mask(y: np.ndarray, eps: float = 1e-5) -> np.ndarray:
    """True where y lies within eps of an 8-bit rounding boundary (k + 1/2)/255."""
    t = 255.0 * np.asarray(y, dtype=np.float64)
    frac = t - np.floor(t)
    return np.abs(frac - 0.5) < 255.0 * eps


def f16_boundary_mask(y: np.ndarray, eps: float = 1e-5) -> np.ndarray:
    """True where y lies within eps (relative) of a binary16 rounding midpoint."""
    y = np.asarray(y, dtype=np.float64)
    h = y.astype(np.float16).astype(np.float64)
    up = np.nextafter(y.astype(np.float16), np.float16(np.inf)).astype(np.float64)
    dn = np.nextafter(y.astype(np.float16), np.float16(-np.inf)).astype(np.float64)
    mid_up = 0.5 * (h + up)
    mid_dn = 0.5 * (h + dn)
    tol = eps * np.maximum(1.0, np.abs(y))
    return (np.abs(y - mid_up) < tol) | (np.abs(y - mid_dn) < tol)


# ------------------------------------------------------ local frame sequences ----
def local_coord(L: np.ndarray, ldr: bool, delta: float = 1e-4, lmin: float = 0.0, lmax: float = 0.0) -> np.ndarray:
    """Coordinate plane u of the local operator (L for 8-bit input, else the log
    luminance normalised by (lmin, lmax)), clamped to [0, 1]."""
    Lc = np.ascontiguousarray(L, dtype=np.float64)
    u = np.empty_like(Lc)
    _load().oracle_local_coord(_dptr(Lc), Lc.size, 1 if ldr else 0, delta, lmin, lmax, _dptr(u))
    return u


def local_tables(u: np.ndarray, block_s: int = 32, radius_blocks: int = 2, bins: int = 32) -> np.ndarray:
    """Per-block cumulative tables (Hb, Wb, bins + 1) of the local operator from a coordinate plane."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    H, W = u.shape
    Hb, Wb = -(-H // block_s), -(-W // block_s)
    e = np.empty((Hb, Wb, bins + 1), dtype=np.float64)
    rc = _load().oracle_local_tables(_dptr(u), W, H, block_s, radius_blocks, bins, _dptr(e))
    if rc != 0:
        raise ValueError("oracle_local_tables failed (%d)" % rc)
    return e


def local_apply(u: np.ndarray, edge: np.ndarray, block_s: int = 32, bins: int = 32, alpha: float = 1.0) -> np.ndarray:
    """Bilinear blend of the four nearest block tables at every pixel's own u."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    edge = np.ascontiguousarray(edge, dtype=np.float64)
    H, W = u.shape
    y = np.empty_like(u)
    rc = _load().oracle_local_apply(_dptr(u), _dptr(edge), W, H, block_s, bins, alpha, _dptr(y))
    if rc != 0:
        raise ValueError("oracle_local_apply failed (%d)" % rc)
    return y


def tonemap_video_local(frames, block_s: int = 32, radius_blocks: int = 2, bins: int = 32, alpha: float = 1.0,
                        delta: float = 1e-4, beta_R: float = BETA_R, beta_k: float = BETA_K,
                        channel: int = LUMA_OURS):
    """A frame sequence through the local operator with the previous frame's tables:
    frame 0 is the local operator on its own (its own log range for HDR input);
    frame t >= 1 takes its coordinates in the previous frame's log range (HDR), is
    mapped through the previous frame's tables, and then its own tables (from those
    coordinates) and its own log range are carried to the next frame.  Returns [y_t]."""
    ys = []
    edge = None
    rng = (0.0, 0.0)
    for img in frames:
        ldr = img.dtype == np.uint8
        L = decolorize(img, beta_R, beta_k, channel)
        own = (0.0, 0.0)
        if not ldr:
            _, lo, hi = log_stats(L, delta)
            own = (lo, hi)
        if edge is None:
            rng = own
        u = local_coord(L, ldr, delta, *rng)
        if edge is None:
            edge = local_tables(u, block_s, radius_blocks, bins)
        ys.append(local_apply(u, edge, block_s, bins, alpha))
        edge = local_tables(u, block_s, radius_blocks, bins)
        rng = own
    return ys


def video_color(frames, ys, s: float = 1.0, beta_R: float = BETA_R, beta_k: float = BETA_K,
                channel: int = LUMA_OURS):
    """Colour reconstruction of every frame of a sequence from its tone-mapped plane:
    [(H, W, 3)] = min(1, y (C/L)^s) per frame."""
    return [color_reconstruct(f, decolorize(f, beta_R, beta_k, channel), y, s) for f, y in zip(frames, ys)]


def tonemap_video_histeq(frames, delta: float = 1e-4, beta_R: float = BETA_R, beta_k: float = BETA_K,
                         channel: int = LUMA_OURS):
    """A frame sequence through global histogram equalisation with the previous frame's
    histogram: frame 0 is equalised with its own (and, HDR, in its own log range);
    frame t >= 1 is mapped through frame t-1's cumulative histogram, its HDR coordinate
    taken in frame t-1's log range (clamped), and its own histogram - binned in that
    same range - and its own range go to frame t+1.  Returns [y_t]."""
    lib = _load()
    ys = []
    hist = None
    rng = (0.0, 0.0)
    for img in frames:
        ldr = img.dtype == np.uint8
        L = np.ascontiguousarray(decolorize(img, beta_R, beta_k, channel))
        _, lo, hi = log_stats(L, delta)
        if hist is None:
            rng = (lo, hi)
            hist = gray_hist(L) if ldr else log_hist(L, delta, *rng)
        y = np.empty_like(L)
        if ldr:
            lib.oracle_tone_histeq_ldr(_dptr(L), L.size, _uptr(hist), _dptr(y))
            hist = gray_hist(L)
        else:
            lib.oracle_tone_histeq_hdr(_dptr(L), L.size, delta, rng[0], rng[1], _uptr(hist), _dptr(y))
            hist = log_hist(L, delta, *rng)
            rng = (lo, hi)
        ys.append(y)
    return ys
