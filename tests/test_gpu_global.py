"""GPU parity of decolorization + the global tone curve (Sec. III-B-1) against the oracle."""
import math

import numpy as np
import pytest

from _cmp import TOL_F32, check_f16, check_f32, check_out, check_u8
from _dev import GuardedOut, to_dev

pytestmark = pytest.mark.gpu
MU_TOL = 4e-6


@pytest.fixture(scope="module")
def dc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2108_13656_gb300 as m
    m.load()
    return m


def hist_bounds(values_scaled, window):
    """Per-bin [lower, upper] counts for bins floor(values_scaled) in [0, 255] when
    values within `window` of an integer may fall on either side."""
    v = np.asarray(values_scaled, dtype=np.float64).ravel()
    fl = np.floor(v)
    k = np.clip(fl, 0, 255).astype(np.int64)
    frac = v - fl
    amb = ((frac < window) & (fl >= 1) & (fl <= 255)) | ((frac > 1 - window) & (fl >= 0) & (fl <= 254))
    sure = np.bincount(k[~amb], minlength=256)
    lo = np.where(frac[amb] < window, k[amb] - 1, k[amb])
    hi = np.where(frac[amb] < window, k[amb], k[amb] + 1)
    upper = sure + np.bincount(np.clip(lo, 0, 255), minlength=256) + np.bincount(np.clip(hi, 0, 255), minlength=256)
    return sure, upper, amb.reshape(np.shape(values_scaled))


def run_global(dc, img, out_dt, mode="sigmoid", gain_k=1.0, delta=1e-4, pad=0, off=0):
    import torch
    H, W = img.shape[:2]
    x = to_dev(img, pad_px=pad, offset_elems=off)
    o = GuardedOut(H, W, out_dt, pad_px=pad, offset_elems=off)
    st = torch.zeros(dc.STATS_BYTES, dtype=torch.uint8, device="cuda")
    dc.decolorize_tonemap_global(x, o.view, mode=mode, gain_k=gain_k, delta=delta, stats=st)
    torch.cuda.synchronize()
    o.check()
    assert dc.query_status() == 0
    return o.numpy(), dc.parse_stats(st, 1)[0]


def check_stats_common(st, ref, N):
    assert st["npix"] == N
    assert abs(st["mu"] - ref["mu"]) <= MU_TOL, (st["mu"], ref["mu"])
    assert abs(st["lmin"] - ref["lmin"]) <= 2e-6 * max(1, abs(ref["lmin"]))
    assert abs(st["lmax"] - ref["lmax"]) <= 2e-6 * max(1, abs(ref["lmax"]))
    # exact fixed-point log-sum: |sum/2^24 - N mu64| within the per-group rounding and binary32 log error
    assert abs(st["logsum_fixed"] / 2.0 ** 24 - N * ref["mu"]) <= N * MU_TOL


@pytest.mark.parametrize("out_dt", ["u8", "f16", "f32"])
def test_sigmoid_ldr(dc, oracle_mod, out_dt):
    from paper_2108_13656_gb300 import synth
    img = synth.s_ldr(512, 384, seed=7)
    L64 = oracle_mod.decolorize(img)
    y64, ref = oracle_mod.tonemap_global_plane(L64, ldr=True)
    y, st = run_global(dc, img, out_dt)
    check_out(y, y64, out_dt, "sigmoid ldr " + out_dt)
    check_stats_common(st, ref, img.shape[0] * img.shape[1])
    lo, hi, _ = hist_bounds(255.0 * L64 + 0.5, 255 * 1e-5)
    assert np.all(st["hist"] >= lo) and np.all(st["hist"] <= hi)
    assert int(st["hist"].sum()) == L64.size


@pytest.mark.parametrize("in_dt", [np.float16, np.float32])
@pytest.mark.parametrize("out_dt", ["u8", "f16", "f32"])
def test_sigmoid_hdr(dc, oracle_mod, in_dt, out_dt):
    from paper_2108_13656_gb300 import synth
    img = synth.s_hdr(400, 300, seed=8, decades=5.0, sigma=2.5).astype(in_dt)
    L64 = oracle_mod.decolorize(img)
    y64, ref = oracle_mod.tonemap_global_plane(L64, ldr=False)
    y, st = run_global(dc, img, out_dt)
    check_out(y, y64, out_dt, "sigmoid hdr " + out_dt)
    check_stats_common(st, ref, img.shape[0] * img.shape[1])
    assert int(st["hist"].sum()) == 0  # HDR sigmoid does not build the u histogram


@pytest.mark.parametrize("gain_k", [0.0, 0.5, 2.5])
def test_sigmoid_gain(dc, oracle_mod, gain_k):
    from paper_2108_13656_gb300 import synth
    img = synth.s_hdr(200, 150, seed=9)
    L64 = oracle_mod.decolorize(img)
    y64, _ = oracle_mod.tonemap_global_plane(L64, ldr=False, k=gain_k)
    y, _ = run_global(dc, img, "f32", gain_k=gain_k)
    check_f32(y, y64, what="gain %g" % gain_k)


@pytest.mark.parametrize("out_dt", ["u8", "f32"])
def test_histeq_ldr(dc, oracle_mod, out_dt):
    from paper_2108_13656_gb300 import synth
    img = synth.s_ldr(333, 250, seed=10)
    L64 = oracle_mod.decolorize(img)
    y64, ref = oracle_mod.tonemap_global_plane(L64, ldr=True, mode=oracle_mod.MODE_HISTEQ)
    y, st = run_global(dc, img, out_dt, mode="histeq")
    lo, hi, amb = hist_bounds(255.0 * L64 + 0.5, 255 * 1e-5)
    assert np.all(st["hist"] >= lo) and np.all(st["hist"] <= hi)
    n_amb = int(amb.sum())
    slack = n_amb / L64.size
    if out_dt == "f32":
        err = np.abs(y.astype(np.float64) - y64)
        assert np.all(err[~amb] <= TOL_F32 + slack), float(err[~amb].max())
    else:
        near = oracle_mod.u8_boundary_mask(y64, 1e-5 + slack)
        check_u8(y, y64, "histeq ldr u8", extra_exempt=amb | near)


@pytest.mark.parametrize("in_dt", [np.float16, np.float32])
@pytest.mark.parametrize("out_dt", ["f16", "f32"])
def test_histeq_hdr(dc, oracle_mod, in_dt, out_dt):
    from paper_2108_13656_gb300 import synth
    img = synth.s_hdr(301, 203, seed=11, decades=6.0, sigma=2.76).astype(in_dt)
    delta = 1e-4
    L64 = oracle_mod.decolorize(img)
    y64, ref = oracle_mod.tonemap_global_plane(L64, ldr=False, mode=oracle_mod.MODE_HISTEQ, delta=delta)
    y, st = run_global(dc, img, out_dt, mode="histeq", delta=delta)
    u64 = (np.log(L64 + delta) - ref["lmin"]) / (ref["lmax"] - ref["lmin"])
    lo, hi, amb = hist_bounds(256.0 * u64, 256 * 1e-6)
    assert np.all(st["hist"] >= lo) and np.all(st["hist"] <= hi)
    assert int(st["hist"].sum()) == L64.size
    slack = int(amb.sum()) / L64.size
    if out_dt == "f32":
        check_f32(y, y64, tol=TOL_F32 + slack, what="histeq hdr")
    else:
        h = y.astype(np.float64)
        assert np.all(np.abs(h - y64) <= 2 ** -11 * np.maximum(np.abs(y64), 2 ** -14) + TOL_F32 + slack)


def test_constant_images(dc, oracle_mod):
    img = np.full((37, 53, 3), 128, dtype=np.uint8)
    y, st = run_global(dc, img, "f32")
    check_f32(y, np.full((37, 53), 0.5), what="constant sigmoid")
    y, st = run_global(dc, img, "f32", mode="histeq")
    check_f32(y, np.ones((37, 53)), what="constant histeq")
    assert st["hist"][128] == 37 * 53


@pytest.mark.parametrize("H,W,pad,off", [(1, 1, 0, 0), (3, 17, 2, 1), (50, 33, 0, 3), (17, 1, 4, 0)])
@pytest.mark.parametrize("in_dt", [np.uint8, np.float32])
def test_odd_layouts(dc, oracle_mod, H, W, pad, off, in_dt):
    from paper_2108_13656_gb300 import synth
    if in_dt == np.uint8:
        img = synth.s_ldr(max(W, 4), max(H, 4), seed=H + W)[:H, :W]
    else:
        img = synth.s_hdr(max(W, 4), max(H, 4), seed=H + W)[:H, :W]
    L64 = oracle_mod.decolorize(img)
    y64, _ = oracle_mod.tonemap_global_plane(L64, ldr=in_dt == np.uint8)
    y, _ = run_global(dc, img, "f32", pad=pad, off=off)
    check_f32(y, y64, what="odd %dx%d" % (H, W))
