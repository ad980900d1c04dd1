"""Parity at the full workload sizes, in the launch configuration bench.py times.

- 512 x 512 8-bit S-LDR (seed 0), decolorize only: every pixel against the oracle.
- 3840 x 2160 8-bit S-LDR (seed 1) and FP32 S-HDR over 5 decades (seed 2), both
  tone-mapping operators: every pixel against the oracle; the 8-bit image also with
  f32 outputs (the local operator's precise bin coordinate).
- 7680 x 4320 S-HDR over 6 decades (mu = 0, sigma = 2.76, seed 4), local operator, FP16 storage and FP32
  storage with FP32 arithmetic: every pixel against the oracle run on the stored
  samples, and the error against the FP32 original reported (the precision study;
  run with -s to see the numbers).
"""
import numpy as np
import pytest

from _cmp import TOL_F32, check_f32, check_u8
from _dev import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2108_13656_gb300 as m
    m.load()
    return m


def _run(dc, op, img, out_dtype, **kw):
    """One call through the C ABI with the default (bench) launch configuration."""
    import torch
    x = to_dev(img)
    y = torch.empty(img.shape[:2], dtype=out_dtype, device="cuda")
    ws = dc.Workspace()
    dc.PreparedCall(op, x, y, workspace=ws, **kw)()
    torch.cuda.synchronize()
    assert dc.query_status(ws) == 0
    return y.cpu().numpy()


def test_config_512_decolorize(dc, oracle_mod):
    import torch
    from paper_2108_13656_gb300 import synth
    img = synth.s_ldr(512, 512, seed=0)
    y = _run(dc, "decolorize", img, torch.uint8)
    check_u8(y, oracle_mod.decolorize(img), "512x512 decolorize")


@pytest.mark.parametrize("variant", ["u8", "f32"])
@pytest.mark.parametrize("op", ["global", "local"])
def test_config_4k(dc, oracle_mod, variant, op):
    import torch
    from paper_2108_13656_gb300 import synth
    if variant == "u8":
        img = synth.s_ldr(3840, 2160, seed=1)
    else:
        img = synth.s_hdr(3840, 2160, seed=2, decades=5.0, sigma=2.5)
    L64 = oracle_mod.decolorize(img)
    ldr = variant == "u8"
    if op == "global":
        y64, _ = oracle_mod.tonemap_global_plane(L64, ldr=ldr)
    else:
        y64 = oracle_mod.tonemap_local_plane(L64, ldr=ldr)
    if variant == "u8":
        y = _run(dc, op, img, torch.uint8)
        check_u8(y, y64, "4K u8 %s" % op)
    else:
        y = _run(dc, op, img, torch.float32)
        err = check_f32(y, y64, what="4K f32 %s" % op)
        print("4K f32 %s: max |err| %.3g" % (op, err))


@pytest.mark.parametrize("op", ["global", "local"])
def test_config_4k_u8_input_f32_output(dc, oracle_mod, op):
    # 8-bit input with an f32 output: the local operator takes its bin coordinate from
    # the float-float luminance, so its output meets the f32 tolerance like the rest
    import torch
    from paper_2108_13656_gb300 import synth
    img = synth.s_ldr(3840, 2160, seed=1)
    L64 = oracle_mod.decolorize(img)
    if op == "global":
        y64, _ = oracle_mod.tonemap_global_plane(L64, ldr=True)
    else:
        y64 = oracle_mod.tonemap_local_plane(L64, ldr=True)
    y = _run(dc, op, img, torch.float32)
    err = check_f32(y, y64, what="4K u8 -> f32 %s" % op)
    print("4K u8 -> f32 %s: max |err| %.3g" % (op, err))


@pytest.mark.parametrize("storage", [np.float16, np.float32])
def test_config_8k_local_precision(dc, oracle_mod, storage):
    import torch
    from paper_2108_13656_gb300 import synth
    img32 = synth.s_hdr(7680, 4320, seed=4, decades=6.0, sigma=2.76)
    img = img32.astype(storage)
    y = _run(dc, "local", img, torch.float32).astype(np.float64)
    y64 = oracle_mod.tonemap_local(img)  # oracle on the stored samples
    err = np.abs(y - y64)
    assert err.max() <= TOL_F32, err.max()
    if storage == np.float16:
        y64_orig = oracle_mod.tonemap_local(img32)  # effect of FP16 storage itself
        e2 = np.abs(y - y64_orig)
        print("8K local f16 storage: vs oracle(stored) max %.3g mean %.3g; vs oracle(f32 original) max %.3g mean %.3g"
              % (err.max(), err.mean(), e2.max(), e2.mean()))
    else:
        print("8K local f32 storage: vs oracle max %.3g mean %.3g" % (err.max(), err.mean()))


@pytest.mark.parametrize("op", ["global", "local"])
@pytest.mark.parametrize("variant", ["u8", "f32"])
def test_config_4k_colour(dc, oracle_mod, variant, op):
    # colour reconstruction of both operators at the bench's 3840x2160 workload, every
    # sample of the interleaved output against the oracle
    import torch
    from paper_2108_13656_gb300 import synth
    img = synth.s_ldr(3840, 2160, seed=1) if variant == "u8" else synth.s_hdr(3840, 2160, seed=2, decades=5.0, sigma=2.5)
    odt = torch.uint8 if variant == "u8" else torch.float32
    x = to_dev(img)
    y = torch.empty(img.shape[:2] + (3,), dtype=odt, device="cuda")
    dc.PreparedCall(op, x, y, workspace=dc.Workspace())()
    torch.cuda.synchronize()
    ref = oracle_mod.tonemap_global_color(img) if op == "global" else oracle_mod.tonemap_local_color(img)
    got = y.cpu().numpy()
    for c in range(3):
        if variant == "u8":
            check_u8(got[..., c], ref[..., c], "4K colour %s channel %d" % (op, c))
        else:
            check_f32(got[..., c], ref[..., c], what="4K colour %s channel %d" % (op, c))


@pytest.mark.parametrize("luma", ["y", "v"])
def test_config_4k_channels(dc, oracle_mod, luma):
    import torch
    from paper_2108_13656_gb300 import synth
    img = synth.s_hdr(3840, 2160, seed=2, decades=5.0, sigma=2.5)
    L64 = oracle_mod.decolorize(img, channel={"y": oracle_mod.LUMA_Y, "v": oracle_mod.LUMA_V}[luma])
    for op in ("global", "local"):
        y = _run(dc, op, img, torch.float32, luma=luma)
        ref = (oracle_mod.tonemap_global_plane(L64, ldr=False)[0] if op == "global"
               else oracle_mod.tonemap_local_plane(L64, ldr=False))
        check_f32(y, ref, what="4K %s %s" % (luma, op))


@pytest.mark.parametrize("variant", ["u8", "f32"])
def test_config_4k_video(dc, oracle_mod, variant):
    # three 4K frames of one stream (the scene shifted and brightened frame to frame)
    # through the one-pass frame-sequence kernel, each against the oracle's sequence
    import torch
    from paper_2108_13656_gb300 import synth
    base = synth.s_ldr(3840, 2160, seed=1) if variant == "u8" else synth.s_hdr(3840, 2160, seed=2, decades=5.0, sigma=2.5)
    frames = []
    for t in range(3):
        f = synth.shifted(base, 7 * t, 11 * t).astype(np.float64) * (1.0 + 0.1 * t)
        frames.append(np.ascontiguousarray(np.clip(f, 0, 255).astype(np.uint8) if variant == "u8" else f.astype(np.float32)))
    ys64, ms64 = oracle_mod.tonemap_video_global(frames, lam=0.5)
    vs = dc.VideoStreams(1, lam=0.5)
    for t, f in enumerate(frames):
        y = torch.empty(f.shape[:2], dtype=torch.float32, device="cuda")
        vs(to_dev(f), y)
        torch.cuda.synchronize()
        check_f32(y.cpu().numpy(), ys64[t], what="4K video %s frame %d" % (variant, t))
        assert abs(vs.states()[0]["m"] - ms64[t]) <= 1e-6 * max(1.0, abs(ms64[t]))
