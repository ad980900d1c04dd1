"""GPU parity of the comparison channels, colour reconstruction, frame sequences and
parameter presets against the FP64 oracle.

- Channels (Sec. I rgb2gray Y, V of HSV; Fig. GTMO): decolorize, global and local
  tone mapping of each channel.
- Colour outputs (reading of the colour results of Fig. tmo_1 / Fig. GTMO):
  C_out = min(1, y (C/L)^s) for both operators, every input and output sample type,
  several exponents, ragged and padded layouts, and a batch mixing gray and colour
  outputs.
- Frame sequences: every frame and the carried estimate against the oracle's
  sequence; a restarted frame equals the global call bit for bit.
- TM1 / TM2 presets (Fig. SLHE_TMO(c)): the local operator at the preset's betas
  against the oracle, and the background boost / suppression they stand for.
"""
import numpy as np
import pytest

from _cmp import check_f32, check_out
from _dev import to_dev

pytestmark = pytest.mark.gpu

TDT = {"u8": "uint8", "f16": "float16", "f32": "float32"}


@pytest.fixture(scope="module")
def dc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2108_13656_gb300 as m
    m.load()
    return m


def _empty(shape, dt):
    import torch
    return torch.empty(shape, dtype=getattr(torch, TDT[dt]), device="cuda")


def _img(kind, w, h, seed):
    from paper_2108_13656_gb300 import synth
    if kind == "u8":
        return synth.s_ldr(w, h, seed=seed)
    hdr = synth.s_hdr(w, h, seed=seed)
    return hdr.astype(np.float16) if kind == "f16" else hdr


def _check_rgb(got, ref, dt, what):
    for c in range(3):
        check_out(got[..., c], ref[..., c], dt, what="%s channel %d" % (what, c))


# -------------------------------------------------------------- channels ----
CH = {"y": 1, "v": 2, "lstar": 3}


@pytest.mark.parametrize("luma", ["y", "v", "lstar"])
@pytest.mark.parametrize("kind", ["u8", "f16", "f32"])
def test_channel_decolorize(dc, oracle_mod, luma, kind):
    import torch
    img = _img(kind, 203, 61, 21)
    ch = CH[luma]
    L64 = oracle_mod.decolorize(img, channel=ch)
    odt = "u8" if kind == "u8" else "f32"
    y = _empty(img.shape[:2], odt)
    dc.decolorize(to_dev(img), y, luma=luma)
    torch.cuda.synchronize()
    check_out(y.cpu().numpy(), L64, odt, what="decolorize %s %s" % (luma, kind), rel=True)


@pytest.mark.parametrize("luma", ["y", "v", "lstar"])
@pytest.mark.parametrize("op", ["global", "histeq", "local"])
@pytest.mark.parametrize("kind", ["u8", "f32"])
def test_channel_tonemap(dc, oracle_mod, luma, op, kind):
    import torch
    img = _img(kind, 333, 190, 22)
    ch = CH[luma]
    L64 = oracle_mod.decolorize(img, channel=ch)
    ldr = kind == "u8"
    for odt in ("u8", "f32"):
        y = _empty(img.shape[:2], odt)
        x = to_dev(img)
        if op == "local" and luma == "lstar" and kind == "u8" and odt == "f32":
            with pytest.raises(dc.DcError) as e:  # not offered: see DC_LUMA_LSTAR
                dc.decolorize_tonemap_local(x, y, luma=luma, block_s=16)
            assert e.value.status == 2
            continue
        if op == "local":
            dc.decolorize_tonemap_local(x, y, luma=luma, block_s=16)
            ref = oracle_mod.tonemap_local_plane(L64, ldr=ldr, block_s=16)
        else:
            mode = "sigmoid" if op == "global" else "histeq"
            dc.decolorize_tonemap_global(x, y, mode=mode, luma=luma)
            ref, _ = oracle_mod.tonemap_global_plane(L64, ldr=ldr, mode=1 if op == "histeq" else 0)
        torch.cuda.synchronize()
        check_out(y.cpu().numpy(), ref, odt, what="%s %s %s -> %s" % (op, luma, kind, odt))


# ------------------------------------------------------- colour outputs ----
@pytest.mark.parametrize("kind", ["u8", "f16", "f32"])
@pytest.mark.parametrize("op", ["global", "histeq", "local"])
@pytest.mark.parametrize("odt", ["u8", "f16", "f32"])
def test_colour_output(dc, oracle_mod, kind, op, odt):
    import torch
    img = _img(kind, 259, 97, 23)
    x = to_dev(img)
    for s in (1.0, 0.6):
        out = _empty(img.shape[:2] + (3,), odt)
        if op == "local":
            dc.decolorize_tonemap_local(x, out, block_s=16, color_s=s)
            ref = oracle_mod.tonemap_local_color(img, s=s, block_s=16)
        else:
            mode = 0 if op == "global" else 1
            dc.decolorize_tonemap_global(x, out, mode=mode, color_s=s)
            ref = oracle_mod.tonemap_global_color(img, s=s, mode=mode)
        torch.cuda.synchronize()
        _check_rgb(out.cpu().numpy(), ref, odt, "colour %s %s -> %s s=%g" % (op, kind, odt, s))


@pytest.mark.parametrize("s", [0.0, 2.0])
@pytest.mark.parametrize("luma", ["ours", "y", "v"])
def test_colour_exponents_and_channels(dc, oracle_mod, s, luma):
    import torch
    img = _img("f32", 190, 77, 24)
    ch = {"ours": 0, "y": 1, "v": 2}[luma]
    out = _empty(img.shape[:2] + (3,), "f32")
    dc.decolorize_tonemap_global(to_dev(img), out, color_s=s, luma=luma)
    torch.cuda.synchronize()
    _check_rgb(out.cpu().numpy(), oracle_mod.tonemap_global_color(img, s=s, channel=ch), "f32",
               "colour s=%g %s" % (s, luma))


@pytest.mark.parametrize("H,W,pad,off", [(1, 1, 0, 0), (3, 17, 1, 1), (41, 67, 3, 0), (9, 130, 0, 5)])
@pytest.mark.parametrize("kind", ["u8", "f32"])
def test_colour_odd_layouts(dc, oracle_mod, H, W, pad, off, kind):
    import torch
    img = _img(kind, max(W, 4), max(H, 4), H * W + 1)[:H, :W]
    x = to_dev(img, pad_px=pad, offset_elems=off)
    for op in ("global", "local"):
        for odt in ("u8", "f32"):
            buf = _empty((off + H * (W + pad) * 3 + 64,), odt)
            out = buf[off:off + H * (W + pad) * 3].view(H, W + pad, 3)[:, :W, :]
            if op == "global":
                dc.decolorize_tonemap_global(x, out)
                ref = oracle_mod.tonemap_global_color(img)
            else:
                dc.decolorize_tonemap_local(x, out, block_s=8, bins=16)
                ref = oracle_mod.tonemap_local_color(img, block_s=8, bins=16)
            torch.cuda.synchronize()
            _check_rgb(out.cpu().numpy(), ref, odt, "colour %s %dx%d %s -> %s" % (op, H, W, kind, odt))


def test_batch_mixing_gray_and_colour(dc, oracle_mod):
    import torch
    imgs = [_img("u8", 200, 90, 25), _img("f32", 150, 70, 26), _img("u8", 64, 33, 27), _img("f16", 80, 40, 28)]
    outs = [_empty(imgs[0].shape[:2] + (3,), "u8"), _empty(imgs[1].shape[:2], "f32"),
            _empty(imgs[2].shape[:2], "u8"), _empty(imgs[3].shape[:2] + (3,), "f32")]
    xs = [to_dev(im) for im in imgs]
    for op in ("global", "local"):
        if op == "global":
            dc.decolorize_tonemap_global(xs, outs)
        else:
            dc.decolorize_tonemap_local(xs, outs, block_s=16)
        torch.cuda.synchronize()
        for im, o in zip(imgs, outs):
            g = o.cpu().numpy()
            odt = "u8" if o.dtype == torch.uint8 else "f32"
            if g.ndim == 3:
                ref = (oracle_mod.tonemap_global_color(im) if op == "global"
                       else oracle_mod.tonemap_local_color(im, block_s=16))
                _check_rgb(g, ref, odt, "mixed batch colour " + op)
            else:
                ref = (oracle_mod.tonemap_global(im)[0] if op == "global" else oracle_mod.tonemap_local(im, block_s=16))
                check_out(g, ref, odt, what="mixed batch gray " + op)


# ------------------------------------------------------- frame sequences ----
def _frames(kind, n, w=320, h=180):
    """A short synthetic sequence: one scene shifted frame to frame with a brightness ramp."""
    from paper_2108_13656_gb300 import synth
    base = _img(kind, w, h, 29)
    out = []
    for t in range(n):
        f = synth.shifted(base, 3 * t, 5 * t)
        if kind == "u8":
            f = np.clip(f.astype(np.float64) * (1.0 + 0.08 * t), 0, 255).astype(np.uint8)
        else:
            f = (f.astype(np.float64) * (1.0 + 0.5 * t)).astype(f.dtype)
        out.append(np.ascontiguousarray(f))
    return out


@pytest.mark.parametrize("lam", [1.0, 0.3])
@pytest.mark.parametrize("kind", ["u8", "f32"])
def test_video_sequence(dc, oracle_mod, lam, kind):
    import torch
    frames = _frames(kind, 5)
    ys64, ms64 = oracle_mod.tonemap_video_global(frames, lam=lam)
    vs = dc.VideoStreams(1, lam=lam)
    for t, f in enumerate(frames):
        odt = "f32"
        y = _empty(f.shape[:2], odt)
        vs(to_dev(f), y)
        torch.cuda.synchronize()
        check_f32(y.cpu().numpy(), ys64[t], what="video %s frame %d" % (kind, t))
        st = vs.states()[0]
        assert st["frames"] == t + 1
        assert abs(st["m"] - ms64[t]) <= 1e-6 * max(1.0, abs(ms64[t])), (st, ms64[t])


def test_video_streams_batch_and_restart(dc, oracle_mod):
    import torch
    seqs = [_frames("u8", 3, 256, 128), _frames("f16", 3, 200, 100)]
    vs = dc.VideoStreams(2, lam=0.5)
    refs = [oracle_mod.tonemap_video_global(s, lam=0.5)[0] for s in seqs]
    for t in range(3):
        outs = [_empty(seqs[0][t].shape[:2], "u8"), _empty(seqs[1][t].shape[:2], "f32")]
        vs([to_dev(seqs[0][t]), to_dev(seqs[1][t])], outs)
        torch.cuda.synchronize()
        check_out(outs[0].cpu().numpy(), refs[0][t], "u8", what="stream 0 frame %d" % t)
        check_out(outs[1].cpu().numpy(), refs[1][t], "f32", what="stream 1 frame %d" % t)
    # a restarted frame is the global call's result, bit for bit
    vs.restart()
    f = seqs[1][2]
    a, b = _empty(f.shape[:2], "f32"), _empty(f.shape[:2], "f32")
    vs([to_dev(seqs[0][2]), to_dev(f)], [_empty(seqs[0][2].shape[:2], "u8"), a])
    dc.decolorize_tonemap_global(to_dev(f), b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert [s["frames"] for s in vs.states()] == [1, 1]


def test_video_one_launch_per_frame(dc):
    import torch
    frames = _frames("f32", 3)
    vs = dc.VideoStreams(1)
    for t, f in enumerate(frames):
        vs(to_dev(f), _empty(f.shape[:2], "f32"))
        assert dc.last_launch_count() == (2 if t == 0 else 1)
    torch.cuda.synchronize()


# ---------------------------------------------------------------- presets ----
def test_presets_local_against_oracle(dc, oracle_mod):
    import torch
    img = _img("u8", 300, 160, 30)
    for name, bk in (("tm1", 0.55), ("tm2", 0.95), ("paper", 0.8)):
        p, lp = dc.preset(name)
        y = _empty(img.shape[:2], "f32")
        dc.decolorize_tonemap_local(to_dev(img), y, beta_r=p.beta_r, beta_k=p.beta_k, block_s=lp.block_s,
                                    radius_blocks=lp.radius_blocks, bins=lp.bins, alpha=lp.alpha)
        torch.cuda.synchronize()
        ref = oracle_mod.tonemap_local(img, beta_R=0.55, beta_k=bk)
        check_f32(y.cpu().numpy(), ref, what="preset " + name)


def test_presets_boost_and_suppress_the_background(dc):
    # a warm (red) foreground on a cool (cyan-blue) background, locally tone-mapped:
    # the background comes out brighter relative to the foreground under TM1 than TM2
    import torch
    H, W = 256, 256
    img = np.zeros((H, W, 3), np.uint8)
    img[...] = (40, 110, 170)
    img[96:160, 96:160] = (200, 40, 30)
    fg = np.zeros((H, W), bool)
    fg[96:160, 96:160] = True
    res = {}
    for name in ("tm1", "tm2"):
        p, lp = dc.preset(name)
        y = _empty((H, W), "f32")
        dc.decolorize(to_dev(img), y, beta_r=p.beta_r, beta_k=p.beta_k)
        torch.cuda.synchronize()
        L = y.cpu().numpy()
        res[name] = L[~fg].mean() - L[fg].mean()
    assert res["tm1"] > res["tm2"]


# ------------------------------------------------- local frame sequences ----
@pytest.mark.parametrize("kind,odt", [("u8", "u8"), ("u8", "f32"), ("f16", "f32"), ("f32", "f32"), ("f32", "u8")])
def test_local_video_sequence(dc, oracle_mod, kind, odt):
    import torch
    frames = _frames(kind, 4, 330, 190)
    kw = dict(block_s=16, radius_blocks=2, bins=24)
    ys64 = oracle_mod.tonemap_video_local(frames, **kw)
    vs = dc.VideoLocalStreams(1, **kw)
    for t, f in enumerate(frames):
        y = _empty(f.shape[:2], odt)
        vs(to_dev(f), y)
        assert dc.last_launch_count() == ((3 if kind == "u8" else 4) if t == 0 else 2)
        torch.cuda.synchronize()
        check_out(y.cpu().numpy(), ys64[t], odt, what="local video %s -> %s frame %d" % (kind, odt, t))


def test_local_video_restart_equals_local_call_and_batches(dc, oracle_mod):
    import torch
    seqs = [_frames("u8", 3, 256, 120), _frames("f32", 3, 200, 96)]
    kw = dict(block_s=8, radius_blocks=1, bins=16, alpha=0.7)
    refs = [oracle_mod.tonemap_video_local(sq, **kw) for sq in seqs]
    vs = dc.VideoLocalStreams(2, **kw)
    for t in range(3):
        outs = [_empty(seqs[0][t].shape[:2], "u8"), _empty(seqs[1][t].shape[:2], "f32")]
        vs([to_dev(seqs[0][t]), to_dev(seqs[1][t])], outs)
        torch.cuda.synchronize()
        check_out(outs[0].cpu().numpy(), refs[0][t], "u8", what="stream 0 frame %d" % t)
        check_out(outs[1].cpu().numpy(), refs[1][t], "f32", what="stream 1 frame %d" % t)
    vs.restart()
    f = seqs[1][2]
    a, b = _empty(f.shape[:2], "f32"), _empty(f.shape[:2], "f32")
    vs([to_dev(seqs[0][2]), to_dev(f)], [_empty(seqs[0][2].shape[:2], "u8"), a])
    dc.decolorize_tonemap_local(to_dev(f), b, **kw)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("H,W,pad,off", [(1, 1, 0, 0), (7, 33, 1, 1), (70, 17, 0, 5)])
def test_local_video_odd_layouts(dc, oracle_mod, H, W, pad, off):
    import torch
    kw = dict(block_s=5, radius_blocks=3, bins=7)
    for kind in ("u8", "f32"):
        base = _img(kind, max(W, 4), max(H, 4), H + W)[:H, :W]
        frames = [base.copy(), base[:, ::-1].copy()]
        ys64 = oracle_mod.tonemap_video_local(frames, **kw)
        vs = dc.VideoLocalStreams(1, **kw)
        for t, f in enumerate(frames):
            x = to_dev(f, pad_px=pad, offset_elems=off)
            buf = _empty((off + H * (W + pad) + 64,), "f32")
            y = buf[off:off + H * (W + pad)].view(H, W + pad)[:, :W]
            vs(x, y)
            torch.cuda.synchronize()
            check_f32(y.cpu().numpy(), ys64[t], what="local video odd %dx%d %s frame %d" % (H, W, kind, t))


@pytest.mark.parametrize("kind,odt", [("u8", "u8"), ("u8", "f32"), ("f32", "f32"), ("f16", "u8")])
@pytest.mark.parametrize("op", ["global", "local"])
def test_video_colour(dc, oracle_mod, kind, odt, op):
    import torch
    frames = _frames(kind, 3, 260, 150)
    if op == "global":
        ys, _ = oracle_mod.tonemap_video_global(frames, lam=0.5)
        vs = dc.VideoStreams(1, lam=0.5)
    else:
        ys = oracle_mod.tonemap_video_local(frames, block_s=16, bins=24)
        vs = dc.VideoLocalStreams(1, block_s=16, bins=24)
    refs = oracle_mod.video_color(frames, ys)
    for t, f in enumerate(frames):
        out = _empty(f.shape[:2] + (3,), odt)
        vs(to_dev(f), out)
        torch.cuda.synchronize()
        _check_rgb(out.cpu().numpy(), refs[t], odt, "colour video %s %s -> %s frame %d" % (op, kind, odt, t))


def _near_edge(x, eps):
    """True where x lies within eps of an integer (a gray-code or bin edge)."""
    return np.abs(x - np.round(x)) < eps


@pytest.mark.parametrize("kind,odt", [("u8", "u8"), ("u8", "f32"), ("f16", "f32"), ("f32", "f32")])
def test_video_histeq_sequence(dc, oracle_mod, kind, odt):
    # frame t is mapped through frame t-1's cumulative histogram: pixels whose own code
    # or bin is within rounding of an edge are exempt, and the previous frame's such
    # pixels (which may have landed in a neighbouring bin of its histogram) bound the
    # slack of every output, as in the single-image histogram-equalisation tests
    import torch
    from _cmp import TOL_F32, check_u8
    frames = _frames(kind, 4, 300, 170)
    ys64 = oracle_mod.tonemap_video_histeq(frames)
    vs = dc.VideoStreams(1, mode="histeq")
    ldr = kind == "u8"
    prev_amb, rng = 0, None
    for t, f in enumerate(frames):
        y = _empty(f.shape[:2], odt)
        vs(to_dev(f), y)
        assert dc.last_launch_count() == ((2 if ldr else 3) if t == 0 else 1)
        torch.cuda.synchronize()
        L64 = oracle_mod.decolorize(f)
        _, lo, hi = oracle_mod.log_stats(L64, 1e-4)
        if ldr:
            amb = _near_edge(255.0 * L64 + 0.5, 255 * 1e-5)
        else:
            r = (lo, hi) if rng is None else rng
            amb = _near_edge(256.0 * np.clip((np.log(L64 + 1e-4) - r[0]) / (r[1] - r[0]), 0, 1), 256 * 1e-6)
        slack = max(int(amb.sum()) if t == 0 else 0, prev_amb) / L64.size
        got = y.cpu().numpy()
        if odt == "f32":
            err = np.abs(got.astype(np.float64) - ys64[t])
            assert np.all(err[~amb] <= TOL_F32 + slack), (t, float(err[~amb].max()))
        else:
            check_u8(got, ys64[t], "histeq video frame %d" % t,
                     extra_exempt=amb | oracle_mod.u8_boundary_mask(ys64[t], 1e-5 + slack))
        prev_amb, rng = int(amb.sum()), (lo, hi)
        st = vs.states()[0]
        assert st["frames"] == t + 1 and int(st["hist"].sum()) == L64.size


def test_video_histeq_restart_equals_the_global_call(dc):
    import torch
    f = _frames("f32", 1)[0]
    a, b = _empty(f.shape[:2], "f32"), _empty(f.shape[:2], "f32")
    dc.VideoStreams(1, mode="histeq")(to_dev(f), a)
    dc.decolorize_tonemap_global(to_dev(f), b, mode="histeq")
    torch.cuda.synchronize()
    assert torch.equal(a, b)
