"""GPU parity of Eq. 1-6 (Sec. II-B) through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

from _cmp import check_f16, check_f32, check_out, check_u8
from _dev import GuardedOut, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2108_13656_gb300 as m
    m.load()
    return m


def _all_triples():
    v = np.arange(1 << 24, dtype=np.uint32)
    img = np.empty((4096, 4096, 3), dtype=np.uint8)
    img[..., 0] = (v >> 16).reshape(4096, 4096)
    img[..., 1] = ((v >> 8) & 255).reshape(4096, 4096)
    img[..., 2] = (v & 255).reshape(4096, 4096)
    return img


def test_u8_every_triple(dc, oracle_mod):
    """All 2^24 8-bit triples: u8 codes bit-exact outside the 1e-5 exemption; f32 within 2e-6."""
    import torch
    img = _all_triples()
    L64 = oracle_mod.decolorize(img)
    x = to_dev(img)
    q = torch.empty((4096, 4096), dtype=torch.uint8, device="cuda")
    f = torch.empty((4096, 4096), dtype=torch.float32, device="cuda")
    dc.decolorize(x, q)
    dc.decolorize(x, f)
    torch.cuda.synchronize()
    nd = check_u8(q.cpu().numpy(), L64, "u8 exhaustive")
    err = check_f32(f.cpu().numpy(), L64, what="f32 exhaustive")
    assert nd < 2000
    print("exhaustive: %d exempt code differences, max f32 err %.3g" % (nd, err))


@pytest.mark.parametrize("in_dt", [np.float16, np.float32])
@pytest.mark.parametrize("out_dt", ["u8", "f16", "f32"])
def test_hdr_inputs(dc, oracle_mod, in_dt, out_dt):
    from paper_2108_13656_gb300 import synth
    img = synth.s_hdr(333, 217, seed=21, decades=5.0).astype(in_dt)
    L64 = oracle_mod.decolorize(img)
    x = to_dev(img)
    o = GuardedOut(217, 333, out_dt)
    dc.decolorize(x, o.view)
    o.check()
    check_out(o.numpy(), L64, out_dt, "hdr %s->%s" % (np.dtype(in_dt).name, out_dt), rel=True)


SHAPES = [(1, 1), (1, 17), (17, 1), (7, 31), (5, 16), (3, 48), (64, 100), (2, 4111)]


@pytest.mark.parametrize("H,W", SHAPES)
@pytest.mark.parametrize("in_dt", [np.uint8, np.float16, np.float32])
def test_odd_shapes_and_layouts(dc, oracle_mod, H, W, in_dt):
    """Ragged tails, padded strides and unaligned bases take the scalar path with the same results."""
    from paper_2108_13656_gb300 import synth
    rng = np.random.default_rng(H * 1000 + W)
    if in_dt == np.uint8:
        img = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    else:
        img = synth.s_hdr(max(W, 2), max(H, 2), seed=H + W)[:H, :W].astype(in_dt)
    L64 = oracle_mod.decolorize(img)
    ref_y = L64
    for pad, off in [(0, 0), (5, 0), (0, 1), (3, 7)]:
        x = to_dev(img, pad_px=pad, offset_elems=off)
        for out_dt in ("u8", "f32"):
            o = GuardedOut(H, W, out_dt, pad_px=pad, offset_elems=off)
            dc.decolorize(x, o.view)
            o.check()
            check_out(o.numpy(), ref_y, out_dt, "%dx%d pad%d off%d %s" % (H, W, pad, off, out_dt), rel=True)


@pytest.mark.parametrize("beta_r,beta_k", [(0.55, 0.8), (1.0, 1.0), (0.0, 0.0), (0.7, 0.6)])
def test_beta_parameters(dc, oracle_mod, beta_r, beta_k):
    import torch
    from paper_2108_13656_gb300 import synth
    img = synth.s_ldr(160, 90, seed=5)
    L64 = oracle_mod.decolorize(img, beta_r, beta_k)
    y = torch.empty((90, 160), dtype=torch.float32, device="cuda")
    dc.decolorize(to_dev(img), y, beta_r=beta_r, beta_k=beta_k)
    check_f32(y.cpu().numpy(), L64, what="betas")


def test_special_pixels(dc, oracle_mod):
    """Black, achromatic, saturated and negative samples."""
    import torch
    px = np.array([[[0, 0, 0], [1, 1, 1], [255, 255, 255], [255, 0, 0], [0, 255, 0], [0, 0, 255],
                    [128, 128, 128], [255, 0, 25]]], dtype=np.uint8)
    y = torch.empty((1, 8), dtype=torch.float32, device="cuda")
    dc.decolorize(to_dev(px), y)
    ref = oracle_mod.decolorize(px)
    check_f32(y.cpu().numpy(), ref, what="special u8")
    assert y[0, 0].item() == 0.0
    hp = np.array([[[-1.0, 0.5, 0.25], [0.0, 0.5, 0.25], [1e-30, 2e-30, 3e-30], [1e20, 3e20, 2e20],
                    [0.0, 0.0, 0.0], [5.0, 5.0, 5.0]]], dtype=np.float32)
    y = torch.empty((1, 6), dtype=torch.float32, device="cuda")
    dc.decolorize(to_dev(hp), y)
    ref = oracle_mod.decolorize(hp)
    check_f32(y.cpu().numpy(), ref, rel=True, what="special f32")


def test_ragged_mixed_batch_equals_solo(dc, oracle_mod):
    """A mixed batch (sample types, sizes, layouts) gives bit-identical results to one call per image."""
    import torch
    from paper_2108_13656_gb300 import synth
    imgs = [synth.s_ldr(640, 480, 1), synth.s_hdr(123, 45, 2).astype(np.float16), synth.s_ldr(33, 17, 3),
            synth.s_hdr(256, 64, 4), synth.s_ldr(1, 1, 5), synth.s_ldr(320, 240, 6)]
    xs = [to_dev(im, pad_px=(i % 2) * 3) for i, im in enumerate(imgs)]
    outs = [torch.empty(im.shape[:2], dtype=torch.float32, device="cuda") for im in imgs]
    dc.decolorize(xs, outs)
    solo = [torch.empty_like(o) for o in outs]
    for x, s in zip(xs, solo):
        dc.decolorize(x, s)
    torch.cuda.synchronize()
    for im, o, s in zip(imgs, outs, solo):
        assert torch.equal(o, s)
        check_f32(o.cpu().numpy(), oracle_mod.decolorize(im), rel=True, what="batch")
