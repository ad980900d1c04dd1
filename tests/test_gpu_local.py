"""GPU parity of decolorization + smoothed local-histogram equalisation (Sec. III-B-2)."""
import numpy as np
import pytest

from _cmp import check_f32, check_out
from _dev import GuardedOut, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2108_13656_gb300 as m
    m.load()
    return m


def run_local(dc, img, out_dt, pad=0, off=0, **kw):
    import torch
    H, W = img.shape[:2]
    x = to_dev(img, pad_px=pad, offset_elems=off)
    o = GuardedOut(H, W, out_dt, pad_px=pad, offset_elems=off)
    dc.decolorize_tonemap_local(x, o.view, **kw)
    torch.cuda.synchronize()
    o.check()
    assert dc.query_status() == 0
    return o.numpy()


@pytest.mark.parametrize("out_dt", ["u8", "f32"])
def test_local_ldr(dc, oracle_mod, out_dt):
    from paper_2108_13656_gb300 import synth
    img = synth.s_ldr(300, 200, seed=12)
    y64 = oracle_mod.tonemap_local(img)
    y = run_local(dc, img, out_dt)
    check_out(y, y64, out_dt, "local ldr " + out_dt)


@pytest.mark.parametrize("in_dt", [np.float16, np.float32])
@pytest.mark.parametrize("out_dt", ["u8", "f16", "f32"])
def test_local_hdr(dc, oracle_mod, in_dt, out_dt):
    from paper_2108_13656_gb300 import synth
    img = synth.s_hdr(350, 260, seed=13, decades=6.0, sigma=2.76).astype(in_dt)
    y64 = oracle_mod.tonemap_local(img)
    y = run_local(dc, img, out_dt)
    check_out(y, y64, out_dt, "local hdr " + out_dt)


@pytest.mark.parametrize("s,R,B,alpha", [(16, 1, 16, 0.7), (24, 2, 32, 1.0), (5, 0, 8, 1.0), (32, 3, 2, 0.5),
                                         (64, 1, 20, 1.0), (1, 2, 4, 1.0)])
def test_local_parameters(dc, oracle_mod, s, R, B, alpha):
    from paper_2108_13656_gb300 import synth
    img = synth.s_hdr(170, 97, seed=14)
    kw = dict(block_s=s, radius_blocks=R, bins=B, alpha=alpha)
    y64 = oracle_mod.tonemap_local(img, **kw)
    y = run_local(dc, img, "f32", **kw)
    check_f32(y, y64, what="local params %r" % (kw,))


@pytest.mark.parametrize("H,W,pad,off", [(1, 1, 0, 0), (2, 3, 1, 1), (33, 65, 3, 0), (70, 17, 0, 5)])
def test_local_odd_layouts(dc, oracle_mod, H, W, pad, off):
    from paper_2108_13656_gb300 import synth
    img = synth.s_ldr(max(W, 4), max(H, 4), seed=H * W)[:H, :W]
    y64 = oracle_mod.tonemap_local(img, block_s=16, radius_blocks=1, bins=16)
    y = run_local(dc, img, "f32", pad=pad, off=off, block_s=16, radius_blocks=1, bins=16)
    check_f32(y, y64, what="local odd %dx%d" % (H, W))


def test_local_constant_image(dc, oracle_mod):
    img = np.full((64, 96, 3), 77, dtype=np.uint8)
    y64 = oracle_mod.tonemap_local(img)
    y = run_local(dc, img, "f32")
    check_f32(y, y64, what="local constant")


def test_local_batch_equals_solo(dc, oracle_mod):
    import torch
    from paper_2108_13656_gb300 import synth
    imgs = [synth.s_hdr(200, 100, 1), synth.s_hdr(64, 300, 2).astype(np.float16), synth.s_hdr(31, 7, 3)]
    xs = [to_dev(im) for im in imgs]
    outs = [torch.empty(im.shape[:2], dtype=torch.float32, device="cuda") for im in imgs]
    dc.decolorize_tonemap_local(xs, outs)
    for im, x, o in zip(imgs, xs, outs):
        s = torch.empty_like(o)
        dc.decolorize_tonemap_local(x, s)
        torch.cuda.synchronize()
        assert torch.equal(o, s)
        check_f32(o.cpu().numpy(), oracle_mod.tonemap_local(im), what="local batch")
