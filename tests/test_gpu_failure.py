"""A call that fails partway through its chain of passes must not spoil the next one.

The library's launch-failure hook (dc_debug_fail_launch) makes the k-th kernel
launch of a call return DC_ERR_CUDA without issuing it, after the earlier passes
were enqueued; those passes leave partial counters in the workspace's control
block.  The next call on the same workspace - a registered one, whose control
block is normally left clean by the previous call's last pass, or the
allocation-free entry point's fixed scratch - must clear them and give exactly the
result of a call on a fresh workspace.  No GPU fault is involved.
"""
import ctypes

import pytest

from _cmp import check_out
from _dev import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture
def dc():
    import torch
    import paper_2108_13656_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    m.debug_fail_launch(0)
    yield m
    m.debug_fail_launch(0)


def _images():
    from paper_2108_13656_gb300 import synth
    return [synth.s_ldr(517, 203, seed=41), synth.s_hdr(389, 266, seed=42)]


def _outs(imgs, dt):
    import torch
    tdt = {"u8": torch.uint8, "f32": torch.float32}[dt]
    return [torch.full(im.shape[:2], 7, dtype=tdt, device="cuda") for im in imgs]


@pytest.mark.parametrize("op,fail_at", [("global", 2), ("local", 2), ("local", 3), ("local", 4)])
def test_registered_workspace_after_a_failed_launch(dc, op, fail_at):
    import torch
    imgs = _images()
    xs = [to_dev(im) for im in imgs]
    kw = {"mode": "sigmoid"} if op == "global" else {"block_s": 16}
    for odt in ("u8", "f32"):
        xs_, imgs_ = xs, imgs
        ref = _outs(imgs_, odt)
        dc.PreparedCall(op, xs_, ref, workspace=dc.Workspace(), **kw)()
        ws = dc.Workspace()
        call = dc.PreparedCall(op, xs_, _outs(imgs_, odt), workspace=ws, **kw)
        call()  # a clean call first: the block is registered clean afterwards
        dc.debug_fail_launch(fail_at)
        with pytest.raises(dc.DcError) as e:
            call()
        assert e.value.status == 4  # DC_ERR_CUDA
        dc.debug_fail_launch(0)
        for _ in range(2):
            ys = _outs(imgs_, odt)
            dc.PreparedCall(op, xs_, ys, workspace=ws, **kw)()
            torch.cuda.synchronize()
            for a, b in zip(ys, ref):
                assert torch.equal(a, b)
        assert dc.query_status(ws) == 0


def test_failed_call_then_oracle(dc, oracle_mod):
    import torch
    img = _images()[0]
    x = to_dev(img)
    ws = dc.Workspace()
    y = torch.empty(img.shape[:2], dtype=torch.float32, device="cuda")
    dc.decolorize_tonemap_global(x, y, workspace=ws)
    dc.debug_fail_launch(2)
    with pytest.raises(dc.DcError):
        dc.decolorize_tonemap_global(x, y, workspace=ws)
    dc.debug_fail_launch(0)
    dc.decolorize_tonemap_global(x, y, workspace=ws)
    torch.cuda.synchronize()
    ref, _ = oracle_mod.tonemap_global(img)
    check_out(y.cpu().numpy(), ref, "f32", what="global after a failed call")


def test_noalloc_scratch_after_a_failed_launch(dc):
    import torch
    from paper_2108_13656_gb300 import _abi
    imgs = _images()
    xs = [to_dev(im) for im in imgs]
    ref = _outs(imgs, "f32")
    dc.decolorize_tonemap_global(xs, ref, workspace=dc.Workspace())
    p = _abi.dc_decolor_params(_abi.BETA_R, _abi.BETA_K)
    g = _abi.dc_global_params(_abi.DC_SIGMOID, 1.0, 1e-4, 0)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(ys):
        ins, outs = _abi._arrays(xs, ys)
        return _abi.load().dc_decolorize_tonemap_global_noalloc(ins, outs, len(xs), ctypes.byref(p),
                                                                ctypes.byref(g), None, st)

    assert call(_outs(imgs, "f32")) == 0
    dc.debug_fail_launch(2)
    assert call(_outs(imgs, "f32")) == _abi.DC_ERR_CUDA
    dc.debug_fail_launch(0)
    for _ in range(2):
        ys = _outs(imgs, "f32")
        assert call(ys) == 0
        torch.cuda.synchronize()
        for a, b in zip(ys, ref):
            assert torch.equal(a, b)


def test_hook_rejects_negative(dc):
    with pytest.raises(dc.DcError):
        dc.debug_fail_launch(-1)
