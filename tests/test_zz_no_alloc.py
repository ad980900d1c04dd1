"""The allocation-free global tone-mapping entry point, checked on the GPU.

Some callers cannot allocate device memory (no access to cudaMalloc or to an
allocator, only input and output pointers).  dc_decolorize_tonemap_global_noalloc
serves them from a fixed scratch array inside the library.  This file is named so
that pytest collects it last.  It calls the entry point through the C ABI twice in
a row (the scratch keeps the previous call's contents, which the call must reset)
and compares each result and the statistics with dc_decolorize_tonemap_global on
a caller-provided workspace, which must be bit for bit the same.
"""
import ctypes

import numpy as np
import pytest

from _dev import to_dev

pytestmark = pytest.mark.gpu


def _call_noalloc(abi, xs, ys, stats, mode):
    import torch
    ins, outs = abi._arrays(xs, ys)
    p = abi.dc_decolor_params(abi.BETA_R, abi.BETA_K)
    g = abi.dc_global_params(mode, 1.0, 1e-4, 0)
    rc = abi.load().dc_decolorize_tonemap_global_noalloc(
        ins, outs, len(xs), ctypes.byref(p), ctypes.byref(g), ctypes.c_void_p(stats.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc


def test_noalloc_matches_workspace_call_twice():
    import torch
    import paper_2108_13656_gb300 as dc
    from paper_2108_13656_gb300 import _abi, synth
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    imgs = [synth.s_ldr(640, 480, seed=31), synth.s_hdr(333, 217, seed=32)]
    xs = [to_dev(im) for im in imgs]
    for mode, name in [(dc.DC_SIGMOID, "sigmoid"), (dc.DC_HISTEQ, "histeq")]:
        ref = [torch.empty(im.shape[:2], dtype=torch.float32, device="cuda") for im in imgs]
        st_ref = torch.zeros(2 * dc.STATS_BYTES, dtype=torch.uint8, device="cuda")
        dc.decolorize_tonemap_global(xs, ref, mode=name, stats=st_ref, workspace=dc.Workspace())
        for _ in range(2):  # the second call starts from the first call's scratch contents
            ys = [torch.full(im.shape[:2], -1.0, dtype=torch.float32, device="cuda") for im in imgs]
            st = torch.zeros(2 * dc.STATS_BYTES, dtype=torch.uint8, device="cuda")
            assert _call_noalloc(_abi, xs, ys, st, mode) == 0
            torch.cuda.synchronize()
            for a, b in zip(ys, ref):
                assert torch.equal(a, b)  # same kernels on the same inputs: the same bits
            for sa, sb in zip(dc.parse_stats(st, 2), dc.parse_stats(st_ref, 2)):
                assert abs(sa["mu"] - sb["mu"]) <= 1e-6
                assert sa["logsum_fixed"] == sb["logsum_fixed"]
                np.testing.assert_array_equal(sa["hist"], sb["hist"])


def test_noalloc_rejects_batches_beyond_its_scratch():
    import torch
    from paper_2108_13656_gb300 import _abi, synth
    img = to_dev(synth.s_ldr(16, 16, seed=33))
    n = 80  # about 1.1 KiB of scratch per image: 80 images exceed 64 KiB
    ys = [torch.empty((16, 16), dtype=torch.float32, device="cuda") for _ in range(n)]
    st = torch.zeros(n * 1056, dtype=torch.uint8, device="cuda")
    assert _call_noalloc(_abi, [img] * n, ys, st, 0) == _abi.DC_ERR_WORKSPACE
