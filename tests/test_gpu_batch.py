"""Ragged batch of 256 8-bit images (sizes from 320x240 to 4096x3072, seed 3):
decolorize + global sigmoid as one batched call replayed from a CUDA graph, against
256 single-image calls and against the FP64 oracle; the autotuner's choice changes
no result."""
import numpy as np
import pytest

from _cmp import check_u8

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2108_13656_gb300 as m
    m.load()
    return m


def ragged_batch_on_device(n, seed):
    """The ragged batch built on the device from one base image per size (host copies
    of the bases are returned for the oracle)."""
    import torch
    from paper_2108_13656_gb300 import synth
    sizes, shifts = synth.ragged_batch_spec(n, seed)
    bases = {sz: synth.ragged_base(sz) for sz in sorted(set(sizes))}
    dev_bases = {sz: torch.from_numpy(b).cuda() for sz, b in bases.items()}
    xs = [torch.roll(dev_bases[sz], shifts=sh, dims=(0, 1)).contiguous() for sz, sh in zip(sizes, shifts)]
    return sizes, shifts, bases, xs


def test_ragged_256_graph_equals_plain_and_oracle(dc, oracle_mod):
    import torch
    from paper_2108_13656_gb300 import synth
    from paper_2108_13656_gb300.batch import GraphCall, plain_calls
    sizes, shifts, bases, xs = ragged_batch_on_device(256, 3)
    ys = [torch.empty(x.shape[:2], dtype=torch.uint8, device="cuda") for x in xs]
    g = GraphCall("global", xs, ys)
    assert g.launches == 2  # statistics pass + curve pass for the whole batch
    for y in ys:
        y.fill_(7)
    g.replay()
    torch.cuda.synchronize()
    assert dc.query_status(g.workspace) == 0
    ref = [torch.empty_like(y) for y in ys]
    for c in plain_calls("global", xs, ref):
        c()
    torch.cuda.synchronize()
    for i, (a, b) in enumerate(zip(ys, ref)):
        assert torch.equal(a, b), "image %d differs between the batch and its own call" % i
    # oracle on the first image of every size
    seen = set()
    for i, (sz, sh) in enumerate(zip(sizes, shifts)):
        if sz in seen:
            continue
        seen.add(sz)
        img = synth.shifted(bases[sz], *sh)
        y64, _ = oracle_mod.tonemap_global(img)
        check_u8(ys[i].cpu().numpy(), y64, "ragged image %d %s" % (i, sz))
    assert len(seen) == len(synth.RAGGED_SIZE_CHOICES)


def test_autotuner_choice_changes_no_result(dc, tmp_path):
    import torch
    from paper_2108_13656_gb300.autotune import Autotuner, TuneCache
    sizes, shifts, bases, xs = ragged_batch_on_device(24, 11)
    ys0 = [torch.empty(x.shape[:2], dtype=torch.float32, device="cuda") for x in xs]
    ys1 = [torch.empty_like(y) for y in ys0]
    orig = dc.get_tuning(dc.DC_OP_GLOBAL, dc.DC_U8)
    try:
        dc.decolorize_tonemap_global(xs, ys0)
        tuner = Autotuner(TuneCache(str(tmp_path / "tune.json")), reps=2)
        choice, timings = tuner.tune("global", xs, ys1)
        assert len(timings) >= 4 and all(t > 0 for t in timings.values())
        dc.decolorize_tonemap_global(xs, ys1)
        torch.cuda.synchronize()
        for a, b in zip(ys0, ys1):
            assert torch.equal(a, b)
        # a second tuner with the same cache file answers from the cache
        again, _ = Autotuner(TuneCache(str(tmp_path / "tune.json"))).tune("global", xs, ys1)
        assert again == choice
    finally:
        dc.set_tuning(dc.DC_OP_GLOBAL, dc.DC_U8, *orig)


def test_local_batch_graph_equals_plain(dc):
    import torch
    from paper_2108_13656_gb300 import synth
    from paper_2108_13656_gb300.batch import GraphCall, plain_calls
    imgs = [synth.s_hdr(w, h, 20 + i).astype(np.float16) for i, (w, h) in
            enumerate([(640, 480), (333, 97), (1280, 720), (64, 64)])]
    xs = [torch.from_numpy(im).cuda() for im in imgs]
    ys = [torch.empty(x.shape[:2], dtype=torch.float32, device="cuda") for x in xs]
    ref = [torch.empty_like(y) for y in ys]
    g = GraphCall("local", xs, ys)
    assert g.launches == 4
    g.replay()
    for c in plain_calls("local", xs, ref):
        c()
    torch.cuda.synchronize()
    for a, b in zip(ys, ref):
        assert torch.equal(a, b)
