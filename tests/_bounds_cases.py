"""Odd shapes, strides, offsets, batches and parameters run through the library;
used by test_gpu_bounds.py in two processes (the bounds-checked build and the normal
one).  Run as a script it writes the outputs to the .npz file named on the command
line and prints the bounds flags."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))


def cases():
    from paper_2108_13656_gb300 import synth
    sizes = [(1, 1), (17, 1), (1, 17), (97, 61), (333, 97), (64, 48)]
    imgs = {}
    for i, (w, h) in enumerate(sizes):
        imgs[("u8", w, h)] = synth.s_ldr(w, h, 40 + i)
        hdr = synth.s_hdr(max(w, 2), max(h, 2), 50 + i)[:h, :w]
        imgs[("f32", w, h)] = np.ascontiguousarray(hdr)
        imgs[("f16", w, h)] = np.ascontiguousarray(hdr.astype(np.float16))
    return imgs


def run():
    import torch
    import paper_2108_13656_gb300 as dc
    from _dev import to_dev
    imgs = cases()
    out = {}
    keys = sorted(imgs)
    for j, key in enumerate(keys):
        img = imgs[key]
        h, w = img.shape[:2]
        for pad, off in [(0, 0), (3, 5)]:
            x = to_dev(img, pad_px=pad, offset_elems=off)
            for odt in (torch.uint8, torch.float16, torch.float32):
                y = torch.zeros((h, w + pad), dtype=odt, device="cuda")[:, :w]
                tag = "%s_%dx%d_p%d_%s" % (key[0], w, h, pad, str(odt).split(".")[-1])
                dc.decolorize(x, y)
                out["dec_" + tag] = y.cpu().numpy().copy()
                dc.decolorize_tonemap_global(x, y, mode="sigmoid")
                out["sig_" + tag] = y.cpu().numpy().copy()
                dc.decolorize_tonemap_global(x, y, mode="histeq")
                out["he_" + tag] = y.cpu().numpy().copy()
                dc.decolorize_tonemap_local(x, y)
                out["loc_" + tag] = y.cpu().numpy().copy()
                dc.decolorize_tonemap_local(x, y, block_s=5, radius_blocks=3, bins=7, alpha=0.6)
                out["loc5_" + tag] = y.cpu().numpy().copy()
                # comparison channels
                for luma in ("y", "v"):
                    dc.decolorize(x, y, luma=luma)
                    out["dec%s_" % luma + tag] = y.cpu().numpy().copy()
                    dc.decolorize_tonemap_local(x, y, luma=luma, block_s=8)
                    out["loc%s_" % luma + tag] = y.cpu().numpy().copy()
                # colour outputs (3 interleaved samples per pixel, padded rows)
                y3 = torch.zeros((h, w + pad, 3), dtype=odt, device="cuda")[:, :w, :]
                for s in (1.0, 0.6):
                    dc.decolorize_tonemap_global(x, y3, mode="sigmoid", color_s=s)
                    out["csig%g_" % s + tag] = y3.cpu().numpy().copy()
                    dc.decolorize_tonemap_local(x, y3, color_s=s, block_s=8, bins=12)
                    out["cloc%g_" % s + tag] = y3.cpu().numpy().copy()
                dc.decolorize_tonemap_global(x, y3, mode="histeq")
                out["che_" + tag] = y3.cpu().numpy().copy()
                # frame sequences: a restarted frame and a running one
                vs = dc.VideoStreams(1, lam=0.5)
                vs(x, y)
                out["vid0_" + tag] = y.cpu().numpy().copy()
                vs(x, y)
                out["vid1_" + tag] = y.cpu().numpy().copy()
                lv = dc.VideoLocalStreams(1, block_s=8, bins=12)
                lv(x, y)
                out["lvid0_" + tag] = y.cpu().numpy().copy()
                lv(x, y)
                out["lvid1_" + tag] = y.cpu().numpy().copy()
    # a ragged batch of every image, each type through the same call
    xs = [to_dev(imgs[k]) for k in keys]
    ys = [torch.zeros(x.shape[:2], dtype=torch.float32, device="cuda") for x in xs]
    dc.decolorize_tonemap_local(xs, ys, block_s=64)
    for k, y in zip(keys, ys):
        out["batchloc_%s_%dx%d" % k] = y.cpu().numpy().copy()
    dc.decolorize_tonemap_global(xs, ys, mode="histeq")
    for k, y in zip(keys, ys):
        out["batchhe_%s_%dx%d" % k] = y.cpu().numpy().copy()
    torch.cuda.synchronize()
    return out


if __name__ == "__main__":
    import paper_2108_13656_gb300 as dc
    res = run()
    np.savez(sys.argv[1], **res)
    checked, flags = dc.debug_bounds()
    print("bounds checked=%d flags=%d" % (checked, flags))
