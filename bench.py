#!/usr/bin/env python3
"""Benchmark: decolorization (Eq. 1-6) fused with global and local tone mapping on GB300.

Workload (one "step"): the 3840x2160 image in its two variants - 8-bit sRGB
(S-LDR, seed 1) and FP32 linear HDR with log-normal luminance over 5 decades
(S-HDR, mu = 0, sigma = 2.5, seed 2) - each through decolorize -> global
centred-sigmoid tone map and decolorize -> local smoothed-LHE tone map, i.e. four
C-ABI calls per step and every step of the hot path.  Inputs are synthetic and
resident in HBM before timing.  `value` times K steps back to back between two CUDA
events, the four calls of a step (independent images, a workspace each) on four side
streams so that their pass chains overlap, rotating through 8 copies of every input
and output so that no step finds its data in L2; the same steps on one stream give
`config.serial_value`.  The per-call breakdown and the roofline time each call alone
between two events after a 256 MiB L2-flushing write.

Prints ONE JSON line (rank 0).  `value` is whole-job Gpix/s (output pixels of all
four calls, all ranks) over device time; `e2e` repeats the step through the public
API with pinned host buffers, host<->device copies inside the timed region, steps
pipelined (paper_2108_13656_gb300.pipeline; the serial form is reported beside it).
`--impl reference` times the FP64 CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

W, H = 3840, 2160
NPIX = W * H
METRIC = "Gpix/s and % of HBM roofline"
L2_FLUSH_BYTES = 256 << 20
ROT = 8  # input / output sets the steady-state loop rotates through
# pass kernels of each call of the step, in launch order
PASSES = {("u8", "global"): ["STATS", "APPLY_G"], ("f32", "global"): ["STATS", "APPLY_G"],
          ("u8", "local"): ["BLOCKH", "CDF", "APPLY_L"], ("f32", "local"): ["STATS_LOG", "BLOCKH", "CDF", "APPLY_L"]}
OPS = [  # (name, input variant, operation, output dtype, algorithmic bytes per pixel)
    ("u8_global", "u8", "global", "u8", 3 + 1),
    ("f32_global", "f32", "global", "f32", 12 + 4),
    ("u8_local", "u8", "local", "u8", 3 + 1),
    ("f32_local", "f32", "local", "f32", 12 + 4),
]
WORKLOAD = ("3840x2160 8-bit sRGB (S-LDR seed 1) + FP32 linear HDR, 5 decades log-normal "
            "(S-HDR mu=0 sigma=2.5 seed 2); each -> decolorize+global sigmoid TM and "
            "decolorize+local smoothed-LHE TM (s=32, R=2, 32 bins)")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--busy-s", type=float, default=0.3, help="device-busy period while clock sampling starts")
    ap.add_argument("--no-extras", action="store_true", help="skip the ragged-batch and serving measurements")
    ap.add_argument("--ragged-images", type=int, default=256)
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate(local_ms: float, world: int, reduce_max) -> tuple[float, float]:
    """Whole-job time = max over ranks; units = every rank's pixels (weak scaling)."""
    t = reduce_max(local_ms)
    return t, world * 4 * NPIX / (t * 1e-3) / 1e9


def make_inputs():
    from paper_2108_13656_gb300 import synth
    ldr = synth.s_ldr(W, H, seed=1)
    hdr = synth.s_hdr(W, H, seed=2, decades=5.0, sigma=2.5)
    return {"u8": ldr, "f32": hdr}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    """Hash of the CUDA/C++ sources with comments and whitespace removed: it changes
    exactly when the code that was profiled changes."""
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2108_13656_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, fn), encoding="utf-8") as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        src = " ".join(src.split())
        h.update(fn.encode() + b"\0" + src.encode())
    return h.hexdigest()[:16]


def ncu_traffic(op_name: str):
    """DRAM bytes per launch from a committed ncu summary, if taken on the current kernels."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    v = d.get("per_launch_bytes", {}).get(op_name)
    return float(v) if v is not None else None


def issue_roofline(op_ms: dict, sm_mhz: float, n_sm: int):
    """Per call, the time the SMs need just to issue its instructions - warp
    instructions (ncu smsp__inst_executed.sum over the call's passes, from the committed
    summary, taken on the current kernels) at one warp instruction per clock per SM
    sub-partition (4 per SM) at the sampled SM clock - and that time over the measured
    call time.  The 8-bit calls move 4 bytes a pixel, so their bound is instruction
    issue, not HBM."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("kernel_source_hash") != kernel_source_hash() or not sm_mhz:
        return None
    per = d.get("per_pass", {})
    out = {}
    for name, var, op, _, _ in OPS:
        keys = ["%s/%s" % (name, k) for k in PASSES[(var, op)]]
        if not all("inst" in per.get(k, {}) for k in keys):
            continue
        inst = sum(per[k]["inst"] for k in keys)
        tinst = sum(per[k].get("thread_inst", 0.0) for k in keys)
        t_issue_us = inst / (4.0 * n_sm * sm_mhz)
        out[name] = {"warp_inst": inst, "thread_inst_per_px": tinst / NPIX, "issue_bound_us": t_issue_us,
                     "measured_us": op_ms[name] * 1e3, "frac": t_issue_us / (op_ms[name] * 1e3),
                     "peak": "%d SMs x 4 warp-instr/clk x %.0f MHz" % (n_sm, sm_mhz)}
    return out or None


# ----------------------------------------------------------------- CPU oracle ----
def oracle_step(imgs, rows: int, r0: int = 0):
    """The FP64 oracle on the band of `rows` rows from row r0 of each variant, all four
    operations."""
    import oracle
    n = 0
    for name, var, op, _, _ in OPS:
        img = imgs[var][r0:r0 + rows]
        if op == "global":
            oracle.tonemap_global(img)
        else:
            oracle.tonemap_local(img)
        n += img.shape[0] * img.shape[1]
    return n


def cpu_baseline(imgs, budget_s: float = 12.0):
    import oracle
    oracle.build()
    rows = 135  # 1/16 of the image per operation
    t0 = time.perf_counter()
    n = oracle_step(imgs, rows)
    dt = time.perf_counter() - t0
    reps = max(1, int(budget_s / max(dt, 1e-3)))
    reps = min(reps, 16)
    t0 = time.perf_counter()
    tot = 0
    for _ in range(reps):
        tot += oracle_step(imgs, rows)
    dt = time.perf_counter() - t0
    out = {"value": tot / dt / 1e9, "unit": "Gpix/s", "cores": 1, "kind": "oracle",
           "sample": "%d repetitions of a %d-row band (%d px) of both 3840-wide variants through all "
                     "four operations, FP64 C oracle, single thread" % (reps, rows, rows * W)}
    # the same oracle on every host core: one thread per core, each on its own band
    # (the C calls release the interpreter lock)
    try:
        ncores = len(os.sched_getaffinity(0))
    except AttributeError:
        ncores = os.cpu_count() or 1
    counts = [0] * ncores

    def worker(k):
        for _ in range(max(1, reps // 2)):
            counts[k] += oracle_step(imgs, rows, (k % (H // rows)) * rows)
    t0 = time.perf_counter()
    ths = [threading.Thread(target=worker, args=(k,)) for k in range(ncores)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    dt = time.perf_counter() - t0
    out["all_cores"] = {"value": sum(counts) / dt / 1e9, "unit": "Gpix/s", "cores": ncores,
                        "sample": "%d threads, each %d repetitions of its own %d-row band" % (ncores, max(1, reps // 2), rows)}
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    imgs = make_inputs()
    import oracle
    oracle.build()
    rows = 135
    for _ in range(max(0, args.warmup)):
        oracle_step(imgs, rows)
    t0 = time.perf_counter()
    n = 0
    for _ in range(args.steps):
        n += oracle_step(imgs, rows)
    dt = time.perf_counter() - t0
    val = n / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Gpix/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD + "; each step a %d-row band of each variant" % rows},
            "cpu_baseline": {"value": val, "unit": "Gpix/s", "cores": 1, "kind": "oracle",
                             "sample": "%d-row band (%d px) of both variants through all four operations "
                                       "per step" % (rows, rows * W)},
            "e2e": {"value": val, "unit": "Gpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------- ragged batch ----
def _event_ms(fn, reps, flush=None):
    import torch
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.fill_(0)
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        fn()
        e.record()
        torch.cuda.synchronize()
        ts.append(s.elapsed_time(e))
    return float(np.median(ts))


def ragged_batch(dev, n_images: int, peak: float) -> dict:
    """Ragged batch of 8-bit images (sizes U{320x240 ... 4096x3072}, seed 3), decolorize
    + global sigmoid: one batched call replayed from a CUDA graph (launch shape from
    the autotuner) against the same batch as one eager call and as one call per image."""
    import torch
    import paper_2108_13656_gb300 as dc
    from paper_2108_13656_gb300 import synth
    from paper_2108_13656_gb300.autotune import Autotuner, TuneCache
    from paper_2108_13656_gb300.batch import GraphCall, plain_calls
    sizes, shifts = synth.ragged_batch_spec(n_images, 3)
    bases = {sz: torch.from_numpy(synth.ragged_base(sz)).to(dev) for sz in sorted(set(sizes))}
    xs = [torch.roll(bases[sz], shifts=sh, dims=(0, 1)).contiguous() for sz, sh in zip(sizes, shifts)]
    del bases
    ys = [torch.empty(x.shape[:2], dtype=torch.uint8, device=dev) for x in xs]
    px = sum(w * h for w, h in sizes)
    orig = dc.get_tuning(dc.DC_OP_GLOBAL, dc.DC_U8)
    try:
        tune_path = os.path.join(os.path.expanduser("~"), ".cache", "decolor_gb300", "bench_tune.json")
        choice, timings = Autotuner(TuneCache(tune_path), reps=3).tune("global", xs, ys)
        g = GraphCall("global", xs, ys)
        graph_ms = _event_ms(g.replay, 7)
        eager = dc.PreparedCall("global", xs, ys, workspace=dc.Workspace(device=dev))
        eager_ms = _event_ms(eager, 7)
        eager_launches = dc.last_launch_count()
        calls = plain_calls("global", xs, ys)

        def run_plain():
            for c in calls:
                c()
        plain_ms = _event_ms(run_plain, 5)
        plain_launches = sum(1 for _ in calls) * 2
        same = True
        ref = [torch.empty_like(y) for y in ys[:16]]
        for c, y in zip(plain_calls("global", xs[:16], ref), ref):
            c()
        g.replay()
        torch.cuda.synchronize()
        same = all(torch.equal(a, b) for a, b in zip(ys[:16], ref))
    finally:
        dc.set_tuning(dc.DC_OP_GLOBAL, dc.DC_U8, *orig)
    alg = 4 * px
    return {"images": n_images, "mpix": px / 1e6, "input_gb": 3 * px / 1e9,
            "graph": {"ms": graph_ms, "gpix_s": px / graph_ms / 1e6, "launches": g.launches,
                      "GBps": alg / graph_ms / 1e6, "frac_of_measured_hbm": alg / graph_ms / 1e6 / peak},
            "batched_eager": {"ms": eager_ms, "gpix_s": px / eager_ms / 1e6, "launches": eager_launches},
            "plain_per_image": {"ms": plain_ms, "gpix_s": px / plain_ms / 1e6, "launches": plain_launches},
            "speedup_graph_vs_plain": plain_ms / graph_ms,
            "autotune": {"choice_tile_cols_ctas_per_sm": list(choice), "us": timings},
            "batch_equals_per_image_first16": same,
            "l2": "inputs (%.2f GB) larger than L2" % (3 * px / 1e9)}


# ------------------------------------------------------------ small decolorize ----
def decolorize_512(dev) -> dict:
    """512x512 8-bit S-LDR (seed 0), decolorize only, u8 output: one launch."""
    import torch
    import paper_2108_13656_gb300 as dc
    from paper_2108_13656_gb300 import synth
    x = torch.from_numpy(synth.s_ldr(512, 512, seed=0)).to(dev)
    y = torch.empty((512, 512), dtype=torch.uint8, device=dev)
    call = dc.PreparedCall("decolorize", x, y, workspace=dc.Workspace(device=dev))
    call()
    ms = _event_ms(call, 50)
    return {"us": ms * 1e3, "gpix_s": 512 * 512 / ms / 1e6, "launches": 1,
            "note": "launch-bound: 1 MB of traffic, below L2 size; L2 not flushed"}


# ----------------------------------------------------------- precision study ----
def precision_8k(dev, peak: float) -> dict:
    """7680x4320 linear HDR over 6 decades (seed 4) through decolorize + local tone
    mapping with FP16 and with FP32 storage (FP32 arithmetic, f32 output): time per
    call and algorithmic bandwidth (10 and 16 bytes per pixel).  The errors against
    the FP64 oracle are measured by the test suite."""
    import torch
    import paper_2108_13656_gb300 as dc
    from paper_2108_13656_gb300 import synth
    W8, H8 = 7680, 4320
    img32 = synth.s_hdr(W8, H8, seed=4, decades=6.0, sigma=2.76)
    out = {}
    for name, npdt, bpp in (("f16", np.float16, 6 + 4), ("f32", np.float32, 12 + 4)):
        x = torch.from_numpy(img32.astype(npdt)).to(dev)
        y = torch.empty((H8, W8), dtype=torch.float32, device=dev)
        call = dc.PreparedCall("local", x, y, workspace=dc.Workspace(device=dev))
        call()
        ms = _event_ms(call, 10)
        out[name] = {"ms": ms, "gpix_s": W8 * H8 / ms / 1e6, "GBps": bpp * W8 * H8 / ms / 1e6,
                     "frac_of_measured_hbm": bpp * W8 * H8 / ms / 1e6 / peak, "bytes_per_px": bpp}
        del x, y, call
    out["l2"] = "inputs (199 / 398 MB) larger than L2"
    return out


# Device sleeps (cycles, about 30 ms) that keep the host ahead of the device: the
# per-call timings enqueue in chunks of HOST_AHEAD_ROUNDS rounds, each behind its own
# sleep (outside every timed event pair), so no timed call waits on the host.
SLEEP_CYCLES = 60_000_000
HOST_AHEAD_ROUNDS = 16


def _alone_ms(calls, flush, reps: int) -> list:
    """Mean device time of each call alone, after an L2-flushing write (none when
    `flush` is None: the call then finds its own data of the previous repetition in
    L2): the host enqueues ahead of the device (device sleeps between chunks), so the
    events time the device only."""
    import torch
    stream = torch.cuda.current_stream()
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
          for _ in calls]
    torch.cuda.synchronize()
    for k in range(reps):
        if k % HOST_AHEAD_ROUNDS == 0:
            torch.cuda._sleep(SLEEP_CYCLES)
        for i, fn in enumerate(calls):
            if flush is not None:
                flush.fill_(k & 0xFF)
            a, b = ev[i][k]
            a.record(stream)
            fn(k)
            b.record(stream)
    torch.cuda.synchronize()
    return [float(np.mean([a.elapsed_time(b) for a, b in e])) for e in ev]


# ------------------------------------------------------------ frame sequences ----
def video_4k(dev, peak: float) -> dict:
    """Frame sequences at 3840x2160: a frame of a running stream is ONE pass for the
    global curve (Eq. 1-6, the sigmoid around the carried log-mean, and the frame's own
    log-sum) and two for the local operator (the fused block-histogram and mapping
    pass, then the table pass).  Each variant alone after an L2-flushing write, and
    frames back to back: 8 frames on rotating buffers captured in one CUDA graph and
    replayed (inputs far above L2)."""
    import torch
    import paper_2108_13656_gb300 as dc
    imgs = make_inputs()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    out = {}
    for var, op, odt, bpp in (("u8", "global", torch.uint8, 4), ("f32", "global", torch.float32, 16),
                              ("u8", "local", torch.uint8, 4), ("f32", "local", torch.float32, 16)):
        xs = [torch.from_numpy(imgs[var]).to(dev) for _ in range(ROT)]
        ys = [torch.empty((H, W), dtype=odt, device=dev) for _ in range(ROT)]
        if op == "global":
            vs = dc.VideoStreams(1, lam=0.5, device=dev, workspace=dc.Workspace(device=dev))
        else:
            vs = dc.VideoLocalStreams(1, device=dev, workspace=dc.Workspace(device=dev))
        calls = [vs.prepare(xs[r], ys[r]) for r in range(ROT)]
        calls[0](restart=True)
        for r in range(ROT):
            calls[r]()
        launches = dc.last_launch_count()
        ms_alone = _alone_ms([lambda k: calls[k % ROT]()], flush, 60)[0]
        g = torch.cuda.CUDAGraph()
        main = torch.cuda.current_stream()
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(main)
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                for r in range(ROT):
                    calls[r](stream=side)
        main.wait_stream(side)
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        reps = 40
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main)
        for _ in range(reps):
            g.replay()
        e1.record(main)
        torch.cuda.synchronize()
        ms_b2b = e0.elapsed_time(e1) / (reps * ROT)
        out[var if op == "global" else var + "_local"] = {"launches_per_frame": launches, "bytes_per_px": bpp,
                    "alone_us": ms_alone * 1e3, "alone_GBps": bpp * NPIX / ms_alone / 1e6,
                    "alone_frac_of_measured_hbm": bpp * NPIX / ms_alone / 1e6 / peak,
                    "back_to_back_us": ms_b2b * 1e3, "back_to_back_gpix_s": NPIX / ms_b2b / 1e6,
                    "back_to_back_GBps": bpp * NPIX / ms_b2b / 1e6,
                    "back_to_back_frac_of_measured_hbm": bpp * NPIX / ms_b2b / 1e6 / peak}
        del g, calls, vs, xs, ys
        torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------- colour outputs ----
def color_4k(dev, peak: float) -> dict:
    """Colour reconstruction at 3840x2160 (interleaved RGB out, s = 1): each call alone
    after an L2-flushing write; algorithmic bytes = input + 3-channel output."""
    import torch
    import paper_2108_13656_gb300 as dc
    imgs = make_inputs()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    out = {}
    for var, odt, bpp in (("u8", torch.uint8, 3 + 3), ("f32", torch.float32, 12 + 12)):
        x = torch.from_numpy(imgs[var]).to(dev)
        y = torch.empty((H, W, 3), dtype=odt, device=dev)
        for op in ("global", "local"):
            kw = {"mode": "sigmoid"} if op == "global" else {}
            call = dc.PreparedCall(op, x, y, workspace=dc.Workspace(device=dev), **kw)
            call()
            ms = _alone_ms([lambda k: call()], flush, 40)[0]
            out["%s_%s" % (var, op)] = {"us": ms * 1e3, "gpix_s": NPIX / ms / 1e6, "bytes_per_px": bpp,
                                        "GBps": bpp * NPIX / ms / 1e6,
                                        "frac_of_measured_hbm": bpp * NPIX / ms / 1e6 / peak,
                                        "launches": dc.last_launch_count()}
    return out


# ------------------------------------------------------------------ serving ----
def host_link_gbps(dev, nbytes: int = 256 << 20, reps: int = 5) -> dict:
    """Pinned host<->device copy bandwidth right now (the serving loop's bound; the
    link is shared with the machine's other GPUs): one direction at a time, then both
    at once on two streams."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    ho = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    d2 = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    s1, s2 = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

    def timed(fn, nb):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize(dev)
        return round(nb * reps / (time.perf_counter() - t0) / 1e9, 1)

    def both():
        with torch.cuda.stream(s1):
            d.copy_(h, non_blocking=True)
        with torch.cuda.stream(s2):
            ho.copy_(d2, non_blocking=True)

    return {"h2d": timed(lambda: d.copy_(h, non_blocking=True), nbytes),
            "d2h": timed(lambda: ho.copy_(d, non_blocking=True), nbytes),
            "both": timed(both, 2 * nbytes)}


def serving(dev, n_requests: int, rate: float) -> dict:
    """The serving trace (Poisson arrivals, sizes 720p..8K, 70% u8 / 30% f16, half
    global, half local, 16 GB budget) through the continuous-batching loop and through
    serial single-image calls."""
    from paper_2108_13656_gb300 import serve
    trace = serve.make_trace(n_requests, rate, seed=5)
    pool = serve.HostPool(trace, device=dev)
    warm = serve.make_trace(min(200, n_requests), rate, seed=6)
    serve.serve_batched(warm, pool, device=dev)
    serve.serve_serial(warm, pool, device=dev)
    link = host_link_gbps(dev)
    b = serve.serve_batched(trace, pool, budget_bytes=16 << 30, device=dev).summary()
    s = serve.serve_serial(trace, pool, device=dev).summary()
    u = serve.serve_batched(trace, pool, budget_bytes=16 << 30, device=dev, inflight_cap=None).summary()
    return {"requests": n_requests, "rate_per_s": rate, "budget_gb": 16, "host_link_gbps": link,
            "offered_gpix_s": sum(r.size[0] * r.size[1] for r in trace) / (trace[-1].t_arrive - trace[0].t_arrive) / 1e9,
            "inflight_cap_gb": serve.INFLIGHT_CAP_BYTES / 2 ** 30,
            "batched": b, "serial_plain": s, "batched_budget_only": u,
            "note": "latency = host-observed completion (event after the device-to-host copy) minus arrival; "
                    "inputs start in pinned host memory, outputs end there"}


# --------------------------------------------------------------------- native ----
def run_native(args):
    import torch
    import paper_2108_13656_gb300 as dc

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dc.load()
    imgs = make_inputs()
    # ROT copies of every input and output: consecutive steps of the steady-state loop
    # touch different buffers (8 x 166 MB, far above L2), so no step finds the previous
    # one's data in L2 and no flush is needed between them
    xs = {k: [torch.from_numpy(v).to(dev) for _ in range(ROT)] for k, v in imgs.items()}
    x = {k: v[0] for k, v in xs.items()}
    outs_r = {}
    for name, var, op, odt, _ in OPS:
        outs_r[name] = [torch.empty((H, W), dtype=torch.uint8 if odt == "u8" else torch.float32, device=dev)
                        for _ in range(ROT)]
    outs = {name: v[0] for name, v in outs_r.items()}
    wss = {name: dc.Workspace(device=dev) for name, *_ in OPS}
    ws = wss[OPS[0][0]]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    calls_r = {}
    for name, var, op, _, _ in OPS:
        kw = {"mode": "sigmoid"} if op == "global" else {}
        calls_r[name] = [dc.PreparedCall(op, xs[var][r], outs_r[name][r], workspace=wss[name], **kw)
                         for r in range(ROT)]
    calls = {name: v[0] for name, v in calls_r.items()}

    def call(name, var, op, out):
        calls[name]()

    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(max(3, args.warmup)):
        for r in range(ROT):
            for name, *_ in OPS:
                calls_r[name][r]()
    torch.cuda.synchronize()
    assert all(dc.query_status(w) == 0 for w in wss.values())
    # keep the device busy while the samplers start
    t_end = time.perf_counter() + args.busy_s
    while time.perf_counter() < t_end:
        for name, var, op, _, _ in OPS:
            call(name, var, op, outs[name])
        torch.cuda.synchronize()

    # steady state: K steps back to back on rotating buffers, one pair of events.  The
    # four calls of a step are independent images with workspaces of their own: each
    # runs on a side stream of its own (dc.CallStreams, forked from and joined back to
    # the timing stream), so that one call's pass fills the SMs another call leaves
    # idle between its passes.  The same steps on one stream give the serial figure.
    K = args.steps
    cs = dc.CallStreams(len(OPS), device=dev)

    def steps(concurrent: bool) -> tuple[float, int]:
        n_launch = 0
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        torch.cuda._sleep(20_000_000)  # let the host queue run ahead of the device
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if concurrent:
            cs.fork(stream)
        for k in range(K):
            r = k % ROT
            for j, (name, *_) in enumerate(OPS):
                if concurrent:
                    cs.run(j, calls_r[name][r])
                else:
                    calls_r[name][r]()
                n_launch += dc.last_launch_count()
        if concurrent:
            cs.join(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        return e0.elapsed_time(e1) / K, n_launch

    serial_step_ms, _ = steps(False)
    step_ms, launches = steps(True)

    # per call, for the roofline and the breakdown: L2 flushed (256 MiB write) before
    # each call, the call alone between two events
    KC = min(K, 200)
    ev = {name: [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(KC)]
          for name, *_ in OPS}
    for k in range(KC):
        if k % HOST_AHEAD_ROUNDS == 0:
            torch.cuda._sleep(SLEEP_CYCLES)
        for name, var, op, _, _ in OPS:
            flush.fill_(k & 0xFF)
            s0, s1 = ev[name][k]
            s0.record(stream)
            call(name, var, op, outs[name])
            s1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    op_ms = {name: float(np.mean([a.elapsed_time(b) for a, b in ev[name]])) for name, *_ in OPS}
    assert all(dc.query_status(w) == 0 for w in wss.values())
    # warm L2: each call repeated on its own buffers, the host enqueueing ahead: the
    # 8-bit calls' input, plane and output (66 MB) stay in L2
    warm_ms = {}
    for name, *_ in OPS:
        calls[name]()
        warm_ms[name] = _alone_ms([lambda k, c=calls[name]: c()], None, 50)[0]

    # per pass, in the stream (after the timed region): the library's profile mode
    # stamps each pass's first tile start and last tile end with the GPU global timer;
    # median of 7 calls, each after the L2-flushing write
    per_pass = {}
    dc.debug_profile(True)
    try:
        for name, var, op, _, _ in OPS:
            durs = []
            for rep in range(7):
                flush.fill_(rep)
                calls[name]()
                prof = dc.read_profile(calls[name], 1)
                durs.append([(b - a) / 1e3 for a, b in (q for q in prof["images"][0] if q)])
            us = [round(float(v), 2) for v in np.median(np.array(durs), axis=0)]
            kinds = PASSES[(var, op)]
            in_bytes = imgs[var].nbytes
            per_pass[name] = {"passes": kinds, "us": us,
                              "first_pass_input_GBps": round(in_bytes / (us[0] * 1e-6) / 1e9, 1)}
    finally:
        dc.debug_profile(False)

    def reduce_max(v):
        if world == 1:
            return v
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    t_max, gpix = aggregate(step_ms, world, reduce_max)
    serial_t_max, _ = aggregate(serial_step_ms, world, reduce_max)

    # end to end through the public API with pinned host buffers: every step copies
    # both inputs in and all four outputs out.  Steps one after another on one stream
    # (serial), and pipelined (HostPipeline: one step's input copy, the previous
    # step's calls and the one before's output copy overlap on three streams)
    from paper_2108_13656_gb300.pipeline import HostPipeline
    hx = {k: torch.from_numpy(v).pin_memory() for k, v in imgs.items()}
    hy = {name: torch.empty(outs[name].shape, dtype=outs[name].dtype).pin_memory() for name in outs}
    h2d = sum(t.numel() * t.element_size() for t in hx.values())
    d2h = sum(t.numel() * t.element_size() for t in hy.values())
    E = max(3, args.e2e_steps)
    for it in range(2 + E):
        if it == 2:
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        for k in x:
            x[k].copy_(hx[k], non_blocking=True)
        for name, var, op, _, _ in OPS:
            call(name, var, op, outs[name])
        for name in outs:
            hy[name].copy_(outs[name], non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    serial_ms = reduce_max(e0.elapsed_time(e1) / E)
    pipe = HostPipeline(hx, hy, [(op, var, name, {"mode": "sigmoid"} if op == "global" else {})
                                 for name, var, op, _, _ in OPS], depth=2, device=dev)
    for _ in range(3):
        pipe.submit(hx, hy)
    pipe.synchronize()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(pipe.s_in)
    for _ in range(E):
        pipe.submit(hx, hy)
    e1.record(pipe.s_out)
    torch.cuda.synchronize()
    e2e_ms = reduce_max(e0.elapsed_time(e1) / E)
    e2e_val = world * 4 * NPIX / (e2e_ms * 1e-3) / 1e9
    assert all(dc.query_status(w) == 0 for w in pipe.workspaces)

    if world > 1:
        torch.distributed.destroy_process_group()
    if rank != 0:
        return 0

    peak, peak_kind = measured_peak()
    dom = max(op_ms, key=op_ms.get)
    bpp = {name: b for name, _, _, _, b in OPS}[dom]
    achieved = bpp * NPIX / (op_ms[dom] * 1e-3) / 1e9
    traffic = ncu_traffic(dom)
    per_op = {name: {"ms": op_ms[name],
                     "GBps": {n: b for n, _, _, _, b in OPS}[name] * NPIX / (op_ms[name] * 1e-3) / 1e9,
                     "frac_of_measured_hbm": {n: b for n, _, _, _, b in OPS}[name] * NPIX / (op_ms[name] * 1e-3) / 1e9 / peak,
                     "warm_l2_ms": warm_ms[name]}
              for name in op_ms}
    line = {
        "metric": METRIC, "value": gpix, "unit": "Gpix/s", "n_gpus": world, "steps": K,
        "warmup": max(3, args.warmup), "ms_per_step": t_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "pixels_per_step": 4 * NPIX,
                   "l2": "value: steps back to back over %d rotating input/output sets (%.2f GB, far above L2); "
                         "per_op and roofline: each call alone after a 256 MiB L2-flushing write "
                         "(per_op warm_l2_ms: repeated on its own buffers, L2 warm)" % (
                             ROT, ROT * (sum(v.nbytes for v in imgs.values()) +
                                         sum(t.numel() * t.element_size() for t in outs.values())) / 1e9),
                   "per_op_sum_ms": sum(op_ms.values()),
                   "streams": "the four calls of a step on four side streams (CallStreams)",
                   "serial_ms_per_step": serial_t_max,
                   "serial_value": world * 4 * NPIX / (serial_t_max * 1e-3) / 1e9,
                   "parallelism": "replicas" if world > 1 else "single GPU", "per_op": per_op,
                   "per_pass": per_pass},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                     "algorithmic_bytes_per_launch": bpp * NPIX},
        "e2e": {"value": e2e_val, "unit": "Gpix/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_ms, "form": "pipelined over 3 streams, 2 device buffer sets",
                "serial_ms_per_step": serial_ms, "serial_value": world * 4 * NPIX / (serial_ms * 1e-3) / 1e9},
        "clocks": clk,
        "gpu_launches": launches,
    }
    iss = issue_roofline(op_ms, (clk or {}).get("sm_mhz") or 0.0,
                         torch.cuda.get_device_properties(dev).multi_processor_count)
    if iss:
        line["issue_roofline"] = iss
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(imgs)
    if not args.no_extras:
        line["decolorize_512"] = decolorize_512(dev)
        line["ragged_batch"] = ragged_batch(dev, args.ragged_images, peak)
        torch.cuda.empty_cache()
        line["precision_8k_local"] = precision_8k(dev, peak)
        torch.cuda.empty_cache()
        line["video_4k"] = video_4k(dev, peak)
        line["color_4k"] = color_4k(dev, peak)
        torch.cuda.empty_cache()
        line["serving"] = serving(dev, args.serve_requests, args.serve_rate)
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
