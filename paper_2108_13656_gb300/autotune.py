"""Autotuner for the launch shape of the pass kernels.

The knobs are those of `dc_set_tuning`: the tile width of the pixel passes (0 lets
the library size tiles per call; otherwise pixels per tile, i.e. tile_cols / 256
pixels per thread and tile) and the resident CTAs per SM; for the local operator the
tile width along a block row (0 lets the library pick the width whose tiles balance
best over the resident CTAs).  None of them changes a result (every reduction in the
library is exact integer arithmetic, and the test suite checks bitwise equality
across launch shapes), so the tuner only measures time.  Choices are cached in a
JSON file keyed by operation, input sample type, batch-size class, pixel-count class
and GPU name; the file is $DC_TUNE_CACHE or ~/.cache/decolor_gb300/tune.json.
"""
from __future__ import annotations

import json
import os
import threading

from . import _abi

GLOBAL_CANDIDATES = [(0, 0), (0, 2), (0, 3), (2048, 0), (8192, 0), (32768, 0), (131072, 0), (8192, 2)]
LOCAL_CANDIDATES = [(0, 0), (128, 0), (256, 0), (512, 0), (1024, 0), (256, 2), (256, 3)]
OP_CODES = {"decolorize": _abi.DC_OP_DECOLORIZE, "global": _abi.DC_OP_GLOBAL, "local": _abi.DC_OP_LOCAL}


def default_cache_path() -> str:
    return os.environ.get("DC_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "decolor_gb300",
                                                            "tune.json")


def size_class(n_images: int, total_pixels: int) -> str:
    """Batch-size class (1, 2-16, 17-256, more) and pixel-count class (power of 4)."""
    nb = "1" if n_images <= 1 else ("16" if n_images <= 16 else ("256" if n_images <= 256 else "many"))
    pc = (max(int(total_pixels), 1).bit_length() - 1) // 2  # floor(log4), exact
    return "n%s/p4^%d" % (nb, pc)


def tuning_key(op: str, in_dtype: int, n_images: int, total_pixels: int, device_name: str) -> str:
    return "%s/%d/%s/%s" % (op, in_dtype, size_class(n_images, total_pixels), device_name)


class TuneCache:
    """JSON cache of tuning choices (read once, written after every new entry)."""

    def __init__(self, path: str | None = None):
        self.path = path or default_cache_path()
        self.lock = threading.Lock()
        self.data = {}
        try:
            with open(self.path) as f:
                self.data = json.load(f)
        except (OSError, ValueError):
            self.data = {}

    def get(self, key: str):
        v = self.data.get(key)
        return None if v is None else tuple(v["choice"])

    def put(self, key: str, choice, timings: dict):
        with self.lock:
            self.data[key] = {"choice": list(choice), "us": timings}
            d = os.path.dirname(self.path)
            if d:
                os.makedirs(d, exist_ok=True)
            tmp = self.path + ".tmp%d" % os.getpid()
            with open(tmp, "w") as f:
                json.dump(self.data, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def apply_choice(op: str, in_dtype: int, choice) -> None:
    """Set the library's launch shape for (op, in_dtype) to a (tile_cols, ctas_per_sm) choice."""
    tile_cols, cps = choice
    if op == "local":
        _abi.set_tuning(OP_CODES[op], in_dtype, 256, 32, tile_cols, cps)
    else:
        _abi.set_tuning(OP_CODES[op], in_dtype, 256, 1, tile_cols, cps)


def _time_call(call, reps: int, flush) -> float:
    import torch
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.fill_(0)
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        call()
        e.record()
        torch.cuda.synchronize()
        ts.append(s.elapsed_time(e) * 1e3)
    ts.sort()
    return ts[len(ts) // 2]


class Autotuner:
    """Pick the fastest launch shape for a call by timing the candidates on the call's
    own inputs (CUDA events, L2 flushed before each timed call when `flush_l2`)."""

    def __init__(self, cache: TuneCache | None = None, reps: int = 5, flush_l2: bool = True):
        self.cache = cache or TuneCache()
        self.reps = reps
        self.flush_l2 = flush_l2

    def tune(self, op: str, inputs, outputs, workspace=None, force: bool = False, **params):
        """Return ((tile_cols, ctas_per_sm), timings) for this call and leave the library
        set to it.  All inputs must share one sample type."""
        import torch
        inputs = list(inputs) if isinstance(inputs, (list, tuple)) else [inputs]
        outputs = list(outputs) if isinstance(outputs, (list, tuple)) else [outputs]
        dts = {_abi.dtype_code(x) for x in inputs}
        if len(dts) != 1:
            raise ValueError("autotuning needs inputs of one sample type")
        dt = dts.pop()
        px = sum(int(x.shape[0]) * int(x.shape[1]) for x in inputs)
        key = tuning_key(op, dt, len(inputs), px, torch.cuda.get_device_name())
        hit = None if force else self.cache.get(key)
        if hit is not None:
            apply_choice(op, dt, hit)
            return hit, self.cache.data[key].get("us", {})
        orig = _abi.get_tuning(OP_CODES[op], dt)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=inputs[0].device) if self.flush_l2 else None
        ws = workspace or _abi.Workspace()
        timings = {}
        try:
            for cand in (LOCAL_CANDIDATES if op == "local" else GLOBAL_CANDIDATES):
                apply_choice(op, dt, cand)
                call = _abi.PreparedCall(op, inputs, outputs, workspace=ws, **params)
                call()
                timings["%d,%d" % cand] = _time_call(call, self.reps, flush)
        finally:
            _abi.set_tuning(OP_CODES[op], dt, *orig)
        best = min(timings, key=timings.get)
        choice = tuple(int(v) for v in best.split(","))
        self.cache.put(key, choice, timings)
        apply_choice(op, dt, choice)
        return choice, timings
