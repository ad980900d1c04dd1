"""Serving loop: decolorize + tone-map requests with continuous batching.

Requests (an image in pinned host memory, an operation, a sample type) arrive on a
trace.  The loop admits every request that has arrived as soon as the device-memory
budget has room for its input, output and tables, FIFO; admitted requests are
launched in batches - one C-ABI call per operation for everything admitted since
the last launch, on the least loaded of a few CUDA streams, each with its own
workspace - with the host->device copies, the call and the device->host copies
stream-ordered.  So requests that arrive while others run are admitted as memory
frees up and their copies and kernels overlap with the work already on the device.
A request completes when the host sees the event recorded after its batch's copies;
its latency is completion minus arrival.  `serve_serial` runs the same trace one
request at a time with a single-image call, the per-image baseline.

Every step on the device is a library call or a copy; the Python here only
schedules.
"""
from __future__ import annotations

import collections
import dataclasses
import gc
import time

import numpy as np

from . import _abi, synth

SERVE_SIZES = ((1280, 720), (1920, 1080), (3840, 2160), (7680, 4320))


@dataclasses.dataclass
class Request:
    rid: int
    t_arrive: float  # seconds after the start of the trace
    op: str          # "global" or "local"
    dtype: str       # "u8" (sRGB, output u8) or "f16" (linear HDR, output f32)
    size: tuple      # (width, height)
    variant: int     # which pooled image of that size and type
    t_cancel: float | None = None  # the client withdraws the request at this time (if still waiting)


class Admission:
    """FIFO admission of requests against a device-memory budget (host logic only).

    `capacity` = budget minus what the server holds for itself (its per-stream
    workspaces).  A request whose own bytes exceed the capacity can never be admitted:
    it is rejected when it arrives, so it cannot block the requests behind it.  A
    waiting request can be cancelled; once admitted its work is on the device and it
    completes normally."""

    def __init__(self, budget_bytes: int, reserved_bytes: int = 0, max_batch: int = 64, inflight_cap: int | None = None):
        self.capacity = int(budget_bytes) - int(reserved_bytes)
        if self.capacity <= 0:
            raise ValueError("the budget does not cover the server's own buffers")
        self.max_batch = max_batch
        # bytes in flight beyond which later arrivals wait on the host (FIFO) instead of
        # queueing on the device behind the copies already in flight; a request is always
        # admitted when nothing is in flight
        self.limit = self.capacity if inflight_cap is None else min(self.capacity, int(inflight_cap))
        self.waiting = collections.deque()  # (request, bytes)
        self.used = 0
        self.peak = 0
        self.rejected = {}       # rid -> reason
        self.cancelled = set()

    def arrive(self, r: Request, need: int) -> bool:
        if need > self.capacity:
            self.rejected[r.rid] = "needs %d bytes, more than the budget's %d" % (need, self.capacity)
            return False
        self.waiting.append((r, need))
        return True

    def cancel(self, rid: int) -> bool:
        """Withdraw a waiting request; False if it is not waiting (admitted, done or unknown)."""
        for k, (r, _) in enumerate(self.waiting):
            if r.rid == rid:
                del self.waiting[k]
                self.cancelled.add(rid)
                return True
        return False

    def admit(self) -> list:
        """Requests that fit now, in arrival order, at most max_batch: [(request, bytes)]."""
        out = []
        while self.waiting and len(out) < self.max_batch:
            need = self.waiting[0][1]
            if self.used + need > self.limit and self.used > 0:
                break
            r, need = self.waiting.popleft()
            self.used += need
            out.append((r, need))
        self.peak = max(self.peak, self.used)
        return out

    def release(self, nbytes: int):
        self.used -= nbytes
        assert self.used >= 0


def make_trace(n: int, rate: float, seed: int, sizes=SERVE_SIZES, p_u8: float = 0.7, p_global: float = 0.5,
               variants: int = 2) -> list[Request]:
    """n requests with Poisson arrivals of mean `rate` per second (seeded)."""
    rng = synth.rng_for(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    size_idx = rng.integers(0, len(sizes), n)
    u8 = rng.random(n) < p_u8
    glob = rng.random(n) < p_global
    var = rng.integers(0, variants, n)
    return [Request(i, float(t[i]), "global" if glob[i] else "local", "u8" if u8[i] else "f16",
                    tuple(sizes[int(size_idx[i])]), int(var[i])) for i in range(n)]


class _BufPool:
    """Recycled buffers per (shape, dtype): pinned host memory, or device memory
    (allocating and pinning are slow and may synchronise the device, so the loop
    reuses what it allocated; a buffer goes back only after its batch completed)."""

    def __init__(self, device=None):
        self.device = device  # None: pinned host memory
        self.free = collections.defaultdict(list)

    def new(self, shape, dtype):
        import torch
        if self.device is None:
            return torch.empty(shape, dtype=dtype).pin_memory()
        return torch.empty(shape, dtype=dtype, device=self.device)

    def get(self, shape, dtype):
        lst = self.free[(tuple(shape), dtype)]
        return lst.pop() if lst else self.new(tuple(shape), dtype)

    def put(self, t):
        self.free[(tuple(t.shape), t.dtype)].append(t)


class HostPool:
    """Pinned host images, one per (size, sample type, variant) of a trace: S-LDR for
    u8, S-HDR (5 decades) stored as binary16 for f16; variants are cyclic shifts.
    Also the reusable buffers: pinned host outputs and device inputs and outputs,
    `buffers_per_class` of each per (size, sample type) allocated up front (more
    are added on demand)."""

    def __init__(self, trace, seed: int = 5, buffers_per_class: int = 12, device=None):
        import torch
        self.images = {}
        self.outpool = _BufPool()
        self.devpool = _BufPool(torch.device(device or "cuda"))
        keys = sorted({(r.size, r.dtype, r.variant) for r in trace})
        bases = {}
        for size, dt, var in keys:
            if (size, dt) not in bases:
                w, h = size
                base = synth.s_ldr(w, h, seed) if dt == "u8" else synth.s_hdr(w, h, seed).astype(np.float16)
                bases[(size, dt)] = base
            base = bases[(size, dt)]
            img = synth.shifted(base, (97 * var) % size[1], (389 * var) % size[0]) if var else base
            self.images[(size, dt, var)] = torch.from_numpy(np.ascontiguousarray(img)).pin_memory()
        for size, dt in sorted({(r.size, r.dtype) for r in trace}):
            odt = torch.uint8 if dt == "u8" else torch.float32
            idt = torch.uint8 if dt == "u8" else torch.float16
            for _ in range(buffers_per_class):
                self.outpool.put(self.outpool.new((size[1], size[0]), odt))
                self.devpool.put(self.devpool.new((size[1], size[0]), odt))
                self.devpool.put(self.devpool.new((size[1], size[0], 3), idt))

    def host_input(self, r: Request):
        return self.images[(r.size, r.dtype, r.variant)]


def out_dtype(r: Request):
    import torch
    return torch.uint8 if r.dtype == "u8" else torch.float32


def request_bytes(r: Request, lp=None) -> int:
    """Device bytes a request holds while admitted: input, output and its share of the
    local operator's tables."""
    w, h = r.size
    nbytes = w * h * (3 if r.dtype == "u8" else 6) + w * h * (1 if r.dtype == "u8" else 4)
    if r.op == "local":
        hb, wb = (h + 31) // 32, (w + 31) // 32
        nbytes += hb * wb * (32 * 8 + 33 * 4) + 4096
    return nbytes + 2048


@dataclasses.dataclass
class ServeResult:
    latency_s: np.ndarray      # per completed request, in request order
    makespan_s: float          # first arrival to last completion
    pixels: int                # of the completed requests
    batches: int
    max_inflight_bytes: int
    outputs: dict | None       # rid -> host tensor, when kept
    sizes: list | None = None  # per completed request (width, height), in request order
    queue_s: np.ndarray | None = None  # per completed request: arrival to launch of its batch
    rejected: dict = dataclasses.field(default_factory=dict)  # rid -> reason (larger than the budget)
    cancelled: list = dataclasses.field(default_factory=list)  # rids withdrawn while waiting

    def summary(self) -> dict:
        lat = self.latency_s * 1e3
        if len(lat) == 0:
            return {"requests": 0, "rejected": len(self.rejected), "cancelled": len(self.cancelled)}
        out = {"requests": int(len(lat)), "rejected": len(self.rejected), "cancelled": len(self.cancelled),
               "p50_ms": float(np.percentile(lat, 50)),
               "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
               "gpix_s": self.pixels / self.makespan_s / 1e9, "makespan_s": self.makespan_s,
               "batches": self.batches, "max_inflight_gb": self.max_inflight_bytes / 1e9}
        if self.queue_s is not None:
            q = self.queue_s * 1e3
            out["queue_p50_ms"] = float(np.percentile(q, 50))
            out["queue_p99_ms"] = float(np.percentile(q, 99))
        out["p999_ms"] = float(np.percentile(lat, 99.9))
        out["max_ms"] = float(lat.max())
        if self.sizes:
            per = {}
            for sz in sorted(set(self.sizes)):
                m = np.array([q == sz for q in self.sizes])
                per["%dx%d" % sz] = {"p50_ms": float(np.percentile(lat[m], 50)),
                                     "p99_ms": float(np.percentile(lat[m], 99))}
            out["by_size"] = per
        return out


def _wait_until(t_abs: float):
    while True:
        d = t_abs - time.perf_counter()
        if d <= 0:
            return
        if d > 2e-4:
            time.sleep(d - 1e-4)


def schedule(trace, adm: Admission, n_streams: int, launch, done, retire, clock=time.perf_counter,
             wait_until=None, idle=None, bytes_fn=None) -> dict:
    """The continuous-batching loop, with the device side passed in.

    launch(si, admitted) enqueues one batch [(request, bytes)] on stream si and
    returns a handle; done(handle) says whether it has completed (a stream completes
    its batches in order, so only the oldest batch of each stream is polled);
    retire(handle) runs once per completed batch.  Arrivals are admitted through
    `adm` (oversize requests are rejected there), cancellations of waiting requests
    take effect at their t_cancel.  Returns per-request latencies and queueing times
    (completed requests only) and the number of batches."""
    wait_until = wait_until or _wait_until
    idle = idle or (lambda: time.sleep(2e-5))
    bytes_fn = bytes_fn or request_bytes
    pending = collections.deque(sorted(trace, key=lambda r: r.t_arrive))
    cancels = collections.deque(sorted((r.t_cancel, r.rid) for r in trace if r.t_cancel is not None))
    inflight = [collections.deque() for _ in range(n_streams)]
    lat, queued = {}, {}
    batches = 0
    t0 = clock()
    while pending or adm.waiting or any(inflight):
        now = clock() - t0
        while pending and pending[0].t_arrive <= now:
            r = pending.popleft()
            adm.arrive(r, bytes_fn(r))
        while cancels and cancels[0][0] <= now:
            adm.cancel(cancels.popleft()[1])
        for q in inflight:
            while q and done(q[0][0]):
                h, items, nbytes = q.popleft()
                t_done = clock() - t0
                for r, _ in items:
                    lat[r.rid] = t_done - r.t_arrive
                retire(h)
                adm.release(nbytes)
        admitted = adm.admit()
        if admitted:
            t_launch = clock() - t0
            for r, _ in admitted:
                queued[r.rid] = t_launch - r.t_arrive
            si = min(range(n_streams), key=lambda k: len(inflight[k]))
            inflight[si].append((launch(si, admitted), admitted, sum(n for _, n in admitted)))
            batches += 1
            continue
        # nothing to launch: wait for the next arrival or completion
        if pending and not any(inflight) and not adm.waiting:
            wait_until(t0 + pending[0].t_arrive)
        else:
            idle()
    return {"lat": lat, "queued": queued, "batches": batches}


def _result(trace, lat, queued, batches, peak, outputs, rejected, cancelled) -> "ServeResult":
    done = sorted((r for r in trace if r.rid in lat), key=lambda r: r.rid)
    makespan = (max(r.t_arrive + lat[r.rid] for r in done) - min(r.t_arrive for r in done)) if done else 0.0
    return ServeResult(np.array([lat[r.rid] for r in done]), makespan, sum(r.size[0] * r.size[1] for r in done),
                       batches, peak, outputs, [r.size for r in done], np.array([queued[r.rid] for r in done]),
                       dict(rejected), sorted(cancelled))


WORKSPACE_BYTES = 128 << 20  # per stream, sized up front


INFLIGHT_CAP_BYTES = 1 << 30  # about 5 ms of the host link's traffic


def serve_batched(trace, pool: HostPool, budget_bytes: int = 16 << 30, n_streams: int = 4, max_batch: int = 64,
                  keep_outputs: bool = False, device=None, inflight_cap: int | None = INFLIGHT_CAP_BYTES) -> ServeResult:
    """Continuous batching over the trace (arrival times are honoured in real time).
    The per-stream workspaces count against the budget; `inflight_cap` bounds the bytes
    in flight (None: only the budget)."""
    import torch
    dev = torch.device(device or "cuda")
    streams = [torch.cuda.Stream(device=dev) for _ in range(n_streams)]
    # sized up front and grown only when a batch's least need exceeds it (growing
    # inside the loop would allocate); the optional 8-bit plane is used while it fits
    wss = [_abi.Workspace(device=dev, optional=False) for _ in range(n_streams)]
    for w in wss:
        w.get(WORKSPACE_BYTES)
    adm = Admission(budget_bytes, reserved_bytes=sum(w.buf.numel() for w in wss), max_batch=max_batch,
                    inflight_cap=inflight_cap)
    outpool, devpool = pool.outpool, pool.devpool
    outputs = {} if keep_outputs else None

    def launch(si, admitted):
        s = streams[si]
        with torch.cuda.stream(s):
            items = []
            for r, _ in admitted:
                hx = pool.host_input(r)
                x = devpool.get(hx.shape, hx.dtype)
                x.copy_(hx, non_blocking=True)
                y = devpool.get(hx.shape[:2], out_dtype(r))
                items.append((r, x, y, outpool.get(tuple(hx.shape[:2]), out_dtype(r))))
            for op in ("global", "local"):
                sel = [(x, y) for r, x, y, _ in items if r.op == op]
                if sel:
                    _abi.PreparedCall(op, [a for a, _ in sel], [b for _, b in sel], workspace=wss[si])(s)
            for r, x, y, ho in items:
                ho.copy_(y, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        return ev, items

    def retire(h):
        for r, x, y, ho in h[1]:
            if keep_outputs:
                outputs[r.rid] = ho.clone()
            outpool.put(ho)
            devpool.put(x)
            devpool.put(y)

    torch.cuda.synchronize(dev)
    gc_was = gc.isenabled()
    gc.collect()
    gc.disable()  # a collection pause would stall every request in flight
    try:
        res = schedule(trace, adm, n_streams, launch, lambda h: h[0].query(), retire)
    finally:
        if gc_was:
            gc.enable()
    return _result(trace, res["lat"], res["queued"], res["batches"], adm.peak, outputs, adm.rejected,
                   adm.cancelled)


def serve_serial(trace, pool: HostPool, keep_outputs: bool = False, device=None) -> ServeResult:
    """The per-image baseline: each request in arrival order, alone, as a single-image
    call with its copies, synchronously."""
    import torch
    dev = torch.device(device or "cuda")
    ws = _abi.Workspace(device=dev)
    ws.get(128 << 20)
    outpool, devpool = pool.outpool, pool.devpool
    lat = {}
    outputs = {} if keep_outputs else None
    torch.cuda.synchronize(dev)
    gc_was = gc.isenabled()
    gc.collect()
    gc.disable()
    queued = {}
    t0 = time.perf_counter()
    cancelled = []
    for r in sorted(trace, key=lambda q: q.t_arrive):
        _wait_until(t0 + r.t_arrive)
        if r.t_cancel is not None and time.perf_counter() - t0 >= r.t_cancel:
            cancelled.append(r.rid)  # withdrawn before the server got to it
            continue
        queued[r.rid] = time.perf_counter() - t0 - r.t_arrive
        hx = pool.host_input(r)
        x = devpool.get(hx.shape, hx.dtype)
        x.copy_(hx, non_blocking=True)
        y = devpool.get(hx.shape[:2], out_dtype(r))
        _abi.PreparedCall(r.op, x, y, workspace=ws)()
        ho = outpool.get(tuple(hx.shape[:2]), out_dtype(r))
        ho.copy_(y, non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()
        devpool.put(x)
        devpool.put(y)
        lat[r.rid] = time.perf_counter() - t0 - r.t_arrive
        if keep_outputs:
            outputs[r.rid] = ho.clone()
        outpool.put(ho)
    if gc_was:
        gc.enable()
    return _result(trace, lat, queued, len(lat), 0, outputs, {}, cancelled)
