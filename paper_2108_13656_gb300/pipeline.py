"""Host-to-host pipelining: the copies and calls of consecutive steps overlapped.

A step takes host images (pinned memory), copies them to the device, runs a fixed
list of ABI calls on them and copies the outputs back to host buffers.
`HostPipeline` keeps `depth` device copies of every input and output and three CUDA
streams - host to device, calls, device to host - so that one step's input copy,
the previous step's calls and the one before's output copy run at the same time.
The dependencies are CUDA events: a device input is refilled only after the calls
of the step that used it `depth` steps earlier have finished, and a device output is
rewritten only after that step's output copy has finished.  Every step therefore
gives exactly what it gives when the steps run one after another.

Host buffers: a step's host inputs are read by its input copy, which runs after
`submit` returns, so they must not change until `input_consumed(step)` is true (or
the pipeline is synchronised); its host outputs are complete once `done(step)` is.

`CallStreams` runs independent calls (different images, different workspaces) on
streams of their own, so that the device works on one call while another is between
passes: a call's passes depend on the whole previous pass of that call, and the
launch, the ramp-up and the tail of each pass leave SMs idle that a concurrent
call's pass fills.
"""
from __future__ import annotations

from ._abi import PreparedCall, Workspace


class HostPipeline:
    """calls: list of (op, input name, output name, params) - op as for PreparedCall,
    params a dict of its keyword parameters.  inputs / outputs: name -> a tensor
    whose shape and dtype the device buffers take (host or device, any contents)."""

    def __init__(self, inputs: dict, outputs: dict, calls: list, depth: int = 2, device=None):
        import torch
        if depth < 1:
            raise ValueError("depth must be at least 1")
        dev = torch.device(device or "cuda")
        self.depth = depth
        self.s_in, self.s_run, self.s_out = (torch.cuda.Stream(device=dev) for _ in range(3))
        self.x = [{k: torch.empty(t.shape, dtype=t.dtype, device=dev) for k, t in inputs.items()}
                  for _ in range(depth)]
        self.y = [{k: torch.empty(t.shape, dtype=t.dtype, device=dev) for k, t in outputs.items()}
                  for _ in range(depth)]
        # one workspace per call position: the calls of all slots run in order on one stream
        wss = [Workspace(device=dev) for _ in calls]
        self.calls = [[PreparedCall(op, self.x[b][i], self.y[b][o], workspace=w, **dict(params or {}))
                       for (op, i, o, params), w in zip(calls, wss)] for b in range(depth)]
        self.workspaces = wss
        self.ev_in = [torch.cuda.Event() for _ in range(depth)]
        self.ev_run = [torch.cuda.Event() for _ in range(depth)]
        self.ev_out = [torch.cuda.Event() for _ in range(depth)]
        self.steps = 0
        self._ev_in_of, self._ev_out_of = {}, {}

    def submit(self, host_inputs: dict, host_outputs: dict) -> int:
        """Enqueue one step; returns its number."""
        import torch
        k, b = self.steps, self.steps % self.depth
        used = k >= self.depth  # slot b served step k - depth
        with torch.cuda.stream(self.s_in):
            if used:
                self.s_in.wait_event(self.ev_run[b])  # its calls have read x[b]
            for name, dst in self.x[b].items():
                dst.copy_(host_inputs[name], non_blocking=True)
            self.ev_in[b].record(self.s_in)
        with torch.cuda.stream(self.s_run):
            self.s_run.wait_event(self.ev_in[b])
            if used:
                self.s_run.wait_event(self.ev_out[b])  # its output copy has read y[b]
            for c in self.calls[b]:
                c(self.s_run)
            self.ev_run[b].record(self.s_run)
        with torch.cuda.stream(self.s_out):
            self.s_out.wait_event(self.ev_run[b])
            for name, src in self.y[b].items():
                host_outputs[name].copy_(src, non_blocking=True)
            self.ev_out[b].record(self.s_out)
        # per-step completion markers (the slot events are re-recorded later)
        ei, eo = torch.cuda.Event(), torch.cuda.Event()
        ei.record(self.s_in)
        eo.record(self.s_out)
        self._ev_in_of[k], self._ev_out_of[k] = ei, eo
        for old in [s for s in self._ev_in_of if s < k - 4 * self.depth]:
            del self._ev_in_of[old], self._ev_out_of[old]
        self.steps += 1
        return k

    def input_consumed(self, step: int) -> bool:
        e = self._ev_in_of.get(step)
        return e is None or e.query()

    def done(self, step: int) -> bool:
        e = self._ev_out_of.get(step)
        return e is None or e.query()

    def synchronize(self):
        for s in (self.s_in, self.s_run, self.s_out):
            s.synchronize()


class CallStreams:
    """n CUDA streams for independent calls.  `fork(stream)` makes every side stream
    wait for what `stream` (default: the current stream) has enqueued so far;
    `run(i, call)` enqueues `call` (anything called with a stream, e.g. a
    PreparedCall) on side stream i; `join(stream)` makes `stream` wait for everything
    enqueued on the side streams.  Calls on one side stream run in order; calls on
    different side streams may overlap, so they must not share a workspace or write
    a buffer another one reads - `run` refuses a workspace already used on another
    side stream since the last join (after a join, and a fork from the joined stream,
    every side stream's earlier work is ordered before the new calls)."""

    def __init__(self, n: int, device=None):
        import torch
        if n < 1:
            raise ValueError("need at least one stream")
        dev = torch.device(device or "cuda")
        self.streams = [torch.cuda.Stream(device=dev) for _ in range(n)]
        self._owner = {}

    def fork(self, stream=None):
        import torch
        src = stream or torch.cuda.current_stream()
        ev = torch.cuda.Event()
        ev.record(src)
        for s in self.streams:
            s.wait_event(ev)

    def run(self, i: int, call):
        ws = getattr(call, "ws_ptr", None)  # the device address of a PreparedCall's workspace
        if ws is not None:
            if self._owner.setdefault(ws, i) != i:
                raise ValueError("a workspace is in use on another side stream; give each stream its own")
        return call(self.streams[i])

    def join(self, stream=None):
        import torch
        dst = stream or torch.cuda.current_stream()
        for s in self.streams:
            ev = torch.cuda.Event()
            ev.record(s)
            dst.wait_event(ev)
        self._owner = {}
