"""Ragged batches: one call per batch, captured into a CUDA graph.

A call of the C ABI takes a whole ragged batch (images of different sizes, strides
and sample types) and runs each pass of the operation as one persistent launch over
the tiles of every image.  `GraphCall` captures such a call once and replays it with
a single graph launch: the descriptors, the workspace and the launch shapes (the
tuning table at capture time) are frozen into the graph, so a replay costs no host
work beyond `cudaGraphLaunch`.  Inputs and outputs must stay at the same addresses;
their contents may change between replays.
"""
from __future__ import annotations

from ._abi import PreparedCall, Workspace


class GraphCall:
    """A prepared ABI call (see PreparedCall for the arguments) captured into a CUDA
    graph.  `replay()` enqueues every pass of the call on the current stream."""

    def __init__(self, op: str, inputs, outputs, workspace: Workspace | None = None, **params):
        import torch
        self.workspace = workspace or Workspace()
        self.call = PreparedCall(op, inputs, outputs, workspace=self.workspace, **params)
        self.launches = 0
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.call()  # eager run first: the capture then records a warmed-up call
            from ._abi import last_launch_count
            self.launches = last_launch_count()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, stream=side):
                self.call()
        torch.cuda.current_stream().wait_stream(side)

    def replay(self):
        self.graph.replay()
        return self.call.outputs


def plain_calls(op: str, inputs, outputs, **params) -> list[PreparedCall]:
    """One single-image call per image (the per-image baseline of a batch), each with
    its own workspace."""
    return [PreparedCall(op, x, y, workspace=Workspace(), **params) for x, y in zip(inputs, outputs)]
