"""Host-to-host pipeline: every step's outputs equal those of the same calls run
alone on that step's inputs, with the copies and calls of consecutive steps
overlapped (depths 1, 2 and 3, inputs changing from step to step, a distinct host
output set per step)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CALLS = [("global", "ldr", "g8", {"mode": "sigmoid"}),
         ("local", "ldr", "l8", {}),
         ("local", "hdr", "l32", {"block_s": 16, "bins": 24}),
         ("global", "hdr", "h32", {"mode": "histeq"})]


@pytest.fixture(scope="module")
def dc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2108_13656_gb300 as m
    m.load()
    return m


def host_inputs(step):
    import torch
    from paper_2108_13656_gb300 import synth
    ldr = synth.s_ldr(333, 197, 40 + step)
    hdr = synth.s_hdr(640, 360, 50 + step).astype(np.float16)
    return {"ldr": torch.from_numpy(ldr).pin_memory(), "hdr": torch.from_numpy(hdr).pin_memory()}


def host_outputs():
    import torch
    return {"g8": torch.empty((197, 333), dtype=torch.uint8).pin_memory(),
            "l8": torch.empty((197, 333), dtype=torch.uint8).pin_memory(),
            "l32": torch.empty((360, 640), dtype=torch.float32).pin_memory(),
            "h32": torch.empty((360, 640), dtype=torch.float32).pin_memory()}


def alone(dc, hx):
    import torch
    out = {}
    for op, i, o, params in CALLS:
        x = hx[i].cuda()
        y = torch.empty(hx[i].shape[:2], dtype=torch.uint8 if i == "ldr" else torch.float32, device="cuda")
        dc.PreparedCall(op, x, y, workspace=dc.Workspace(), **params)()
        out[o] = y
    torch.cuda.synchronize()
    return {k: v.cpu() for k, v in out.items()}


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_pipelined_steps_equal_calls_alone(dc, depth):
    import torch
    from paper_2108_13656_gb300.pipeline import HostPipeline
    inputs = [host_inputs(s) for s in range(3)]
    expect = [alone(dc, hx) for hx in inputs]
    pipe = HostPipeline(inputs[0], host_outputs(), CALLS, depth=depth)
    steps = []
    for k in range(8):
        hy = host_outputs()
        for t in hy.values():
            t.fill_(7)
        steps.append((pipe.submit(inputs[k % 3], hy), k % 3, hy))
    pipe.synchronize()
    for k, which, hy in steps:
        assert pipe.done(k) and pipe.input_consumed(k)
        for name, ref in expect[which].items():
            assert torch.equal(hy[name], ref), "step %d output %s differs from the call alone" % (k, name)
    assert all(dc.query_status(w) == 0 for w in pipe.workspaces)


def test_call_streams_equal_calls_alone(dc):
    # the four calls on four side streams, several steps over rotating inputs and
    # outputs without a join between steps: every output is the call's alone
    import torch
    inputs = [host_inputs(s) for s in range(3)]
    expect = [alone(dc, hx) for hx in inputs]
    dev_in = [{k: v.cuda() for k, v in hx.items()} for hx in inputs]
    wss = [dc.Workspace() for _ in CALLS]
    outs, calls = [], []
    for s in range(3):
        y = {o: torch.full(inputs[s][i].shape[:2], 7, dtype=torch.uint8 if i == "ldr" else torch.float32,
                           device="cuda") for op, i, o, params in CALLS}
        outs.append(y)
        calls.append([dc.PreparedCall(op, dev_in[s][i], y[o], workspace=w, **params)
                      for (op, i, o, params), w in zip(CALLS, wss)])
    cs = dc.CallStreams(len(CALLS))
    cs.fork()
    for k in range(9):
        for j, c in enumerate(calls[k % 3]):
            cs.run(j, c)
    cs.join()
    torch.cuda.synchronize()
    for s in range(3):
        for name, ref in expect[s].items():
            assert torch.equal(outs[s][name].cpu(), ref), "input set %d output %s differs from the call alone" % (s, name)
    assert all(dc.query_status(w) == 0 for w in wss)


def test_call_streams_refuse_a_shared_workspace(dc):
    import torch
    x = host_inputs(0)["ldr"].cuda()
    y = torch.empty(x.shape[:2], dtype=torch.uint8, device="cuda")
    w = dc.Workspace()
    a = dc.PreparedCall("global", x, y, workspace=w)
    cs = dc.CallStreams(2)
    cs.fork()
    cs.run(0, a)
    cs.run(0, a)  # the same stream: in order, allowed
    with pytest.raises(ValueError):
        cs.run(1, a)
    cs.join()
    cs.fork()  # after a join every earlier call is ordered before the new ones
    cs.run(1, a)
    cs.join()
    torch.cuda.synchronize()
    assert dc.query_status(w) == 0
