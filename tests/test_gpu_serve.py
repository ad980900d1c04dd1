"""Serving loop: every request's result is the same alone and in the mix (batched
with others, admitted under a tight memory budget, overlapped on several streams),
and the same as in the serial per-image baseline."""
import pytest

pytestmark = pytest.mark.gpu

SMALL_SIZES = ((320, 240), (640, 480), (1280, 720), (97, 61))


@pytest.fixture(scope="module")
def setup():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2108_13656_gb300 as m
    from paper_2108_13656_gb300 import serve
    m.load()
    trace = serve.make_trace(160, rate=20000.0, seed=5, sizes=SMALL_SIZES, variants=3)
    pool = serve.HostPool(trace)
    return m, serve, trace, pool


def alone(m, serve, pool, r):
    import torch
    hx = pool.host_input(r)
    x = hx.cuda()
    y = torch.empty(hx.shape[:2], dtype=serve.out_dtype(r), device="cuda")
    m.PreparedCall(r.op, x, y, workspace=m.Workspace())()
    torch.cuda.synchronize()
    return y.cpu()


def test_alone_equals_in_mix(setup):
    import torch
    m, serve, trace, pool = setup
    res = serve.serve_batched(trace, pool, keep_outputs=True)
    assert res.batches < len(trace)  # requests were batched together
    assert len(res.latency_s) == len(trace) and (res.latency_s > 0).all()
    for r in trace:
        assert torch.equal(res.outputs[r.rid], alone(m, serve, pool, r)), "request %d differs in the mix" % r.rid


def test_tight_budget_admits_in_order_and_matches(setup):
    import torch
    m, serve, trace, pool = setup
    budget = 2 * (serve.WORKSPACE_BYTES + 4096) + 3 * max(serve.request_bytes(r) for r in trace)  # 2 workspaces + 3 requests
    res = serve.serve_batched(trace[:60], pool, budget_bytes=budget, n_streams=2, keep_outputs=True)
    assert res.max_inflight_bytes <= budget
    for r in trace[:60]:
        assert torch.equal(res.outputs[r.rid], alone(m, serve, pool, r))


def test_serial_baseline_matches(setup):
    import torch
    m, serve, trace, pool = setup
    a = serve.serve_serial(trace[:40], pool, keep_outputs=True)
    b = serve.serve_batched(trace[:40], pool, keep_outputs=True)
    for r in trace[:40]:
        assert torch.equal(a.outputs[r.rid], b.outputs[r.rid])
    s = a.summary()
    assert s["p99_ms"] >= s["p50_ms"] > 0
