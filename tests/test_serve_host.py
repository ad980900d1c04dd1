"""Host logic of the serving loop (no GPU): the seeded Poisson trace and the memory
accounting."""
import numpy as np

from paper_2108_13656_gb300 import serve


def test_trace_statistics():
    tr = serve.make_trace(10000, rate=2000.0, seed=5)
    t = np.array([r.t_arrive for r in tr])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 2000.0) < 0.05 / 2000.0           # mean inter-arrival 0.5 ms
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05                # exponential: cv = 1
    assert abs(np.mean([r.dtype == "u8" for r in tr]) - 0.7) < 0.02
    assert abs(np.mean([r.op == "global" for r in tr]) - 0.5) < 0.02
    counts = {s: sum(r.size == s for r in tr) for s in serve.SERVE_SIZES}
    assert all(abs(c / len(tr) - 0.25) < 0.02 for c in counts.values())
    mean_px = np.mean([r.size[0] * r.size[1] for r in tr])
    assert abs(mean_px - 11.1e6) < 0.5e6


def test_trace_is_seeded():
    a = serve.make_trace(50, 1000.0, 7)
    b = serve.make_trace(50, 1000.0, 7)
    assert a == b
    assert a != serve.make_trace(50, 1000.0, 8)


def test_request_bytes():
    r = serve.Request(0, 0.0, "global", "u8", (1920, 1080), 0)
    assert serve.request_bytes(r) == 1920 * 1080 * 4 + 2048
    h = serve.Request(1, 0.0, "local", "f16", (7680, 4320), 0)
    n = serve.request_bytes(h)
    assert n > 7680 * 4320 * 10 and n < 7680 * 4320 * 10 + 16e6
