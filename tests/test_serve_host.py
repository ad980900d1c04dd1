"""Host logic of the serving loop (no GPU): the seeded Poisson trace and the memory
accounting."""
import numpy as np
import pytest

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


class _SimDevice:
    """A fake device for the scheduling loop: a batch completes a fixed time per
    pixel after its launch (streams in parallel); the clock is simulated."""

    def __init__(self, ns_per_px=0.05):
        self.t = 0.0
        self.ns_per_px = ns_per_px
        self.busy_until = {}
        self.launched = []

    def clock(self):
        return self.t

    def wait_until(self, t_abs):
        self.t = max(self.t, t_abs)

    def idle(self):
        self.t += 1e-5

    def launch(self, si, admitted):
        px = sum(r.size[0] * r.size[1] for r, _ in admitted)
        start = max(self.t, self.busy_until.get(si, 0.0))
        self.busy_until[si] = start + px * self.ns_per_px * 1e-9
        self.launched.append([r.rid for r, _ in admitted])
        return self.busy_until[si]

    def done(self, h):
        return self.t >= h


def _trace_with_failures():
    tr = serve.make_trace(60, rate=4000.0, seed=11, sizes=((640, 480), (1280, 720)))
    big = serve.Request(1000, tr[5].t_arrive + 1e-6, "local", "f16", (7680, 4320), 0)   # larger than the budget
    tr.append(big)
    # a request that arrives behind a queue and is withdrawn 0.1 ms later
    tr[30].t_cancel = tr[30].t_arrive + 1e-4
    return tr, big


def test_oversize_request_is_rejected_and_the_loop_ends():
    tr, big = _trace_with_failures()
    budget = 3 * serve.request_bytes(serve.Request(0, 0.0, "local", "f16", (1280, 720), 0))
    adm = serve.Admission(budget, reserved_bytes=0, max_batch=8)
    assert serve.request_bytes(big) > adm.capacity
    dev = _SimDevice(ns_per_px=2.0)  # slow enough that requests queue behind the budget
    res = serve.schedule(tr, adm, 2, dev.launch, dev.done, lambda h: None, clock=dev.clock,
                         wait_until=dev.wait_until, idle=dev.idle)
    assert big.rid in adm.rejected and "budget" in adm.rejected[big.rid]
    assert adm.cancelled == {tr[30].rid}
    done = set(res["lat"])
    assert done == {r.rid for r in tr} - {big.rid, tr[30].rid}
    assert all(v >= 0 for v in res["lat"].values())
    assert adm.used == 0 and adm.peak <= adm.capacity
    # FIFO: launch order follows arrival order
    order = [rid for b in dev.launched for rid in b]
    arrivals = [r.rid for r in sorted(tr, key=lambda r: r.t_arrive) if r.rid in done]
    assert order == arrivals
    summ = serve._result(tr, res["lat"], res["queued"], res["batches"], adm.peak, None, adm.rejected,
                         adm.cancelled).summary()
    assert summ["rejected"] == 1 and summ["cancelled"] == 1 and summ["requests"] == len(tr) - 2


def test_cancel_only_while_waiting():
    adm = serve.Admission(100, max_batch=4)
    rs = [serve.Request(i, 0.0, "global", "u8", (4, 4), 0) for i in range(3)]
    assert all(adm.arrive(r, 40) for r in rs)
    got = adm.admit()
    assert [r.rid for r, _ in got] == [0, 1]          # the third does not fit yet
    assert not adm.cancel(0)                            # admitted: runs to completion
    assert adm.cancel(2) and adm.cancelled == {2}
    assert not adm.cancel(2)
    adm.release(80)
    assert adm.admit() == [] and adm.used == 0


def test_admission_counts_reserved_workspaces():
    with pytest.raises(ValueError):
        serve.Admission(4 << 30, reserved_bytes=4 << 30)
    adm = serve.Admission(16 << 30, reserved_bytes=4 * serve.WORKSPACE_BYTES)
    assert adm.capacity == (16 << 30) - 4 * (128 << 20)
    r = serve.Request(0, 0.0, "global", "u8", (4, 4), 0)
    assert not adm.arrive(r, adm.capacity + 1) and 0 in adm.rejected
    assert adm.arrive(serve.Request(1, 0.0, "global", "u8", (4, 4), 0), adm.capacity)


def test_inflight_cap_holds_arrivals_on_the_host():
    adm = serve.Admission(1000, max_batch=8, inflight_cap=100)
    rs = [serve.Request(i, 0.0, "global", "u8", (4, 4), 0) for i in range(4)]
    for r, n in zip(rs, (60, 30, 150, 20)):
        assert adm.arrive(r, n)
    assert [r.rid for r, _ in adm.admit()] == [0, 1]   # 90 of 100 in flight; the 150-byte one waits
    adm.release(90)
    assert [r.rid for r, _ in adm.admit()] == [2]      # idle: admitted alone although above the cap
    assert adm.admit() == []                            # FIFO: the 20-byte one waits behind it
    adm.release(150)
    assert [r.rid for r, _ in adm.admit()] == [3]
