"""Engine behaviour on the GPU: status word and workspace reuse, launch-shape
invariance, launch counts and CUDA-graph capture."""
import numpy as np
import pytest

from _cmp import check_f32
from _dev import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2108_13656_gb300 as m
    m.load()
    return m


def test_status_word_and_workspace_reuse(dc, oracle_mod):
    """The workspace's error word stays clear and a reused workspace gives the same
    result on a different image size (every call resets what it uses)."""
    import torch
    from paper_2108_13656_gb300 import synth
    ws = dc.Workspace()
    for (W, H, seed) in [(256, 128, 1), (97, 301, 2), (256, 128, 1)]:
        img = synth.s_ldr(W, H, seed=seed)
        y = torch.zeros((H, W), dtype=torch.float32, device="cuda")
        dc.decolorize_tonemap_global(to_dev(img), y, workspace=ws)
        assert dc.query_status(ws) == 0
        y64, _ = oracle_mod.tonemap_global_plane(oracle_mod.decolorize(img), ldr=True)
        check_f32(y.cpu().numpy(), y64, what="workspace reuse %dx%d" % (W, H))


@pytest.mark.parametrize("op", ["decolorize", "global", "histeq", "local"])
@pytest.mark.parametrize("in_dt", [np.uint8, np.float32])
def test_results_independent_of_launch_shape(dc, op, in_dt):
    """Tile shape (fixed, or sized per call) and CTAs per SM change neither the bits of
    the output nor the stats."""
    import torch
    from paper_2108_13656_gb300 import synth
    img = synth.s_ldr(1000, 700, 3) if in_dt == np.uint8 else synth.s_hdr(1000, 700, 3)
    x = to_dev(img)
    dt_code = dc.DC_U8 if in_dt == np.uint8 else dc.DC_F32
    op_code = {"decolorize": dc.DC_OP_DECOLORIZE, "global": dc.DC_OP_GLOBAL, "histeq": dc.DC_OP_GLOBAL,
               "local": dc.DC_OP_LOCAL}[op]
    orig = dc.get_tuning(op_code, dt_code)
    results = []
    try:
        # tile width 0: sized per call (the local operator's balanced width)
        for (tr, tc, cps) in [(4, 4096, 0), (1, 16, 1), (7, 1040, 3), (64, 65536, 2), (2, 512, 0), (1, 0, 0)]:
            dc.set_tuning(op_code, dt_code, 256, tr, tc, cps)
            y = torch.empty((700, 1000), dtype=torch.float32, device="cuda")
            st = torch.zeros(dc.STATS_BYTES, dtype=torch.uint8, device="cuda")
            if op == "decolorize":
                dc.decolorize(x, y)
            elif op == "local":
                dc.decolorize_tonemap_local(x, y)
            else:
                dc.decolorize_tonemap_global(x, y, mode="sigmoid" if op == "global" else "histeq", stats=st)
            torch.cuda.synchronize()
            results.append((y.cpu(), st.cpu()))
    finally:
        dc.set_tuning(op_code, dt_code, *orig)
    for y, st in results[1:]:
        assert torch.equal(y, results[0][0])
        assert torch.equal(st, results[0][1])


def test_launch_counts(dc):
    import torch
    from paper_2108_13656_gb300 import synth
    a = to_dev(synth.s_ldr(64, 32, 1))
    b = to_dev(synth.s_ldr(32, 64, 2))
    c = to_dev(synth.s_hdr(48, 16, 3))
    outs = [torch.empty((32, 64), device="cuda"), torch.empty((64, 32), device="cuda"),
            torch.empty((16, 48), device="cuda")]
    dc.decolorize_tonemap_global([a, b], outs[:2])
    assert dc.last_launch_count() == 2  # stats pass + curve pass, whole batch in each
    dc.decolorize_tonemap_global([a, b, c], outs)
    assert dc.last_launch_count() == 4  # the same per input sample type
    dc.decolorize_tonemap_local([a, b], outs[:2])
    assert dc.last_launch_count() == 3  # block histograms, window CDFs, apply (8-bit input)
    dc.decolorize([a, b, c], outs)
    assert dc.last_launch_count() == 2


def test_cuda_graph_capture_matches_eager(dc):
    import torch
    from paper_2108_13656_gb300 import synth
    imgs = [synth.s_ldr(640, 480, i) for i in range(4)]
    xs = [to_dev(im) for im in imgs]
    eager = [torch.empty((480, 640), dtype=torch.uint8, device="cuda") for _ in imgs]
    outs = [torch.empty_like(e) for e in eager]
    ws = dc.Workspace()
    dc.decolorize_tonemap_global(xs, eager, workspace=ws)  # sizes the workspace
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            dc.decolorize_tonemap_global(xs, outs, workspace=ws)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    for e, o in zip(eager, outs):
        assert torch.equal(e, o)


@pytest.mark.parametrize("op", ["global", "histeq", "local"])
def test_u8_plane_changes_no_result(dc, op):
    """8-bit input: a workspace with the optional luminance plane and the minimum
    workspace (Eq. 1-6 recomputed in every pass) give the same bits."""
    import torch
    from paper_2108_13656_gb300 import synth
    img = synth.s_ldr(1021, 347, 12)
    x = to_dev(img)
    code = dc.DC_OP_LOCAL if op == "local" else dc.DC_OP_GLOBAL
    lp = dc.local_params() if op == "local" else None
    full = dc.workspace_bytes(code, x, lp)
    least = dc.workspace_bytes(code, x, lp, minimum=True)
    assert full >= least + 1021 * 347 * 4
    ys = []
    for nbytes in (full, least):
        ws = dc.Workspace(nbytes=nbytes)  # exactly this many bytes
        y = torch.empty((347, 1021), dtype=torch.float32, device="cuda")
        st = torch.zeros(dc.STATS_BYTES, dtype=torch.uint8, device="cuda")
        if op == "local":
            dc.decolorize_tonemap_local(x, y, workspace=ws)
        else:
            dc.decolorize_tonemap_global(x, y, mode="sigmoid" if op == "global" else "histeq", stats=st, workspace=ws)
        torch.cuda.synchronize()
        assert dc.query_status(ws) == 0
        ys.append((y.cpu(), st.cpu()))
    assert torch.equal(ys[0][0], ys[1][0])
    assert torch.equal(ys[0][1], ys[1][1])


class _RawWorkspace:
    """A plain device buffer that is not registered with dc_workspace_prepare (every
    call clears its control block with a memset first)."""

    def __init__(self, nbytes):
        import torch
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")

    def get(self, nbytes):
        assert nbytes <= self.buf.numel()
        return self.buf.data_ptr(), self.buf.numel()


def test_registered_workspace_stays_clean(dc):
    """Calls on a registered workspace skip the clearing memset when the previous call
    left their control block zero, and clear it again at the end.  A sequence that
    changes sizes, batch sizes (a larger control block over a previous call's planes
    and histograms), operations, sample types, and has a profiled call in between
    gives the same bits and statistics as the same calls on an unregistered buffer."""
    import torch
    from paper_2108_13656_gb300 import synth
    small = [synth.s_ldr(64 + 7 * i, 40 + 3 * i, 60 + i) for i in range(20)]
    seq = [("local", [synth.s_ldr(700, 300, 6)], None),          # planes and histograms after a small block
           ("global", small, "sigmoid"),                           # 20 images: a larger control block
           ("global", [synth.s_ldr(640, 480, 1)], "sigmoid"),
           ("local", [synth.s_hdr(500, 300, 2)], None),
           ("global", [synth.s_hdr(333, 222, 3).astype(np.float16)], "histeq"),
           ("global", [synth.s_ldr(97, 61, 4)], "histeq"),          # profiled on the registered workspace
           ("decolorize", [synth.s_ldr(128, 64, 5)], None),
           ("global", small[:5] + [synth.s_hdr(90, 70, 7)], "histeq"),
           ("global", [synth.s_ldr(640, 480, 1)], "sigmoid")]
    reg = dc.Workspace()
    raw = _RawWorkspace(96 << 20)
    for i, (op, imgs, mode) in enumerate(seq):
        xs = [to_dev(im) for im in imgs]
        res = []
        for ws in (reg, raw):
            ys = [torch.empty(im.shape[:2], dtype=torch.float32, device="cuda") for im in imgs]
            st = torch.zeros(dc.STATS_BYTES * len(imgs), dtype=torch.uint8, device="cuda")
            if i == 5 and ws is reg:
                dc.debug_profile(True)  # this call leaves its counters for reading
            try:
                if op == "global":
                    dc.PreparedCall(op, xs, ys, mode=mode, stats=st, workspace=ws)()
                else:
                    dc.PreparedCall(op, xs, ys, workspace=ws)()
            finally:
                dc.debug_profile(False)
            torch.cuda.synchronize()
            res.append(([y.cpu() for y in ys], st.cpu()))
        for a, b in zip(res[0][0], res[1][0]):
            assert torch.equal(a, b), "call %d (%s) differs" % (i, op)
        assert torch.equal(res[0][1], res[1][1]), "call %d (%s) statistics differ" % (i, op)
    assert dc.query_status(reg) == 0


@pytest.mark.parametrize("mode", ["sigmoid", "histeq"])
@pytest.mark.parametrize("in_dt", [np.uint8, np.float16, np.float32])
def test_stats_record_changes_no_output(dc, mode, in_dt):
    """Without a stats record the statistics pass keeps only the reduction the curve
    uses (a different kernel variant); the output bits are the same as with one."""
    import torch
    from paper_2108_13656_gb300 import synth
    img = synth.s_ldr(517, 389, 8) if in_dt == np.uint8 else synth.s_hdr(517, 389, 8).astype(in_dt)
    x = to_dev(img)
    y0 = torch.empty((389, 517), dtype=torch.float32, device="cuda")
    y1 = torch.empty_like(y0)
    st = torch.zeros(dc.STATS_BYTES, dtype=torch.uint8, device="cuda")
    dc.decolorize_tonemap_global(x, y0, mode=mode)
    dc.decolorize_tonemap_global(x, y1, mode=mode, stats=st)
    torch.cuda.synchronize()
    assert torch.equal(y0, y1)
    rec = dc.parse_stats(st, 1)[0]
    assert rec["lmin"] <= rec["mu"] <= rec["lmax"]
