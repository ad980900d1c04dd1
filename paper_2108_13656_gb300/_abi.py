"""Thin ctypes binding of include/decolor.h (argument marshalling only).

Every step of the hot path runs inside libdecolor.so; this module converts torch
tensors into the ABI's plain descriptors (device pointers, sizes, strides, sample
types) and passes torch's current CUDA stream.  There is no fallback: when the
library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build_lib

DC_OK, DC_ERR_INVALID_ARG, DC_ERR_UNSUPPORTED_DTYPE, DC_ERR_WORKSPACE = 0, 1, 2, 3
DC_ERR_CUDA, DC_ERR_TIMEOUT, DC_ERR_TOO_MANY = 4, 5, 6
DC_U8, DC_F16, DC_F32 = 0, 1, 2
DC_OP_DECOLORIZE, DC_OP_GLOBAL, DC_OP_LOCAL = 0, 1, 2
DC_SIGMOID, DC_HISTEQ = 0, 1
DC_LUMA_OURS, DC_LUMA_Y, DC_LUMA_V, DC_LUMA_LSTAR = 0, 1, 2, 3
DC_PRESET_PAPER, DC_PRESET_TM1, DC_PRESET_TM2 = 0, 1, 2
BETA_R, BETA_K = 0.55, 0.8
LUMA = {"ours": DC_LUMA_OURS, "y": DC_LUMA_Y, "v": DC_LUMA_V, "lstar": DC_LUMA_LSTAR}
VIDEO_STATE_BYTES = 1056  # sizeof(dc_video_state)


class DcError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__("%s failed: %s (status %d)" % (what, status_string(status), status))
        self.status = status


class dc_image_in(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("stride_bytes", ctypes.c_int64), ("dtype", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class dc_image_out(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("stride_bytes", ctypes.c_int64), ("dtype", ctypes.c_int32),
                ("channels", ctypes.c_int32)]


class dc_decolor_params(ctypes.Structure):
    _fields_ = [("beta_r", ctypes.c_float), ("beta_k", ctypes.c_float), ("luma", ctypes.c_int32),
                ("color_s", ctypes.c_float)]

    def __init__(self, beta_r=0.55, beta_k=0.8, luma=0, color_s=1.0):
        super().__init__(beta_r, beta_k, luma, color_s)


class dc_video_state(ctypes.Structure):
    _fields_ = [("m", ctypes.c_float), ("mu_last", ctypes.c_float), ("frames", ctypes.c_int64),
                ("vmin", ctypes.c_int32), ("vmax", ctypes.c_int32), ("npix", ctypes.c_int64),
                ("hist", ctypes.c_uint32 * 256)]


class dc_global_params(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("gain_k", ctypes.c_float), ("delta", ctypes.c_float),
                ("reserved", ctypes.c_int32)]


class dc_local_params(ctypes.Structure):
    _fields_ = [("block_s", ctypes.c_int32), ("radius_blocks", ctypes.c_int32), ("bins", ctypes.c_int32),
                ("alpha", ctypes.c_float), ("delta", ctypes.c_float), ("reserved", ctypes.c_int32)]


class dc_tuning(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("tile_rows", ctypes.c_int32), ("tile_cols", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32)]


STATS_BYTES = 4 * 4 + 8 + 8 + 256 * 4  # sizeof(dc_global_stats)

# Every exported symbol of include/decolor.h with its ctypes signature.
_SIGS = {
    "dc_decolorize": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "dc_decolorize_tonemap_global": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                    ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "dc_decolorize_tonemap_local": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                   ctypes.c_size_t, ctypes.c_void_p]),
    "dc_decolorize_tonemap_global_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                            ctypes.c_void_p]),
    "dc_decolorize_tonemap_video": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float, ctypes.c_int32,
                                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                                   ctypes.c_void_p]),
    "dc_preset": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "dc_video_local_state_bytes": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "dc_decolorize_tonemap_local_video": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                                         ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                                         ctypes.c_size_t, ctypes.c_void_p]),
    "dc_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "dc_workspace_min_bytes": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "dc_workspace_prepare": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "dc_workspace_release": (ctypes.c_int, [ctypes.c_void_p]),
    "dc_query_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "dc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "dc_set_tuning": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]),
    "dc_get_tuning": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]),
    "dc_debug_profile": (ctypes.c_int, [ctypes.c_int32]),
    "dc_debug_read_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "dc_last_launch_count": (ctypes.c_int, []),
    "dc_debug_fail_launch": (ctypes.c_int, [ctypes.c_int32]),
    "dc_local_tile_cols": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]),
    "dc_debug_bounds": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "dc_version": (ctypes.c_int, []),
}

_lib = None
_lib_lock = threading.Lock()


def library_path() -> str:
    """The shared library the binding loads: $DC_LIBRARY if set, else the in-tree build."""
    return os.environ.get("DC_LIBRARY") or build_lib.LIB


def load(build_if_missing: bool = True):
    """Load libdecolor.so (building it first when allowed); raises when unavailable."""
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        path = os.environ.get("DC_LIBRARY") or build_lib.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError("libdecolor.so is not built (run __graft_entry__.build())")
            build_lib.build()
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def status_string(status: int) -> str:
    try:
        return load(build_if_missing=False).dc_status_string(int(status)).decode()
    except Exception:  # library not loadable: still give a message
        return "status %d" % status


# ------------------------------------------------------------ descriptors ----
def _torch():
    import torch
    return torch


def dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.uint8:
        return DC_U8
    if t.dtype == torch.float16:
        return DC_F16
    if t.dtype == torch.float32:
        return DC_F32
    raise TypeError("unsupported sample type %s (uint8, float16 or float32)" % t.dtype)


def _in_desc(t) -> dc_image_in:
    if t.dim() != 3 or t.shape[2] != 3:
        raise ValueError("input must be (H, W, 3) interleaved RGB, got %s" % (tuple(t.shape),))
    if t.stride(2) != 1 or t.stride(1) != 3:
        raise ValueError("input pixels must be interleaved (channel stride 1, pixel stride 3)")
    d = dc_image_in()
    d.data = t.data_ptr()
    d.height, d.width = int(t.shape[0]), int(t.shape[1])
    d.stride_bytes = int(t.stride(0)) * t.element_size()
    d.dtype = dtype_code(t)
    d.reserved = 0
    return d


def _out_desc(t) -> dc_image_out:
    """A (H, W) gray plane, or a (H, W, 3) interleaved colour output."""
    d = dc_image_out()
    if t.dim() == 3 and t.shape[2] == 3:
        if t.stride(2) != 1 or t.stride(1) != 3:
            raise ValueError("colour output pixels must be interleaved (channel stride 1, pixel stride 3)")
        d.channels = 3
    elif t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("output must be a (H, W) plane with unit column stride or (H, W, 3) interleaved")
    else:
        d.channels = 0
    d.data = t.data_ptr()
    d.stride_bytes = int(t.stride(0)) * t.element_size()
    d.dtype = dtype_code(t)
    return d


def _arrays(inputs, outputs):
    if len(inputs) == 0:
        raise ValueError("empty batch")
    ins = (dc_image_in * len(inputs))(*[_in_desc(t) for t in inputs])
    outs = None
    if outputs is not None:
        if len(outputs) != len(inputs):
            raise ValueError("inputs and outputs differ in length")
        for a, b in zip(inputs, outputs):
            if tuple(b.shape[:2]) != (a.shape[0], a.shape[1]):
                raise ValueError("output shape %s does not match input %s" % (tuple(b.shape), tuple(a.shape)))
        outs = (dc_image_out * len(outputs))(*[_out_desc(t) for t in outputs])
    return ins, outs


def _as_list(x):
    return list(x) if isinstance(x, (list, tuple)) else [x]


def _stream_handle(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Workspace:
    """Device workspace owned by torch's allocator (256-byte aligned): grown on demand
    to what each call asks for, or, when created with `nbytes`, exactly that size and
    never grown (a call then keeps its optional planes only if they fit).  With
    `optional=False` it grows only to a call's least need (dc_workspace_min_bytes),
    so that the optional 8-bit plane is used only while it fits the current size.
    Each buffer is registered with dc_workspace_prepare (calls keep its control block
    clean, no per-call clearing memset) and released before it is dropped."""

    def __init__(self, device=None, nbytes: int | None = None, optional: bool = True):
        self.device = device
        self.buf = None
        self.fixed = nbytes is not None
        self.optional = optional
        if self.fixed:
            self._set(_torch().empty(max(int(nbytes), 256), dtype=_torch().uint8, device=device or "cuda"))

    def _set(self, buf):
        lib = load()
        if self.buf is not None:
            _torch().cuda.synchronize(self.buf.device)  # calls on the old buffer end first
            lib.dc_workspace_release(ctypes.c_void_p(self.buf.data_ptr()))
        self.buf = buf
        with _torch().cuda.device(buf.device):
            rc = lib.dc_workspace_prepare(ctypes.c_void_p(buf.data_ptr()), buf.numel(), _stream_handle(None))
        if rc != DC_OK:
            raise DcError(rc, "dc_workspace_prepare")

    def get(self, nbytes: int, min_bytes: int | None = None):
        """The buffer for a call that asks for `nbytes` (and accepts `min_bytes`)."""
        torch = _torch()
        nbytes = max(int(nbytes), 256)
        if not self.optional and min_bytes is not None and self.buf is not None:
            nbytes = max(int(min_bytes), 256)
        if not self.fixed and (self.buf is None or self.buf.numel() < nbytes):
            self._set(torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device or "cuda"))
        ptr = self.buf.data_ptr()
        assert ptr % 256 == 0
        return ptr, self.buf.numel()

    def __del__(self):
        try:
            if self.buf is not None and _lib is not None:
                _lib.dc_workspace_release(ctypes.c_void_p(self.buf.data_ptr()))
        except Exception:
            pass


_default_ws: dict = {}


def _workspace(op, ins, n, lp, ws):
    lib = load()
    need = lib.dc_workspace_bytes(op, ins, n, ctypes.byref(lp) if lp is not None else None)
    if need == 0:
        raise DcError(DC_ERR_INVALID_ARG, "dc_workspace_bytes")
    if ws is None:
        torch = _torch()
        dev = torch.cuda.current_device()
        ws = _default_ws.setdefault(dev, Workspace(device="cuda:%d" % dev))
    least = None
    if not getattr(ws, "optional", True):  # (any object with get() serves as a workspace)
        least = lib.dc_workspace_min_bytes(op, ins, n, ctypes.byref(lp) if lp is not None else None)
    ptr, size = ws.get(need, least) if least is not None else ws.get(need)
    return ptr, size, ws.buf


# ------------------------------------------------------------------ calls ----
def local_params(block_s: int = 32, radius_blocks: int = 2, bins: int = 32, alpha: float = 1.0,
                 delta: float = 1e-4) -> dc_local_params:
    return dc_local_params(block_s, radius_blocks, bins, alpha, delta, 0)


class PreparedCall:
    """One ABI call with its descriptors, parameters and workspace resolved once.

    op is "decolorize", "global" or "local"; calling the object enqueues the call on
    `stream` (default: torch's current stream).  The tensors must stay alive and in
    place for as long as the object is used.
    """

    def __init__(self, op: str, inputs, outputs, beta_r: float = BETA_R, beta_k: float = BETA_K,
                 mode="sigmoid", gain_k: float = 1.0, delta: float = 1e-4, stats=None, block_s: int = 32,
                 radius_blocks: int = 2, bins: int = 32, alpha: float = 1.0, workspace=None, luma="ours",
                 color_s: float = 1.0):
        self.lib = load()
        self.inputs, self.outputs = _as_list(inputs), _as_list(outputs)
        self.n = len(self.inputs)
        self.ins, self.outs = _arrays(self.inputs, self.outputs)
        self.p = dc_decolor_params(beta_r, beta_k, LUMA.get(luma, luma), color_s)
        self.op = op
        self.stats = stats
        self.lp = None
        if op == "decolorize":
            code = DC_OP_DECOLORIZE
        elif op == "global":
            code = DC_OP_GLOBAL
            m = {"sigmoid": DC_SIGMOID, "histeq": DC_HISTEQ}.get(mode, mode)
            self.g = dc_global_params(int(m), gain_k, delta, 0)
            self.sp = None
            if stats is not None:
                if not stats.is_cuda or stats.numel() * stats.element_size() < STATS_BYTES * self.n:
                    raise ValueError("stats buffer must be a CUDA tensor of n * STATS_BYTES bytes")
                self.sp = ctypes.c_void_p(stats.data_ptr())
        elif op == "local":
            code = DC_OP_LOCAL
            self.lp = local_params(block_s, radius_blocks, bins, alpha, delta)
        else:
            raise ValueError("unknown op %r" % op)
        # keep the buffer itself: a later, larger request may replace the Workspace's buffer
        self.ws_ptr, self.ws_size, self.ws_buf = _workspace(code, self.ins, self.n, self.lp, workspace)
        self._ws = ctypes.c_void_p(self.ws_ptr)

    def __call__(self, stream=None):
        st = _stream_handle(stream)
        if self.op == "decolorize":
            rc = self.lib.dc_decolorize(self.ins, self.outs, self.n, ctypes.byref(self.p), self._ws,
                                        self.ws_size, st)
            name = "dc_decolorize"
        elif self.op == "global":
            rc = self.lib.dc_decolorize_tonemap_global(self.ins, self.outs, self.n, ctypes.byref(self.p),
                                                       ctypes.byref(self.g), self.sp, self._ws, self.ws_size, st)
            name = "dc_decolorize_tonemap_global"
        else:
            rc = self.lib.dc_decolorize_tonemap_local(self.ins, self.outs, self.n, ctypes.byref(self.p),
                                                      ctypes.byref(self.lp), self._ws, self.ws_size, st)
            name = "dc_decolorize_tonemap_local"
        if rc != DC_OK:
            raise DcError(rc, name)
        return self.outputs


def decolorize(inputs, outputs, beta_r: float = BETA_R, beta_k: float = BETA_K, workspace=None,
               stream=None, luma="ours"):
    """Eq. 1-6 (or the comparison channel `luma`: "ours", "y", "v") over a (ragged)
    batch: outputs[i] = L(inputs[i])."""
    return PreparedCall("decolorize", inputs, outputs, beta_r=beta_r, beta_k=beta_k,
                        workspace=workspace, luma=luma)(stream)


def decolorize_tonemap_global(inputs, outputs, mode: str | int = "sigmoid", gain_k: float = 1.0,
                              delta: float = 1e-4, stats=None, beta_r: float = BETA_R,
                              beta_k: float = BETA_K, workspace=None, stream=None, luma="ours",
                              color_s: float = 1.0):
    """Eq. 1-6 then the global curve; `stats` is None or a uint8 CUDA tensor of n*STATS_BYTES.
    An (H, W, 3) output receives the colour reconstruction (saturation exponent color_s)."""
    return PreparedCall("global", inputs, outputs, beta_r=beta_r, beta_k=beta_k, mode=mode, gain_k=gain_k,
                        delta=delta, stats=stats, workspace=workspace, luma=luma, color_s=color_s)(stream)


def decolorize_tonemap_local(inputs, outputs, block_s: int = 32, radius_blocks: int = 2, bins: int = 32,
                             alpha: float = 1.0, delta: float = 1e-4, beta_r: float = BETA_R,
                             beta_k: float = BETA_K, workspace=None, stream=None, luma="ours",
                             color_s: float = 1.0):
    """Eq. 1-6 then smoothed local-histogram equalisation (colour output as for the global call)."""
    return PreparedCall("local", inputs, outputs, beta_r=beta_r, beta_k=beta_k, block_s=block_s,
                        radius_blocks=radius_blocks, bins=bins, alpha=alpha, delta=delta,
                        workspace=workspace, luma=luma, color_s=color_s)(stream)


def preset(name) -> tuple[dc_decolor_params, dc_local_params]:
    """Parameter preset ("paper", "tm1" background boost, "tm2" background suppression)."""
    code = {"paper": DC_PRESET_PAPER, "tm1": DC_PRESET_TM1, "tm2": DC_PRESET_TM2}.get(name, name)
    p, lp = dc_decolor_params(), dc_local_params()
    rc = load().dc_preset(int(code), ctypes.byref(p), ctypes.byref(lp))
    if rc != DC_OK:
        raise DcError(rc, "dc_preset")
    return p, lp


class VideoStreams:
    """n video streams tone-mapped frame by frame with the carried log-mean estimate
    (dc_decolorize_tonemap_video): the first call (or one after restart()) centres each
    frame on its own log-mean, later calls take one pass per frame.  The per-stream
    state lives in a device tensor owned here."""

    def __init__(self, n: int, lam: float = 1.0, gain_k: float = 1.0, delta: float = 1e-4,
                 beta_r: float = BETA_R, beta_k: float = BETA_K, luma="ours", device=None, workspace=None,
                 mode="sigmoid"):
        torch = _torch()
        self.lib = load()
        self.n = int(n)
        self.lam = float(lam)
        self.state = torch.zeros(self.n * VIDEO_STATE_BYTES, dtype=torch.uint8, device=device or "cuda")
        self.p = dc_decolor_params(beta_r, beta_k, LUMA.get(luma, luma), 1.0)
        self.g = dc_global_params(int({"sigmoid": DC_SIGMOID, "histeq": DC_HISTEQ}.get(mode, mode)), gain_k, delta, 0)
        self.ws = workspace
        self._restart = True

    def restart(self):
        self._restart = True

    def prepare(self, frames, outputs):
        """The call for these frame and output buffers with descriptors and workspace
        resolved once: `call(restart=None, stream=None)` enqueues one frame per stream
        (restart None: as the streams' state requires)."""
        frames, outputs = _as_list(frames), _as_list(outputs)
        if len(frames) != self.n:
            raise ValueError("expected %d frames (one per stream)" % self.n)
        ins, outs = _arrays(frames, outputs)
        ptr, size, buf = _workspace(DC_OP_GLOBAL, ins, self.n, None, self.ws)
        ws, st = ctypes.c_void_p(ptr), ctypes.c_void_p(self.state.data_ptr())

        def call(restart=None, stream=None):
            r = self._restart if restart is None else bool(restart)
            rc = self.lib.dc_decolorize_tonemap_video(ins, outs, self.n, ctypes.byref(self.p), ctypes.byref(self.g),
                                                      self.lam, 1 if r else 0, st, ws, size, _stream_handle(stream))
            if rc != DC_OK:
                raise DcError(rc, "dc_decolorize_tonemap_video")
            self._restart = False
            return outputs

        call.keep = (frames, outputs, buf)  # the buffers stay alive with the call
        return call

    def __call__(self, frames, outputs, stream=None):
        return self.prepare(frames, outputs)(stream=stream)

    def states(self) -> list[dict]:
        raw = self.state.cpu().numpy().tobytes()
        out = []
        for i in range(self.n):
            r = dc_video_state.from_buffer_copy(raw[i * VIDEO_STATE_BYTES:(i + 1) * VIDEO_STATE_BYTES])
            out.append({"m": r.m, "mu_last": r.mu_last, "frames": int(r.frames), "vmin": r.vmin, "vmax": r.vmax,
                        "npix": int(r.npix), "hist": np.array(r.hist[:], dtype=np.uint32)})
        return out


def workspace_bytes(op: int, inputs, lparams: dc_local_params | None = None, minimum: bool = False) -> int:
    """dc_workspace_bytes (or dc_workspace_min_bytes with minimum=True) for these inputs."""
    inputs = _as_list(inputs)
    ins, _ = _arrays(inputs, None)
    fn = load().dc_workspace_min_bytes if minimum else load().dc_workspace_bytes
    return int(fn(op, ins, len(inputs), ctypes.byref(lparams) if lparams else None))


def query_status(workspace=None, stream=None) -> int:
    torch = _torch()
    if workspace is None:
        workspace = _default_ws.get(torch.cuda.current_device())
    if workspace is None or workspace.buf is None:
        return DC_OK
    return int(load().dc_query_status(ctypes.c_void_p(workspace.buf.data_ptr()), _stream_handle(stream)))


def set_tuning(op: int, in_dtype: int, threads: int, tile_rows: int, tile_cols: int, ctas_per_sm: int = 0):
    t = dc_tuning(threads, tile_rows, tile_cols, ctas_per_sm)
    rc = load().dc_set_tuning(op, in_dtype, ctypes.byref(t))
    if rc != DC_OK:
        raise DcError(rc, "dc_set_tuning")


def get_tuning(op: int, in_dtype: int) -> tuple[int, int, int, int]:
    t = dc_tuning()
    rc = load().dc_get_tuning(op, in_dtype, ctypes.byref(t))
    if rc != DC_OK:
        raise DcError(rc, "dc_get_tuning")
    return (t.threads, t.tile_rows, t.tile_cols, t.ctas_per_sm)


def debug_profile(on: bool):
    load().dc_debug_profile(1 if on else 0)


def read_profile(workspace, n_img: int = 1, stream=None) -> dict:
    """Profile of the last launch on `workspace` (a Workspace or a PreparedCall)."""
    buf = workspace.ws_buf if hasattr(workspace, "ws_buf") else workspace.buf
    out = (ctypes.c_uint64 * (8 + n_img * 8))()
    rc = load().dc_debug_read_profile(ctypes.c_void_p(buf.data_ptr()), n_img, out, _stream_handle(stream))
    if rc != DC_OK:
        raise DcError(rc, "dc_debug_read_profile")
    v = list(out)
    res = {"dep_wait_ns": v[0], "stage_wait_ns": v[1], "tile_wait_ns": v[2], "data_wait_ns": v[3],
           "tiles": v[4], "kernel_ns": v[6] - v[5], "images": []}
    for i in range(n_img):
        st = v[8 + i * 8: 12 + i * 8]
        en = v[12 + i * 8: 16 + i * 8]
        res["images"].append([(s - v[5], e - v[5]) if s else None for s, e in zip(st, en)])
    return res


def local_tile_cols(sizes, block_s: int = 32, in_dtype: int = DC_U8, n_sm: int = 152) -> int:
    """Local tile width a call on images of the given (height, width) sizes would use."""
    n = len(sizes)
    hs = (ctypes.c_int32 * n)(*[int(h) for h, _ in sizes])
    ws = (ctypes.c_int32 * n)(*[int(w) for _, w in sizes])
    cols = ctypes.c_int32(0)
    rc = load().dc_local_tile_cols(block_s, hs, ws, n, in_dtype, n_sm, ctypes.byref(cols))
    if rc != DC_OK:
        raise DcError(rc, "dc_local_tile_cols")
    return int(cols.value)


def last_launch_count() -> int:
    return int(load().dc_last_launch_count())


def debug_fail_launch(k: int):
    """Make the k-th kernel launch of every later call fail before it is issued
    (k = 0: off).  A host-side test hook for the error paths."""
    rc = load().dc_debug_fail_launch(int(k))
    if rc != DC_OK:
        raise DcError(rc, "dc_debug_fail_launch")


def debug_bounds() -> tuple[bool, int]:
    """(built with bounds checks, flags of buffers accessed out of bounds since the last read)."""
    flags = ctypes.c_uint32(0)
    checked = ctypes.c_int32(0)
    rc = load().dc_debug_bounds(ctypes.byref(flags), ctypes.byref(checked))
    if rc != DC_OK:
        raise DcError(rc, "dc_debug_bounds")
    return bool(checked.value), int(flags.value)


def parse_stats(buf, n: int) -> list[dict]:
    """Decode n dc_global_stats records from a uint8 tensor or bytes."""
    raw = bytes(buf.cpu().numpy().tobytes()) if hasattr(buf, "cpu") else bytes(buf)
    out = []
    for i in range(n):
        rec = raw[i * STATS_BYTES:(i + 1) * STATS_BYTES]
        f = np.frombuffer(rec[:16], dtype=np.float32)
        q = np.frombuffer(rec[16:32], dtype=np.int64)
        h = np.frombuffer(rec[32:], dtype=np.uint32).copy()
        out.append({"mu": float(f[0]), "lmin": float(f[1]), "lmax": float(f[2]), "logsum_fixed": int(q[0]),
                    "npix": int(q[1]), "hist": h})
    return out


class VideoLocalStreams:
    """n video streams through the local operator frame by frame
    (dc_decolorize_tonemap_local_video): the first call (or one after restart()) is
    the local operator on each frame alone; later calls map each frame through its
    stream's previous tables in one pass over the frame and build the next tables.
    The state buffer (one record per stream) is a device tensor owned here, sized for
    the frame sizes of the first call; frames must keep those sizes."""

    def __init__(self, n: int, block_s: int = 32, radius_blocks: int = 2, bins: int = 32, alpha: float = 1.0,
                 delta: float = 1e-4, beta_r: float = BETA_R, beta_k: float = BETA_K, luma="ours", device=None,
                 workspace=None):
        self.lib = load()
        self.n = int(n)
        self.lp = local_params(block_s, radius_blocks, bins, alpha, delta)
        self.p = dc_decolor_params(beta_r, beta_k, LUMA.get(luma, luma), 1.0)
        self.ws = workspace
        self.device = device
        self.state = None
        self._restart = True

    def restart(self):
        self._restart = True

    def prepare(self, frames, outputs):
        """The call for these buffers, descriptors and workspace resolved once:
        `call(restart=None, stream=None)` enqueues one frame per stream."""
        torch = _torch()
        frames, outputs = _as_list(frames), _as_list(outputs)
        if len(frames) != self.n:
            raise ValueError("expected %d frames (one per stream)" % self.n)
        ins, outs = _arrays(frames, outputs)
        need = int(self.lib.dc_video_local_state_bytes(ins, self.n, ctypes.byref(self.lp)))
        if need == 0:
            raise DcError(DC_ERR_INVALID_ARG, "dc_video_local_state_bytes")
        if self.state is None:
            self.state = torch.zeros(need + 256, dtype=torch.uint8, device=self.device or frames[0].device)
        off = (-self.state.data_ptr()) % 256
        if self.state.numel() - off < need:
            raise ValueError("frame sizes changed: the state was sized for the first frames")
        st = ctypes.c_void_p(self.state.data_ptr() + off)
        ptr, size, buf = _workspace(DC_OP_LOCAL, ins, self.n, self.lp, self.ws)
        wsp = ctypes.c_void_p(ptr)

        def call(restart=None, stream=None):
            r = self._restart if restart is None else bool(restart)
            rc = self.lib.dc_decolorize_tonemap_local_video(ins, outs, self.n, ctypes.byref(self.p),
                                                            ctypes.byref(self.lp), 1 if r else 0, st, need, wsp,
                                                            size, _stream_handle(stream))
            if rc != DC_OK:
                raise DcError(rc, "dc_decolorize_tonemap_local_video")
            self._restart = False
            return outputs

        call.keep = (frames, outputs, buf)
        return call

    def __call__(self, frames, outputs, stream=None):
        return self.prepare(frames, outputs)(stream=stream)
