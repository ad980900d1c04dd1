"""Device-buffer helpers for the GPU tests (padding, offsets, guard bands)."""
import numpy as np

GUARD = 0xA5


def torch_dtype(np_dtype):
    import torch
    return {np.dtype(np.uint8): torch.uint8, np.dtype(np.float16): torch.float16,
            np.dtype(np.float32): torch.float32}[np.dtype(np_dtype)]


def to_dev(img: np.ndarray, pad_px: int = 0, offset_elems: int = 0):
    """Copy an (H, W, 3) image to the GPU with `pad_px` extra pixels per row and the
    first pixel `offset_elems` samples into its allocation."""
    import torch
    H, W, _ = img.shape
    row = 3 * (W + pad_px)
    buf = torch.zeros(offset_elems + H * row + 16, dtype=torch_dtype(img.dtype), device="cuda")
    t = buf[offset_elems:offset_elems + H * row].view(H, W + pad_px, 3)[:, :W, :]
    t.copy_(torch.from_numpy(np.ascontiguousarray(img)))
    return t


class GuardedOut:
    """An (H, W) output plane inside a larger allocation whose spare bytes hold a
    guard pattern; check() asserts that nothing outside the plane was written."""

    def __init__(self, H, W, dtype, pad_px=0, offset_elems=0, guard_elems=64):
        import torch
        self.tdt = {"u8": torch.uint8, "f16": torch.float16, "f32": torch.float32}[dtype]
        self.H, self.W, self.pad = H, W, pad_px
        esz = torch.tensor([], dtype=self.tdt).element_size()
        n = guard_elems + offset_elems + H * (W + pad_px) + guard_elems
        self.raw = torch.full((n * esz,), GUARD, dtype=torch.uint8, device="cuda")
        full = self.raw.view(self.tdt)
        start = guard_elems + offset_elems
        self.view = full[start:start + H * (W + pad_px)].view(H, W + pad_px)[:, :W]
        mask = np.ones(n * esz, dtype=bool)
        for r in range(H):
            a = (start + r * (W + pad_px)) * esz
            mask[a:a + W * esz] = False
        self.mask = mask

    def check(self):
        raw = self.raw.cpu().numpy()
        assert np.all(raw[self.mask] == GUARD), "write outside the output plane"

    def numpy(self):
        return self.view.cpu().numpy()
