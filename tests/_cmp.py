"""Comparison rules between the CUDA path and the FP64 oracle.

Tolerances (binary32 arithmetic against an FP64 reference):
 - f32 output on [0,1]: |y - y64| <= 2e-6; unbounded HDR luminance: relative
   2e-6 * max(1, |L64|).
 - u8 output: the 8-bit code equals floor(255 y64 + 1/2) except where y64 lies
   within 1e-5 (in [0,1] units) of a rounding boundary (k + 1/2)/255, where the two
   neighbouring codes are both accepted.
 - f16 output: the nearest binary16 of y64, except within 1e-5 (relative) of a
   rounding midpoint, where both neighbours are accepted.
"""
import numpy as np

TOL_F32 = 2e-6
U8_EPS = 1e-5


def check_f32(got, ref, tol=TOL_F32, rel=False, what=""):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    bound = tol * np.maximum(1.0, np.abs(ref)) if rel else tol
    err = np.abs(got - ref)
    bad = err > bound
    assert not np.any(bad), "%s: %d values beyond tolerance, max err %.3g at %s (got %r ref %r)" % (
        what, int(bad.sum()), float(err.max()), np.unravel_index(np.argmax(err), err.shape),
        float(got.ravel()[np.argmax(err)]), float(ref.ravel()[np.argmax(err)]))
    return float(err.max()) if err.size else 0.0


def check_u8(got, ref_y, what="", extra_exempt=None):
    import oracle
    got = np.asarray(got)
    ref_q = oracle.gray_code(ref_y)
    exempt = oracle.u8_boundary_mask(ref_y, U8_EPS)
    if extra_exempt is not None:
        exempt = exempt | extra_exempt
    d = np.abs(got.astype(np.int32) - ref_q.astype(np.int32))
    bad = (d != 0) & ~exempt
    assert not np.any(bad), "%s: %d u8 codes differ outside the exemption (first at %s: got %d ref %d, y64=%r)" % (
        what, int(bad.sum()), np.argwhere(bad)[0], int(got[tuple(np.argwhere(bad)[0])]),
        int(ref_q[tuple(np.argwhere(bad)[0])]), float(ref_y[tuple(np.argwhere(bad)[0])]))
    if extra_exempt is None:
        assert np.all(d <= 1), what + ": exempt codes differ by more than one"
    return int((d != 0).sum())


def check_f16(got, ref_y, what=""):
    import oracle
    got = np.asarray(got).astype(np.float16)
    ref_h = np.asarray(ref_y, dtype=np.float64).astype(np.float16)
    exempt = oracle.f16_boundary_mask(ref_y, U8_EPS)
    same = (got == ref_h) | (np.isnan(got) & np.isnan(ref_h))
    bad = ~same & ~exempt
    assert not np.any(bad), "%s: %d f16 values differ outside the exemption" % (what, int(bad.sum()))
    return int((~same).sum())


def check_out(got, ref_y, dtype, what="", rel=False):
    if dtype == "u8":
        return check_u8(got, ref_y, what)
    if dtype == "f16":
        return check_f16(got, ref_y, what)
    return check_f32(got, ref_y, rel=rel, what=what)
