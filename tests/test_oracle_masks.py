"""Pins of the parity checker's exemption masks against hand-computed rounding midpoints.

binary16 has 10 fraction bits: in [2^e, 2^(e+1)) neighbouring values are 2^(e-10)
apart, so rounding midpoints sit at k 2^(e-10) + 2^(e-11).  An 8-bit code q is
chosen by floor(255 y + 1/2), so its boundaries are (k + 1/2)/255.  The masks accept
both neighbours within 1e-5 (absolute below 1, relative above) of such a midpoint.
"""
import numpy as np
import pytest

import oracle

# (value, inside the 1e-5 band of a binary16 midpoint?)
F16_CASES = [
    (0.5 + 2.0 ** -12, True),              # midpoint between 0.5 and 0.5 + 2^-11
    (0.5 + 2.0 ** -12 + 0.9e-5, True),
    (0.5 + 2.0 ** -12 - 0.9e-5, True),
    (0.5 + 2.0 ** -12 + 1.1e-5, False),
    (0.5 + 2.0 ** -12 - 1.1e-5, False),
    (0.5 - 2.0 ** -13, True),              # midpoint between 0.5 and 0.5 - 2^-12 (spacing below 0.5)
    (0.5 - 2.0 ** -13 - 0.9e-5, True),
    (0.5 - 2.0 ** -13 - 1.1e-5, False),
    (0.5, False),                          # a binary16 value: 2.4e-4 from either midpoint
    (0.25, False),
    (0.25 + 2.0 ** -13, True),             # midpoint in [1/4, 1/2): spacing 2^-12
    (0.75 + 2.0 ** -12 + 2e-5, False),
    (1000.25, True),                       # [512, 1024): spacing 1/2, midpoint at .25
    (1000.25 + 0.009, True),               # relative band: 1e-5 * 1000 = 0.01
    (1000.25 + 0.011, False),
    (1000.0, False),
    (0.001, True),                         # spacing 2^-20 < 2e-5: every value is near a midpoint
    (-(0.5 + 2.0 ** -12), True),           # sign-symmetric
    (-0.5, False),
]


@pytest.mark.parametrize("y,inside", F16_CASES)
def test_f16_boundary_mask_midpoints(y, inside):
    assert bool(oracle.f16_boundary_mask(np.array([y]))[0]) is inside


def test_f16_boundary_mask_agrees_with_rounding_ties():
    # the midpoints themselves are where numpy's binary16 rounding switches neighbour:
    # just below rounds down, just above rounds up
    for lo in (0.5, 0.625, 0.25, 3.0, 700.0):
        h = np.float16(lo)
        up = np.nextafter(h, np.float16(np.inf))
        mid = 0.5 * (float(h) + float(up))
        assert np.float16(np.nextafter(mid, -np.inf)) == h
        assert np.float16(np.nextafter(mid, np.inf)) == up
        assert oracle.f16_boundary_mask(np.array([mid]))[0]


U8_CASES = [
    (0.5 / 255, True),                     # boundary between codes 0 and 1
    (127.5 / 255, True),
    (127.5 / 255 + 0.9e-5, True),
    (127.5 / 255 - 0.9e-5, True),
    (127.5 / 255 + 1.1e-5, False),
    (127.5 / 255 - 1.1e-5, False),
    (128.0 / 255, False),                  # a code centre
    (1.0, False),
    (0.0, False),
]


@pytest.mark.parametrize("y,inside", U8_CASES)
def test_u8_boundary_mask(y, inside):
    assert bool(oracle.u8_boundary_mask(np.array([y]))[0]) is inside


def test_gray_code_rounding():
    # floor(255 y + 1/2): 127.5/255 rounds up to 128, just below it to 127; clamped at the ends
    assert oracle.gray_code(np.array([127.5 / 255]))[0] == 128
    assert oracle.gray_code(np.array([np.nextafter(127.5 / 255, 0)]))[0] == 127
    assert oracle.gray_code(np.array([-0.1, 1.2]))[0] == 0
    assert oracle.gray_code(np.array([-0.1, 1.2]))[1] == 255
