"""Pins of the oracle's chroma placement: saturated flat colours, one per quadrant of each MCU,
encoded at quality 100 (every quantiser step 1) and decoded back to their known RGB.

At 4:2:0 an MCU is 16 x 16 texels with one 8 x 8 chroma data unit per component covering it
at half resolution: texel (x, y) takes chroma sample (x >> 1, y >> 1) (Sec. 3.1's MCU of
four luma and two chroma blocks; chroma replicated, the reading of the upsampling). Each
8 x 8 quadrant of the MCU gets its own colour, so a chroma sample taken from another
quadrant, Cb and Cr exchanged, or chroma from a wrong data unit, misses its quadrant's colour
by more than 100 levels, far beyond the tolerance. The tolerance covers the round trip the
colour conversion and the integer transform allow at quality 100 away from the quadrant
edges (where the DCT of a step rings): texels 2..5 of each quadrant, whose chroma samples
1..2 lie inside the quadrant's 4 x 4 chroma samples."""

import numpy as np
import pytest

import oracle
import synth

# red, cyan, blue, yellow: each pair far apart in (Cb, Cr), and each far from its own
# colour with Cb and Cr exchanged (see the last test)
QUADRANT_COLOURS = np.array([[255, 0, 0], [0, 255, 255], [0, 0, 255], [255, 255, 0]], np.uint8)  # TL, TR, BL, BR
TOL = 6


def _quadrant_image(mcus: int, mw: int, colours) -> np.ndarray:
    """mcus x mcus MCUs of mw texels; in each, the four mw/2 quadrants take colours 0..3."""
    n = mcus * mw
    img = np.zeros((n, n, 3), np.uint8)
    h = mw // 2
    for y in range(n):
        for x in range(n):
            q = (1 if (x % mw) >= h else 0) + (2 if (y % mw) >= h else 0)
            img[y, x] = colours[q]
    return img


def _interior(mw: int) -> np.ndarray:
    """Texel offsets (within an MCU) at least 2 texels inside their quadrant."""
    h = mw // 2
    return np.array([o for o in range(mw) if 2 <= (o % h) <= h - 3])


def test_saturated_quadrants_decode_to_their_colours_420():
    _check(420, 16, _quadrant_image(2, 16, QUADRANT_COLOURS), lambda mcu, y, x: (x >= 8) + 2 * (y >= 8),
           _interior(16))


def test_saturated_mcus_decode_to_their_colours_444():
    """At 4:4:4 chroma has full resolution and an MCU is one 8 x 8 data unit per component:
    each MCU of a 2 x 2 grid is one flat colour, checked over all its texels."""
    img = np.zeros((16, 16, 3), np.uint8)
    for q in range(4):
        img[(q // 2) * 8:(q // 2) * 8 + 8, (q % 2) * 8:(q % 2) * 8 + 8] = QUADRANT_COLOURS[q]
    _check(444, 8, img, lambda mcu, y, x: mcu, np.arange(8))


def _check(sampling, mw, img, colour_of, inner):
    e = synth.encode(img, 100, sampling)
    seq = oracle.Decoded(e.jfif).rgba
    o = oracle.TexSet()
    o.add(0, 0, e)
    assert len(inner) > 0
    for mcu in range(e.nmcu):
        my, mx = divmod(mcu, e.mcus_x)
        tile = o.decode_mcu(0, 0, mcu, mw)
        np.testing.assert_array_equal(tile, seq[my * mw:(my + 1) * mw, mx * mw:(mx + 1) * mw])
        for y in inner:
            for x in inner:
                q = colour_of(mcu, y, x)
                d = np.abs(tile[y, x, :3].astype(int) - QUADRANT_COLOURS[q].astype(int)).max()
                assert d <= TOL, (sampling, mcu, y, x, tile[y, x], QUADRANT_COLOURS[q])
                assert tile[y, x, 3] == 255


def test_exchanged_chroma_would_fail():
    """The colours are far enough apart in Cb and Cr that exchanging the two chroma planes,
    or taking another quadrant's chroma, cannot stay within the tolerance: the JFIF
    conversion of each colour with Cb and Cr swapped, or with another quadrant's (Cb, Cr),
    differs from the colour by more than 100 in some channel."""
    def ycc(c):
        r, g, b = c.astype(float)
        return (0.299 * r + 0.587 * g + 0.114 * b, 128 - 0.168736 * r - 0.331264 * g + 0.5 * b,
                128 + 0.5 * r - 0.418688 * g - 0.081312 * b)

    def rgb(y, cb, cr):
        return np.array([y + 1.402 * (cr - 128), y - 0.344136 * (cb - 128) - 0.714136 * (cr - 128),
                         y + 1.772 * (cb - 128)]).clip(0, 255)

    for i, c in enumerate(QUADRANT_COLOURS):
        y, cb, cr = ycc(c)
        assert np.abs(rgb(y, cr, cb) - c).max() > 100  # exchanged planes
        for j, c2 in enumerate(QUADRANT_COLOURS):
            if j != i:
                _, cb2, cr2 = ycc(c2)
                assert np.abs(rgb(y, cb2, cr2) - c).max() > 100, (i, j)  # another quadrant's chroma
