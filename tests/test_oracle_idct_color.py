"""Oracle pins for the integer IDCT and the fixed-point colour conversion.

The paper names the steps (Sec. 4.3: dequantisation, IDCT, colour space conversion) but
not their arithmetic; the oracle fixes one integer spec. These tests pin it to the
mathematics rather than to itself:
* IEEE 1180-1990-style accuracy against an FP64 IDCT on random blocks;
* closed forms: zero block -> 128, DC-only block -> a constant near 128 + dq/8;
* the constant matrix is (up to its 2^13 scale) orthonormal;
* colour: neutral chroma gives R = G = B = Y exactly, and every one of the 2^24 inputs is
  within 1 of the rounded float JFIF conversion.
"""

import numpy as np
import pytest

import oracle


def _basis():
    x = np.arange(8)[:, None]
    u = np.arange(8)[None, :]
    c = np.where(u == 0, np.sqrt(0.5), 1.0)
    return 0.5 * c * np.cos((2 * x + 1) * u * np.pi / 16)  # A[x,u], orthonormal


def test_constant_matrix_is_scaled_orthonormal_basis():
    K = oracle.idct_matrix().astype(float) / 16384.0
    A = _basis()
    assert np.abs(K - A).max() <= 0.5 / 16384 + 1e-12  # every entry is A rounded to 2^-14
    np.testing.assert_allclose(K @ K.T, np.eye(8), atol=2e-3)


def test_zero_block():
    assert (oracle.idct_pixels(np.zeros(64, np.int32)) == 128).all()


@pytest.mark.parametrize("dq", [-2896, -1024, -517, -8, -5, -4, -3, -1, 0, 1, 3, 4, 5, 8, 100, 517, 1016, 2047,
                                2896])
def test_dc_only_block_is_constant(dq):
    d = np.zeros(64, np.int32)
    d[0] = dq
    raw = oracle.idct_raw(d)[0]
    assert (raw == raw[0]).all()
    assert abs(raw[0] - dq / 8.0) <= 1.0  # f = dq * (1/(2 sqrt 2))^2 = dq / 8
    px = oracle.idct_pixels(d)[0]
    assert px[0] == min(255, max(0, raw[0] + 128))


def test_dc_only_saturates_in_the_column_pass():
    """Beyond |dq| ~ 2,900 the column pass output (5 fractional bits) leaves int16 and is
    clamped; only adversarial streams get there. The block stays constant."""
    d = np.zeros(64, np.int32)
    d[0] = 32767
    raw = oracle.idct_raw(d)[0]
    assert (raw == raw[0]).all()
    assert raw[0] == (5793 * 32767 + 262144) // 524288


@pytest.mark.parametrize("lim", [(256, 255), (5, 5), (300, 300)])
@pytest.mark.parametrize("sign", [1, -1])
def test_ieee1180_accuracy(lim, sign):
    """IEEE 1180-1990 procedure: random spatial blocks in [-L, H], FP64 forward DCT,
    rounded and clipped to [-2048, 2047]; compare the integer IDCT with the FP64 IDCT
    (both rounded and clipped to [-256, 255]) over 10,000 blocks."""
    L, H = lim
    rng = np.random.default_rng(1180 + L)
    A = _basis()
    f = rng.integers(-L, H + 1, (10000, 8, 8)).astype(np.float64) * sign
    F = np.einsum("xu,byx,yv->bvu", A, f, A)  # forward DCT (A^T f A), F[v,u]
    F = np.clip(np.rint(F), -2048, 2047)
    ref = np.einsum("xu,bvu,yv->byx", A, F, A)
    ref = np.clip(np.rint(ref), -256, 255)
    got = np.clip(oracle.idct_raw(F.reshape(-1, 64).astype(np.int32)).reshape(-1, 8, 8), -256, 255)
    e = got - ref
    assert np.abs(e).max() <= 1
    assert (e ** 2).mean(axis=0).max() <= 0.06        # per-pixel mean square error
    assert (e ** 2).mean() <= 0.02                     # overall mean square error
    assert np.abs(e.mean(axis=0)).max() <= 0.015       # per-pixel mean error
    assert abs(e.mean()) <= 0.0015                     # overall mean error


def test_ieee1180_zero_in_zero_out():
    assert (oracle.idct_raw(np.zeros((3, 64), np.int32)) == 0).all()


def test_idct_orientation():
    """A single horizontal-frequency coefficient varies along x only, vertical along y only."""
    d = np.zeros(64, np.int32)
    d[1] = 400  # (v=0, u=1)
    r = oracle.idct_raw(d)[0].reshape(8, 8)
    assert (r == r[0:1, :]).all() and r[0, 0] > 0 > r[0, 7]
    d = np.zeros(64, np.int32)
    d[8] = 400  # (v=1, u=0)
    r = oracle.idct_raw(d)[0].reshape(8, 8)
    assert (r == r[:, 0:1]).all() and r[0, 0] > 0 > r[7, 0]


def test_neutral_chroma_is_grey():
    y = np.arange(256, dtype=np.uint8)
    ycc = np.stack([y, np.full(256, 128, np.uint8), np.full(256, 128, np.uint8)], axis=1)
    rgb = oracle.ycc_to_rgb(ycc)
    assert (rgb == y[:, None]).all()


def test_colour_exhaustive_within_one():
    Y, Cb, Cr = np.meshgrid(np.arange(256), np.arange(256), np.arange(256), indexing="ij")
    ycc = np.stack([Y, Cb, Cr], axis=-1).reshape(-1, 3).astype(np.uint8)
    got = oracle.ycc_to_rgb(ycc).astype(np.int16)
    y = ycc[:, 0].astype(np.float64)
    cb = ycc[:, 1].astype(np.float64) - 128
    cr = ycc[:, 2].astype(np.float64) - 128
    ref = np.stack([y + 1.402 * cr, y - 0.344136 * cb - 0.714136 * cr, y + 1.772 * cb], axis=1)
    ref = np.clip(np.rint(ref), 0, 255).astype(np.int16)
    assert np.abs(got - ref).max() <= 1
    assert (got == ref).mean() > 0.99
