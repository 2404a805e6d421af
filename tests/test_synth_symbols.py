"""The input generator's per-MCU Huffman symbol counts (used to express the decode's issue
rate per symbol) equal a count made from the quantised coefficients: per data unit one DC
category, one symbol per non-zero AC coefficient, one ZRL per full run of 16 zeros before
a non-zero coefficient, and an EOB when the unit ends in zeros (T.81 F.1.2.2)."""

import numpy as np
import pytest

import synth


def count_symbols(qc: np.ndarray) -> np.ndarray:
    zz = synth.zigzag()  # natural index of each zig-zag position
    out = np.zeros(qc.shape[0], np.int64)
    for m in range(qc.shape[0]):
        for d in range(qc.shape[1]):
            z = qc[m, d][zz]
            n, run = 1, 0
            for k in range(1, 64):
                if z[k] == 0:
                    run += 1
                    continue
                n += run // 16 + 1
                run = 0
            out[m] += n + (1 if run > 0 else 0)
    return out


@pytest.mark.parametrize("quality, sampling", [(50, 420), (95, 420), (90, 444)])
def test_symbol_counts(quality, sampling):
    e = synth.encode(synth.texture(7, 128, 128), quality, sampling, keep_coefs=True)
    qc = e.qcoef.reshape(e.nmcu, -1, 64)
    np.testing.assert_array_equal(e.symbols.astype(np.int64), count_symbols(qc))


def test_symbol_counts_with_long_zero_runs():
    """Blocks with a lone coefficient at k = 63 (three ZRLs before it, no EOB) and with runs
    of exactly 16 zeros."""
    rng = np.random.default_rng(5)
    qc = np.zeros((4, 6, 64), np.int16)
    zz = synth.zigzag()
    qc[0, :, 0] = 3
    qc[0, 0, zz[63]] = 1
    qc[1, :, zz[17]] = -2
    qc[2] = rng.integers(-3, 4, (6, 64))
    qc[3, 2, zz[40]] = 5
    e = synth.encode_coefs(qc, 2, 2, 420)
    np.testing.assert_array_equal(e.symbols.astype(np.int64), count_symbols(qc))
