"""Oracle pins: zig-zag order and canonical Huffman tables (T.81 Annex C, F.2.2.3)."""

import os

import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_zigzag_is_t81_figure_a6():
    ref = []
    with open(os.path.join(GOLDEN, "t81_zigzag.txt")) as f:
        for line in f:
            if not line.startswith("#"):
                ref += [int(v) for v in line.split()]
    assert oracle.zigzag().tolist() == ref


def test_zigzag_structure():
    zz = oracle.zigzag()
    assert sorted(zz.tolist()) == list(range(64))  # a permutation
    diag = [(i // 8) + (i % 8) for i in zz]
    assert all(a <= b for a, b in zip(diag, diag[1:]))  # anti-diagonals in order
    # direction alternates: along odd diagonals the row increases, along even ones it falls
    for s in range(15):
        rows = [i // 8 for i in zz if (i // 8) + (i % 8) == s]
        assert rows == (sorted(rows) if s % 2 else sorted(rows, reverse=True))


def _codes_from_decoder_tables(bits, vals):
    """Expand MINCODE/VALPTR into {symbol: (code, length)}."""
    rc, mn, mx, vp = oracle.huff_tables(bits, vals)
    assert rc == 0
    out = {}
    for l in range(1, 17):
        for j in range(int(bits[l - 1])):
            out[int(vals[vp[l] + j])] = (int(mn[l]) + j, l)
    return out


@pytest.mark.parametrize("t", range(4))
def test_standard_tables_are_valid_prefix_codes(t):
    bits, vals, nv = synth.standard_huffman()
    b, v = bits[t], vals[t][: nv[t]]
    assert int(b.sum()) == nv[t]
    if t % 2 == 0:  # DC: categories 0..11 (8-bit baseline)
        assert sorted(v.tolist()) == list(range(12))
    else:  # AC: EOB, ZRL and every (run, size) with size 1..10
        valid = {0x00, 0xF0} | {(r << 4) | s for r in range(16) for s in range(1, 11)}
        assert sorted(v.tolist()) == sorted(valid)
    kraft = sum(int(b[l - 1]) * 2.0 ** -l for l in range(1, 17))
    assert kraft < 1.0  # strictly below 1: the all-ones code of some length stays unused
    codes = _codes_from_decoder_tables(b, vals[t])
    for sym, (code, ln) in codes.items():
        assert code != (1 << ln) - 1, "no code may be all ones"
    # prefix-free
    items = sorted(codes.values(), key=lambda cl: cl[1])
    for i, (c1, l1) in enumerate(items):
        for c2, l2 in items[i + 1:]:  # l1 <= l2: c1 must not be a prefix of c2
            assert (c2 >> (l2 - l1)) != c1


@pytest.mark.parametrize("t", range(4))
def test_decoder_codes_equal_encoder_codes(t):
    """Annex C built twice, independently (decoder side in the oracle, encoder side in the
    generator), must give the same code for every symbol."""
    bits, vals, nv = synth.standard_huffman()
    dec = _codes_from_decoder_tables(bits[t], vals[t])
    code, ln = synth.encoder_codes(bits[t], vals[t])
    for sym, (c, l) in dec.items():
        assert (int(code[sym]), int(ln[sym])) == (c, l), sym


@pytest.mark.parametrize("t", range(4))
def test_bit_serial_decode_of_every_code(t, rng):
    bits, vals, nv = synth.standard_huffman()
    dec = _codes_from_decoder_tables(bits[t], vals[t])
    for sym, (c, l) in dec.items():
        tail = int(rng.integers(0, 1 << 16))
        word = (c << (32 - l)) | (tail >> l)  # code followed by random bits
        data = word.to_bytes(4, "big")
        s, used = oracle.huff_decode_one(bits[t], vals[t], data)
        assert (s, used) == (sym, l)


def test_invalid_code_is_reported():
    bits, vals, nv = synth.standard_huffman()
    # sixteen one-bits match no code of the AC luminance table
    s, used = oracle.huff_decode_one(bits[1], vals[1], b"\xff\xff\x00\x00")
    assert s == -1
