"""Oracle pins for the paper's compact random-access form (Sec. 5.1 indexing table, Sec. 5.3
DC records): every MCU starts on a byte, the first luma DC and both chroma DCs leave the
entropy stream as 12-bit absolute values, and byte offsets are stored absolutely for every
ninth MCU and relative to it for the next eight.

Pinned against what is fixed independently of the compact reader:
- every MCU decoded from the compact form equals the standard-form random-access decode
  (itself pinned to the sequential decode of the JFIF file);
- the stored DCs are the sequential decode's DC coefficients;
- each MCU's byte length is ceil((its coded bits - its removed DC bits) / 8), with both
  counts taken from a sequential parse of the standard stream;
- the table sizes give the paper's 160/9 + 36 bits per MCU.
"""

import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def _set(seed=11):
    sizes = [(64, 64), (96, 48), (33, 17), (256, 144), (8, 8)]
    return synth.make_texture_set(seed, sizes, [50, 75, 95, 100, 60], [420, 444, 420, 420, 444],
                                  full_chain=True, compact=True)


def test_compact_decode_equals_standard_decode():
    ts = _set()
    std = oracle.texset_from(ts)
    cpt = oracle.texset_from(ts, compact=True)
    n = 0
    for t, l, e in ts.uploads():
        mw = 16 if e.sampling == 420 else 8
        for m in range(e.nmcu):
            np.testing.assert_array_equal(cpt.decode_mcu(t, l, m, mw), std.decode_mcu(t, l, m, mw))
            n += 1
    assert n > 300


def test_stored_dcs_are_the_sequential_dcs():
    ts = _set(12)
    for t, l, e in ts.uploads():
        q = oracle.Decoded(e.jfif).qcoef  # [n, ndu, 64], natural order
        bits = np.unpackbits(e.compact.dc.view(np.uint8), bitorder="little")
        ndu = q.shape[1]
        for m in range(e.nmcu):
            for c, d in enumerate([0, ndu - 2, ndu - 1]):
                v = int(np.dot(bits[36 * m + 12 * c: 36 * m + 12 * c + 12], 1 << np.arange(12)))
                v = v - 4096 if v >= 2048 else v
                assert v == q[m, d, 0], (t, l, m, c)


def test_byte_offsets_follow_from_the_standard_stream():
    ts = _set(13)
    std = oracle.texset_from(ts)
    for t, l, e in ts.uploads():
        bits, dcb = std.mcu_bits(t, l)
        assert bits.sum() == e.scan_bits
        lengths = (bits - dcb + 7) // 8
        starts = np.concatenate([[0], np.cumsum(lengths)[:-1]])
        c = e.compact
        j = np.arange(e.nmcu) // 9
        i = np.arange(e.nmcu) % 9
        rel = np.where(i > 0, c.rel[np.maximum(8 * j + i - 1, 0)], 0).astype(np.int64)
        np.testing.assert_array_equal(c.abs[j].astype(np.int64) + rel, starts)
        assert c.scan.size == lengths.sum()
        assert c.dc_bits_removed == dcb.sum()
        assert c.pad_bits == ((8 - (bits - dcb) % 8) % 8).sum()
        # 4:4:4 MCUs keep no DC in the stream; 4:2:0 MCUs keep three luma differences
        assert (dcb >= (3 if e.sampling == 444 else 2)).all()


def test_table_sizes_give_the_papers_bits_per_mcu():
    with open(GOLDEN) as f:
        g = {k: v["value"] for k, v in json.load(f).items() if not k.startswith("_")}
    e = synth.encode(synth.texture(5, 144, 144), 80, 420, compact=True)  # 81 MCUs, a multiple of 9
    c = e.compact
    n = e.nmcu
    assert n % 9 == 0
    index_bits = (32 * c.abs.size + 16 * c.rel.size) / n
    assert int(index_bits * 1000) / 1000 == g["index_bits_per_mcu"]
    assert c.dc.size * 32 - 36 * n in range(32)  # 36 bits per MCU, padded to a word
    total = index_bits + 36
    assert int(total * 1000) / 1000 == g["overhead_bits_per_mcu"]


@pytest.mark.parametrize("filt", [0, 1, 2])
def test_frame_through_the_compact_form(filt):
    ts = _set(14)
    gb = synth.gbuffer_scene(14, 200, 120, ts.sizes, ts.nlevels, synth.Pose(quad_seed=14), nquads=25)
    std = oracle.texset_from(ts)
    cpt = oracle.texset_from(ts, compact=True)
    np.testing.assert_array_equal(cpt.mark(gb, filt), std.mark(gb, filt))
    np.testing.assert_array_equal(cpt.colorize(gb.uv, gb.tex_id, gb.mip, filt),
                                  std.colorize(gb.uv, gb.tex_id, gb.mip, filt))


def test_bad_table_sizes_are_rejected():
    e = synth.encode(synth.texture(6, 32, 32), 70, 420, compact=True)
    o = oracle.TexSet()
    e.compact.rel = e.compact.rel[:-1]
    with pytest.raises(ValueError):
        o.add_compact(0, 0, e)


def test_data_unit_offsets_and_decode_by_units():
    """Data-unit starts (an index extension: each data unit decodable on its own, its DC
    difference chained afterwards): the generator's offsets equal the starts a sequential
    decode finds, and decoding every MCU unit by unit gives the MCU decode's tiles, also for
    levels reduced from it."""
    ts = _set(15)
    std = oracle.texset_from(ts)
    units = oracle.texset_from(ts)
    for t, l, e in ts.uploads():
        ndu = 6 if e.sampling == 420 else 3
        np.testing.assert_array_equal(std.du_starts(t, l, ndu), e.du_offsets.astype(np.int64))
        units.set_du_offsets(t, l, e.du_offsets)
    n = 0
    for t, l, e in ts.uploads():
        mw = 16 if e.sampling == 420 else 8
        for m in range(e.nmcu):
            np.testing.assert_array_equal(units.decode_mcu(t, l, m, mw), std.decode_mcu(t, l, m, mw))
            n += 1
    assert n > 300
    # a wrong offset is caught: the unit runs past the next unit's start
    e = ts.levels[0][0]
    bad = oracle.texset_from(synth.TextureSet([[e]]))
    offs = e.du_offsets.copy()
    offs[0, 0] -= 1
    bad.set_du_offsets(0, 0, offs)
    with pytest.raises(ValueError):
        bad.decode_mcu(0, 0, 0, 16)
