"""Pins of the oracle's endpoint quantisers (Sec. 3.2: the predicted endpoints are turned into
BC data, RGB565 colours for BC1 and 8-bit values for BC4) against hand-derived values.

tests/golden/endpoint_quant.txt lists FP32 inputs by bit pattern with the expected integer
field, each row carrying its intermediate values: the half-way points (k + 1/2)/L and one FP32
ulp either side, 0 and 1, values that must clamp, and e = 0.5 (which separates a scale of 31
from 32 and the 6-bit G channel from the 5-bit R and B). The test only reads the expected
values; it does not evaluate the quantisation formula itself.
"""
import os
import struct

import numpy as np

from oracle import ntbc as ont

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "endpoint_quant.txt")


def f32(hexbits):
    return np.frombuffer(struct.pack("<I", int(hexbits, 16)), np.float32)[0]


def load():
    fields, words = [], []
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            if line[0] == "word":
                words.append((int(line[1], 16), [f32(b) for b in line[2:5]]))
            else:
                fields.append((int(line[0]), f32(line[1]), int(line[2])))
    return fields, words


def test_golden_file_covers_every_scale():
    fields, words = load()
    assert {L for L, _, _ in fields} == {31, 63, 255}
    assert all(sum(1 for L, _, _ in fields if L == s) >= 20 for s in (31, 63, 255))
    assert len(words) >= 5


def test_u8_quantiser_matches_hand_values():
    fields, _ = load()
    rows = [(e, q) for L, e, q in fields if L == 255]
    got = ont.quantize_endpoints_u8(np.array([e for e, _ in rows], np.float32))
    for (e, q), g in zip(rows, got):
        assert int(g) == q, (float(e), q, int(g))


def _fields565(word):
    word = int(word)
    return word >> 11, (word >> 5) & 63, word & 31


def test_565_channels_match_hand_values():
    """Each 5-bit row is checked in the R and in the B position, each 6-bit row in G; the
    other two channels hold 0 and must stay 0."""
    fields, _ = load()
    for L, e, q in fields:
        if L == 255:
            continue
        positions = (0, 2) if L == 31 else (1,)
        for ch in positions:
            x = np.zeros((1, 3), np.float32)
            x[0, ch] = e
            r, g, b = _fields565(ont.quantize_endpoints_bc1(x)[0])
            got = (r, g, b)
            want = [0, 0, 0]
            want[ch] = q
            assert got == tuple(want), (L, ch, float(e), want, got)


def test_packed_565_words():
    _, words = load()
    for word, (er, eg, eb) in words:
        got = int(ont.quantize_endpoints_bc1(np.array([[er, eg, eb]], np.float32))[0])
        assert got == word, (hex(word), hex(got), float(er), float(eg), float(eb))
