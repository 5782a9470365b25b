"""The byte arithmetic of the small-alphabet kernel's DNA form, checked on the
CPU exhaustively (the GPU parity tests check the kernel itself): for four
keyword bytes that (byte >> 1) & 3 tells apart, one multiply of a word masked
to its code bits gathers the four codes, in order, into the top byte, and a
byte permute selected by twice the codes rebuilds exactly the bytes that are
keyword bytes.  The byte permute below follows the PTX `prmt` default mode
(byte n of the result is byte (selector nibble n & 7) of the pair, sign-
replicated when bit 3 of the nibble is set)."""
import itertools

import pytest


def prmt(a: int, b: int, sel: int) -> int:
    src = [(a >> (8 * i)) & 0xFF for i in range(4)] + [(b >> (8 * i)) & 0xFF for i in range(4)]
    r = 0
    for n in range(4):
        nib = (sel >> (4 * n)) & 0xF
        v = src[nib & 7]
        if nib & 8:
            v = 0xFF if v & 0x80 else 0
        r |= v << (8 * n)
    return r


def word(bs) -> int:
    return bs[0] | bs[1] << 8 | bs[2] << 16 | bs[3] << 24


def test_multiply_gathers_codes_in_order():
    """Every word masked to bits 1-2 of each byte (4^4 cases): the top byte of
    its product with 0x00820820 holds code j at bits 2j, 2j + 1."""
    for codes in itertools.product(range(4), repeat=4):
        x = word([c << 1 for c in codes])
        top = ((x * (0x01041040 >> 1)) & 0xFFFFFFFF) >> 24
        assert top == sum(c << (2 * j) for j, c in enumerate(codes)), codes


@pytest.mark.parametrize("alphabet", [b"ACGT", b"acgt", bytes([0x00, 0x02, 0x04, 0x06])])
def test_byte_check_is_exact(alphabet):
    """Byte j of a word is flagged (non-zero after the XOR) exactly when it is
    not a keyword byte, for all 256 values of that byte, whatever keyword or
    other bytes the other three lanes hold."""
    key = {(b >> 1) & 3: b for b in alphabet}
    assert len(key) == 4
    lo = key[0] | key[1] << 16
    hi = key[2] | key[3] << 16
    fillers = list(alphabet) + [0x4E, 0x00 if 0x00 not in alphabet else 0x01, 0xFF]
    for j in range(4):
        for others in itertools.product(fillers, repeat=3):
            for v in range(256):
                bs = list(others[:j]) + [v] + list(others[j:])
                w = word(bs)
                x = w & 0x06060606
                sel = prmt(x | (x >> 4), 0, 0x4420)
                u = w ^ prmt(lo, hi, sel)
                for i in range(4):
                    assert (((u >> (8 * i)) & 0xFF) != 0) == (bs[i] not in alphabet), (alphabet, bs, i)
