"""Index arithmetic of the interaction's hit-mask words, checked on the CPU.

The candidate test handles two candidate pairs (four candidates, slots
4j .. 4j + 3 of a 32-slot word) per step: the half-precision results of pair
2j (a) and pair 2j + 1 (b) hold each candidate's sign bit at bit 15 (even
slot) or 31 (odd slot); a sign-replicating byte permute with selector 0xFDB9
spreads them over the four bytes of one word, and bit j of byte k is kept.
So slot s lives at bit 8 (s mod 4) + s / 4.  The pair phase decodes a bit b
back to slot 4 (b mod 8) + b / 8 = 4b - 31 (b / 8), and the mask of the slots
in use, [0, lim), comes from a table.  These tests restate those rules
independently and check that they agree with each other."""
import numpy as np


def slot_bit(s):
    return 8 * (s & 3) + (s >> 2)


def decode(b):
    return 4 * b - 31 * (b >> 3)


def keep(lim):
    k = 0
    for s in range(lim):
        k |= 1 << slot_bit(s)
    return k


def prmt_sign(a, b, sel=0xFDB9):
    """Byte n of the result: the sign bit of byte (sel >> 4n) & 7 of (b:a),
    replicated over 8 bits (the selector nibble's high bit is set)."""
    src = a | (b << 32)
    out = 0
    for n in range(4):
        nib = (sel >> (4 * n)) & 0xF
        assert nib & 8
        byte = (src >> (8 * (nib & 7))) & 0xFF
        out |= (0xFF if byte & 0x80 else 0) << (8 * n)
    return out


def test_slot_bit_is_a_bijection_and_decode_inverts_it():
    bits = [slot_bit(s) for s in range(32)]
    assert sorted(bits) == list(range(32))
    for s in range(32):
        assert decode(slot_bit(s)) == s


def test_keep_table_selects_exactly_the_slots_in_use():
    for lim in range(33):
        k = keep(lim)
        assert bin(k).count("1") == lim
        assert {decode(b) for b in range(32) if k >> b & 1} == set(range(lim))
    assert keep(32) == 0xFFFFFFFF


def test_sign_bytes_place_four_candidates_of_a_step():
    rng = np.random.default_rng(5)
    for _ in range(2000):
        hits = rng.integers(0, 2, 32).astype(bool)     # candidate slot -> hit
        m = 0
        for j in range(8):
            # pair 2j: slots 4j (bit 15), 4j + 1 (bit 31); pair 2j + 1: 4j + 2, 4j + 3
            noise = int(rng.integers(0, 1 << 31)) & 0x7FFF7FFF   # non-sign bits
            a = noise | (hits[4 * j] << 15) | (hits[4 * j + 1] << 31)
            noise = int(rng.integers(0, 1 << 31)) & 0x7FFF7FFF
            b = noise | (hits[4 * j + 2] << 15) | (hits[4 * j + 3] << 31)
            m |= prmt_sign(a, b) & (0x01010101 << j)
        got = [bool(m >> slot_bit(s) & 1) for s in range(32)]
        assert got == list(hits)
