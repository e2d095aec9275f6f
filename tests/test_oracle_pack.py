"""Pins of the lossless-stage oracle (bit-plane packing of int32 codes):
zigzag's closed-form pairs, a hand-packed block, the size formula, and the
round trip on extreme and random codes."""
import numpy as np
import pytest

import oracle.pack as PK


def test_zigzag_pairs():
    v = np.array([0, -1, 1, -2, 2, 2**31 - 1, -2**31], dtype=np.int32)
    assert PK.zigzag(v).tolist() == [0, 1, 2, 3, 4, 2**32 - 2, 2**32 - 1]
    assert np.array_equal(PK.unzigzag(PK.zigzag(v)), v)


def test_hand_packed_block():
    # codes 1 at index 0 and -3 at index 5: z = 2 (binary 10) and 5 (binary 101),
    # OR = 111 -> width 3; plane 0 = bit 5, plane 1 = bit 0, plane 2 = bit 5
    codes = np.zeros(40, dtype=np.int32)
    codes[0], codes[5] = 1, -3
    codes[33] = -1  # second block: z = 1 at index 1 -> width 1, plane 0 = bit 1
    buf = PK.pack(codes)
    assert buf[:16] == bytes([3, 1] + [0] * 14)
    words = np.frombuffer(buf[16:], dtype="<u4").tolist()
    assert words == [1 << 5, 1 << 0, 1 << 5, 1 << 1]
    assert len(buf) == PK.packed_size(codes) == 16 + 4 * 4


def test_zero_blocks_take_only_their_width_byte():
    codes = np.zeros(1000, dtype=np.int32)
    assert PK.pack(codes) == bytes(32)   # 32 blocks -> 32 zero widths, no words
    assert np.array_equal(PK.unpack(PK.pack(codes), 1000), codes)


@pytest.mark.parametrize("n", [1, 31, 32, 33, 100, 1023])
def test_round_trip(n):
    rng = np.random.default_rng(n)
    codes = rng.integers(-2**31, 2**31, n, dtype=np.int64).astype(np.int32)
    codes[::7] = rng.integers(-5, 6, codes[::7].size)
    codes[:2] = [-2**31, 2**31 - 1][:min(2, n)]
    buf = PK.pack(codes)
    assert len(buf) == PK.packed_size(codes)
    assert np.array_equal(PK.unpack(buf, n), codes)
