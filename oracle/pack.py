"""Oracle of the lossless stage after quantization (TEST INFRASTRUCTURE ONLY;
only the test suite may import it): bit-plane packing of int32 codes.  The
paper hands its bins to LC's lossless stages and describes none; this is our
own format, written here in plain numpy, one block at a time:

  z = zigzag(code): 2 code for code >= 0, -2 code - 1 for code < 0 (uint32);
  blocks of 32 codes (the last padded with zeros); w = bit length of the OR
  of the block's z;
  bytes: w of every block as uint8, zero-padded to a multiple of 16, then for
  each block w little-endian uint32 words, word j with bit i = bit j of the
  block's i-th z.
"""
import numpy as np


def zigzag(codes):
    v = np.asarray(codes, dtype=np.int64)
    return np.where(v >= 0, 2 * v, -2 * v - 1).astype(np.uint32)


def unzigzag(z):
    z = np.asarray(z, dtype=np.int64)
    return np.where(z % 2 == 0, z // 2, -(z + 1) // 2).astype(np.int32)


def _align16(b):
    return (b + 15) // 16 * 16


def pack(codes):
    codes = np.asarray(codes, dtype=np.int32)
    n = codes.size
    nb = (n + 31) // 32
    z = np.zeros(nb * 32, dtype=np.uint32)
    z[:n] = zigzag(codes)
    widths = np.zeros(_align16(nb), dtype=np.uint8)
    words = []
    for b in range(nb):
        blk = [int(v) for v in z[32 * b:32 * b + 32]]
        acc = 0
        for v in blk:
            acc |= v
        w = acc.bit_length()
        widths[b] = w
        for j in range(w):
            word = 0
            for i, v in enumerate(blk):
                word |= ((v >> j) & 1) << i
            words.append(word)
    return widths.tobytes() + np.asarray(words, dtype="<u4").tobytes()


def unpack(buf, n):
    nb = (n + 31) // 32
    raw = np.frombuffer(buf, dtype=np.uint8)
    widths = raw[:nb]
    words = np.frombuffer(raw[_align16(nb):].tobytes(), dtype="<u4")
    z = np.zeros(nb * 32, dtype=np.uint64)
    k = 0
    for b in range(nb):
        for j in range(int(widths[b])):
            word = int(words[k])
            k += 1
            for i in range(32):
                z[32 * b + i] |= ((word >> i) & 1) << j
    return unzigzag(z[:n])


def packed_size(codes):
    """align16(nb) + 4 * sum of block widths."""
    n = np.asarray(codes).size
    nb = (n + 31) // 32
    z = np.zeros(nb * 32, dtype=np.uint32)
    z[:n] = zigzag(codes)
    acc = np.bitwise_or.reduce(z.reshape(nb, 32), axis=1)
    w = np.array([int(a).bit_length() for a in acc])
    return _align16(nb) + 4 * int(w.sum())
