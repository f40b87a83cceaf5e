"""Compressed Toeplitz operands for a tensor-core reduction (a design check).

A K-major, no-swizzle MMA operand is read as 8x8 core matrices (16 bytes per
row, 128 bytes each) at  start + kblock * LBO + rowgroup * SBO.  For a
Toeplitz matrix B[n][k] = m[n - k] (0 <= n - k < D, else 0) the core matrix at
(row group g, k-block b) depends only on g - b, so one array X of core
matrices indexed by the diagonal g - b, plus a copy Y shifted by one diagonal
(Y[d] = X[d - 1], serving the second k-block of each 16-wide MMA step), stand
in for the dense matrix with both strides positive: SBO = 128 (next row group
= next diagonal) and LBO = Y - X.  This model builds X and Y for D = 256 byte
digits and checks, for every MMA step and every element of its 256 x 16
operand tile, that the descriptor's address holds B[n][k] -- the layout a
4096-bit (2048-bit-prime) reduction would need, in 2 x 63 x 128 B = 16 KB
instead of 128 KB.
"""
import random

D = 256                       # byte digits of the constant (2048-bit prime)
N = 256                       # operand rows (output columns of the MMA)
CORE = 128                    # bytes per 8x8 fp16 core matrix


def dense(m, n, k):
    i = n - k
    return m[i] if 0 <= i < D else 0


def build(m):
    """Byte image: X[d] for d in -31..31 at offset (d + 31) * 128, then Y[d] = core(d - 1)."""
    img = bytearray(2 * 63 * CORE)
    for base, shift in ((0, 0), (63 * CORE, 1)):
        for d in range(-31, 32):
            c = [[m[8 * (d - shift) + r - e] if 0 <= 8 * (d - shift) + r - e < D else 0 for e in range(8)]
                 for r in range(8)]
            off = base + (d + 31) * CORE
            for r in range(8):
                for e in range(8):
                    v = c[r][e]
                    img[off + 16 * r + 2 * e:off + 16 * r + 2 * e + 2] = v.to_bytes(2, "little")
    return img


def test_compressed_toeplitz_matches_dense_under_descriptor_addressing():
    rng = random.Random(4096)
    m = [rng.randrange(256) for _ in range(D)]
    img = build(m)
    LBO, SBO = 63 * CORE, CORE                 # both positive
    assert LBO % 16 == 0 and SBO % 16 == 0 and LBO // 16 < (1 << 14)
    for t in range(D // 16):                   # MMA steps of 16 digits: k-blocks 2t, 2t + 1
        start = (0 - 2 * t + 31) * CORE        # X entry of (row group 0, k-block 2t)
        for n in range(N):
            g, r = divmod(n, 8)
            for kk in range(16):
                b, e = divmod(kk, 8)           # b = 0: k-block 2t (X), b = 1: 2t + 1 (Y)
                addr = start + b * LBO + g * SBO + 16 * r + 2 * e
                assert 0 <= addr < len(img)
                got = int.from_bytes(img[addr:addr + 2], "little")
                assert got == dense(m, n, 16 * t + kk), (t, n, kk)
