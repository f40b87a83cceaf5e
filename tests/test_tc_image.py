"""Host-side checks of the tensor-core CRT path's precomputation (no GPU).

The variant-3 kernel (crt_tc.cu) reduces T = A*B modulo a 1024-bit prime p
with Montgomery's method, R = 2^1024, as two matrix products of byte digits:
  mu = (T mod R) * p' mod R,  p' = -p^-1 mod R      (MMA 1 + a carry pass)
  U  = (T + mu * p) / R                              (MMA 2 + a carry pass)
MMA 2 produces positions 124..251 of mu * p; positions 252..254 (six byte
products) are added on the CUDA cores.
The B operands are Toeplitz matrices of p' and p that the host builds at key
load (rsa_tc_operand_image returns the same bytes).  These tests
  - decode the image (fp16, K-major core-matrix layout) and compare every
    entry with the Toeplitz definition, p' taken from Python's pow(p, -1, R);
  - replay the kernel's arithmetic in float64 (exact at these magnitudes) on
    the decoded matrices -- bias block, column sums, the carry pass, the carry
    estimate from four columns of the low half -- and compare mu, the carry
    and U with plain integer arithmetic (the definition of Montgomery
    reduction), over random and extreme products T.
"""
import numpy as np
import pytest

import workloads

R = 1 << 1024
ROWS_BM, ROWS_BP, KT = 128, 128, 144


@pytest.fixture(scope="module")
def lib():
    from paper_1407_1465_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def key():
    return workloads.gen_keys([(2048, 0)], workloads.DEFAULT_SEED)[0]


def decode(img, off, rows):
    """(rows, KT) float64 values of an fp16 K-major no-swizzle core-matrix image."""
    r = np.arange(rows)[:, None]
    k = np.arange(KT)[None, :]
    byte = (k // 8) * (rows // 8) * 128 + (r // 8) * 128 + (r % 8) * 16 + (k % 8) * 2
    bits = img[off:off + rows * KT * 2].view(np.uint16)
    return bits[byte // 2].view(np.float16).astype(np.float64)


def digits(x, n=128):
    return np.frombuffer(int(x).to_bytes(n, "little"), dtype=np.uint8).astype(np.int64)


def toeplitz(dig, rows, first):
    out = np.zeros((rows, KT))
    for j in range(rows):
        for k in range(128):
            i = first + j - k
            if 0 <= i < 128:
                out[j, k] = dig[i]
    out[:, 128:] = 2048.0
    return out


def test_image_is_the_toeplitz_of_p_and_p_prime(lib, key):
    from paper_1407_1465_gb300 import RSA_TC_IMAGE_BYTES, rsa_tc_operand_image
    for m in (key.p, key.q):
        img = rsa_tc_operand_image(m)
        assert img.size == RSA_TC_IMAGE_BYTES == ROWS_BM * KT * 2 + ROWS_BP * KT * 2
        mp = (-pow(m, -1, R)) % R
        assert (m * mp) % R == R - 1
        bm, bp = decode(img, 0, ROWS_BM), decode(img, ROWS_BM * KT * 2, ROWS_BP)
        assert np.array_equal(bm, toeplitz(digits(mp), ROWS_BM, 0))
        assert np.array_equal(bp, toeplitz(digits(m), ROWS_BP, 124))


def test_image_rejects_even_modulus(lib):
    from paper_1407_1465_gb300 import RsaError, rsa_tc_operand_image
    with pytest.raises(RsaError):
        rsa_tc_operand_image((1 << 1023) + 2)


def carry_pass(cols, x0=0):
    """Digits (mod 256) and carry out of a column-sum vector, low column first."""
    d = np.zeros(len(cols), dtype=np.int64)
    c = x0
    for i, v in enumerate(cols):
        x = int(v) + c
        d[i] = x & 0xFF
        c = x >> 8
    return d, c


def replay_reduction(T, m, bm, bp):
    """The kernel's reduction of T (< m * R) on the decoded B operands."""
    bias_a = np.full(16, 2.0 ** -16)
    t_lo = digits(T % R)
    a1 = np.concatenate([t_lo * 2.0 ** -24, bias_a])      # fp16 subnormals d * 2^-24
    col1 = a1 @ bm.T                                        # 1/2 + v * 2^-24
    v = (col1 - 0.5) * 2.0 ** 24
    assert np.all(v == np.round(v)) and v.max() < 2 ** 23
    mu_d, _ = carry_pass(v.astype(np.int64))
    mu = int.from_bytes(bytes(mu_d.astype(np.uint8)), "little")
    a2 = np.concatenate([mu_d * 2.0 ** -24, bias_a])
    w = ((a2 @ bp.T) - 0.5) * 2.0 ** 24                     # positions 124..251 of mu * m
    assert np.all(w == np.round(w)) and w.max() < 2 ** 23
    w = w.astype(np.int64)
    md = digits(m)                                          # positions 252..255: direct products
    top = [mu_d[125] * md[127] + mu_d[126] * md[126] + mu_d[127] * md[125],
           mu_d[126] * md[127] + mu_d[127] * md[126], mu_d[127] * md[127], 0]
    w = np.concatenate([w, np.array(top, dtype=np.int64)])  # positions 124..255
    # carry out of the low half: ceil((positions 124..127 with T's bytes) / 2^32)
    y, c = carry_pass([w[i] + t_lo[124 + i] for i in range(4)])
    carry = c + (1 if y.any() else 0)
    hi_d, cout = carry_pass(w[4:], carry)
    U = (T >> 1024) + int.from_bytes(bytes(hi_d.astype(np.uint8)), "little") + (cout << 1024)
    return mu, carry, U


def test_reduction_replay_matches_integer_montgomery(lib, key):
    from paper_1407_1465_gb300 import rsa_tc_operand_image
    rng = np.random.default_rng(7)
    for m in (key.p, key.q):
        img = rsa_tc_operand_image(m)
        bm, bp = decode(img, 0, ROWS_BM), decode(img, ROWS_BM * KT * 2, ROWS_BP)
        mp = (-pow(m, -1, R)) % R
        rinv = pow(R, -1, m)
        cases = [0, 1, (m - 1) ** 2, (m - 1) * (R - 1), m * R - 1, R - 1, R, (R - 1) * 3]
        cases += [int.from_bytes(rng.bytes(128), "little") * int.from_bytes(rng.bytes(128), "little") % (m * R)
                  for _ in range(24)]
        for T in cases:
            mu, carry, U = replay_reduction(T, m, bm, bp)
            assert mu == (T % R) * mp % R
            # the carry out of the low half of the column sums (exact convolution),
            # which the kernel estimates from positions 124..127 only
            conv = np.convolve(digits(mu), digits(m))[:128]
            low = (T % R) + sum(int(conv[i]) << (8 * i) for i in range(128))
            assert carry == low // R and low % R == 0
            assert U == (T + mu * m) // R and U < 2 * m
            assert (U - m if U >= m else U) == T * rinv % m


def test_worst_case_columns_stay_below_2_23():
    """128 products of two bytes: the largest column sum the MMAs can produce."""
    assert 128 * 255 * 255 < 2 ** 23


# ---------------------------------------------------------------- RSA-3072/4096: two reduction rounds
# A prime of H limbs (1536 or 2048 bits) reduces in two rounds of r = 2^(16H)
# with D = 2H byte digits per round: MMA 1 is D x D, MMA 2 returns positions
# D-4 .. 3D-5 of mu * m (2D columns), positions 3D-4 .. 3D-2 come directly.


def decode_rows(img, off, rows, kt):
    r = np.arange(rows)[:, None]
    k = np.arange(kt)[None, :]
    byte = (k // 8) * (rows // 8) * 128 + (r // 8) * 128 + (r % 8) * 16 + (k % 8) * 2
    bits = img[off:off + rows * kt * 2].view(np.uint16)
    return bits[byte // 2].view(np.float16).astype(np.float64)


def toeplitz_round(dig, rows, first, ndig, D):
    """rows x (D + 16): row j, column k < D: digit first + j - k of a number of ndig digits; bias 2048."""
    out = np.zeros((rows, D + 16))
    for j in range(rows):
        for k in range(D):
            i = first + j - k
            if 0 <= i < ndig:
                out[j, k] = dig[i]
    out[:, D:] = 2048.0
    return out


@pytest.fixture(scope="module")
def round_keys():
    return workloads.gen_keys([(3072, 0), (4096, 0)], workloads.DEFAULT_SEED)


def round_operands(m, H):
    from paper_1407_1465_gb300 import rsa_tc_round_image_bytes, rsa_tc_round_operand_image
    D = 2 * H
    img = rsa_tc_round_operand_image(32 * H, m)
    assert img.size == rsa_tc_round_image_bytes(32 * H) == D * (D + 16) * 2 + 2 * D * (D + 16) * 2
    return decode_rows(img, 0, D, D + 16), decode_rows(img, D * (D + 16) * 2, 2 * D, D + 16)


def test_round_images_are_the_toeplitz_of_m_and_m_prime(lib, round_keys):
    for key in round_keys:
        H = key.bits // 64
        D, r = 2 * H, 1 << (16 * H)
        for m in (key.p, key.q):
            b1, b2 = round_operands(m, H)
            mp = (-pow(m, -1, r)) % r
            assert np.array_equal(b1, toeplitz_round(digits(mp, D), D, 0, D, D))
            assert np.array_equal(b2, toeplitz_round(digits(m, 2 * D), 2 * D, D - 4, 2 * D, D))


def test_round_image_rejects_bad_arguments(lib, round_keys):
    from paper_1407_1465_gb300 import RsaError, rsa_tc_round_operand_image
    with pytest.raises(RsaError):
        rsa_tc_round_operand_image(2048, (1 << 2047) + 2)
    with pytest.raises(RsaError):
        rsa_tc_round_operand_image(1024, (1 << 1023) + 1)     # only 1536- and 2048-bit primes


def replay_round(V, m, b1, b2, H):
    """One reduction round of crt_tc4.cu on the decoded operands: mu = (V mod r)
    m' mod r by MMA 1 and a carry pass, positions D-4 .. 3D-5 of mu * m by MMA 2
    and 3D-4 .. 3D-1 directly, the carry out of the low half from four columns
    (with V's top bytes), then (V + mu m) / r."""
    D, r = 2 * H, 1 << (16 * H)
    bias_a = np.full(16, 2.0 ** -16)
    v_lo = digits(V % r, D)
    col1 = (np.concatenate([v_lo * 2.0 ** -24, bias_a]) @ b1.T - 0.5) * 2.0 ** 24
    assert np.all(col1 == np.round(col1)) and col1.max() < 2 ** 23
    mu_d, _ = carry_pass(col1.astype(np.int64))
    w = (np.concatenate([mu_d * 2.0 ** -24, bias_a]) @ b2.T - 0.5) * 2.0 ** 24
    assert np.all(w == np.round(w)) and w.max() < 2 ** 23
    w = w.astype(np.int64)
    md = digits(m, 2 * D)
    top = [mu_d[D - 3] * md[2 * D - 1] + mu_d[D - 2] * md[2 * D - 2] + mu_d[D - 1] * md[2 * D - 3],
           mu_d[D - 2] * md[2 * D - 1] + mu_d[D - 1] * md[2 * D - 2], mu_d[D - 1] * md[2 * D - 1], 0]
    w = np.concatenate([w, np.array(top, dtype=np.int64)])                      # positions D-4 .. 3D-1
    y, c = carry_pass([w[i] + v_lo[D - 4 + i] for i in range(4)])
    carry = c + (1 if y.any() else 0)
    hi_d, cout = carry_pass(w[4:], carry)                                        # positions D .. 3D-1
    mu = int.from_bytes(bytes(mu_d.astype(np.uint8)), "little")
    return mu, (V >> (16 * H)) + int.from_bytes(bytes(hi_d.astype(np.uint8)), "little") + (cout << (32 * H))


@pytest.mark.parametrize("bits", [3072, 4096])
def test_two_round_reduction_replay_matches_integer_montgomery(lib, round_keys, bits):
    """Two rounds of r = 2^(16H) give T R^-1 mod m (R = 2^(32H)) below 2m, over
    random and extreme products T < m^2 (the kernel's operands are below m)."""
    key = next(k for k in round_keys if k.bits == bits)
    H = bits // 64
    r, R = 1 << (16 * H), 1 << (32 * H)
    rng = np.random.default_rng(9 + H)
    for m in (key.p, key.q):
        b1, b2 = round_operands(m, H)
        mp1 = (-pow(m, -1, r)) % r
        rinv = pow(R, -1, m)
        cases = [0, 1, (m - 1) ** 2, (m - 1) * (m - 2), (m - 1) * r, r - 1, r, R - 1, (R - 1) * 5 % (m * m)]
        cases += [(int.from_bytes(rng.bytes(4 * H), "little") % m) * (int.from_bytes(rng.bytes(4 * H), "little") % m)
                  for _ in range(12)]
        for T in cases:
            mu1, T1 = replay_round(T, m, b1, b2, H)
            assert mu1 == (T % r) * mp1 % r and T1 == (T + mu1 * m) // r and (T + mu1 * m) % r == 0
            mu2, T2 = replay_round(T1, m, b1, b2, H)
            assert T2 == (T1 + mu2 * m) // r and T2 < 2 * m
            assert (T2 - m if T2 >= m else T2) == T * rinv % m
