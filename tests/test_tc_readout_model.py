"""The column readout of the tensor-core Montgomery reduction, word by word.

An MMA leaves one fp32 word per digit position: the bias 0x3F000000 plus an
integer column sum w < 2^23.  The kernels read a run of such columns as the
integer sum_c w_c 256^c in two steps: adjacent columns pair into base-2^16
columns y_j = w_2j + 256 w_2j+1 (below 2^32; the pairing subtracts one bias
and shifts the other out), and with y_j = L_j + 2^16 H_j the run's value is
X + Y, X the string of the L_j and Y that of the H_j one base-2^16 digit up,
added as 32-bit words with one carry.  Here that readout (mu = T m' mod R, and
the high half of T + mu m added to T_hi with the carry out of the low half
entering as a pending high half) is modelled with 32-bit operations and
compared with plain integer arithmetic, at random and at the largest column
sums the bias allows.
"""
import random

import pytest

BIAS = 0x3F000000
M32 = (1 << 32) - 1


def pair_cols(w_even, w_odd):
    return ((w_odd << 8) + (w_even - BIAS)) & M32


def lo_halves(y_even, y_odd):
    return (y_even & 0xFFFF) | ((y_odd & 0xFFFF) << 16)


def hi_halves(y_below, y_even):
    return (y_below >> 16) | ((y_even >> 16) << 16)


def readout_mod(cols, yb=0):
    """Words of sum_c w_c 256^c mod 2^(8 len(cols)), chunk by chunk of 16
    columns with the carry and the column below kept between chunks."""
    words, cw = [], 0
    for c0 in range(0, len(cols), 16):
        y = [pair_cols(cols[c0 + 2 * j], cols[c0 + 2 * j + 1]) for j in range(8)]
        for k in range(4):
            s = lo_halves(y[2 * k], y[2 * k + 1]) + hi_halves(y[2 * k - 1] if k else yb, y[2 * k]) + cw
            words.append(s & M32)
            cw = s >> 32
        yb = y[7]
    return words


def add_columns(t, j0, v, yb, cs, cin):
    """t[j0 .. j0 + len(v)/4) += the columns v (the kernels' add_columns)."""
    nl = len(v) // 4
    y = [pair_cols(v[2 * i], v[2 * i + 1]) for i in range(2 * nl)]
    x = []
    for i in range(nl):
        s = lo_halves(y[2 * i], y[2 * i + 1]) + hi_halves(y[2 * i - 1] if i else yb, y[2 * i]) + cs
        x.append(s & M32)
        cs = s >> 32
    for i in range(nl):
        s = t[j0 + i] + x[i] + cin
        t[j0 + i] = s & M32
        cin = s >> 32
    return y[-1], cs, cin


def words_to_int(ws):
    return sum(w << (32 * i) for i, w in enumerate(ws))


def columns(rng, n, extreme):
    return [BIAS + ((1 << 23) - 1 if extreme else rng.randrange(1 << 23)) for _ in range(n)]


@pytest.mark.parametrize("extreme", [False, True])
def test_mu_readout_is_the_column_sum_mod_r(extreme):
    rng = random.Random(5)
    for _ in range(200):
        cols = columns(rng, 128, extreme)
        want = sum((w - BIAS) << (8 * c) for c, w in enumerate(cols)) % (1 << 1024)
        assert words_to_int(readout_mod(cols)) == want


@pytest.mark.parametrize("extreme", [False, True])
def test_high_half_readout_adds_the_rounded_quotient(extreme):
    """Positions 124..255 of mu * m (128 MMA columns, the top ones as the CUDA
    cores form them) plus T: limb 0 receives the carry out of the low half,
    ceil(positions 124..127 with T's top limb / 2^32) -- the kernels' rounding
    of the part below position 128 -- and the rest adds to T_hi."""
    rng = random.Random(9)
    for _ in range(200):
        cols = columns(rng, 132, extreme)   # positions 124..255: 128 MMA columns, 4 formed on the CUDA cores
        top = M32 if extreme else rng.getrandbits(32)
        t_hi = [M32 if extreme else rng.getrandbits(32) for _ in range(32)]
        # the model of the kernel's step 5
        t = list(t_hi)
        y0 = pair_cols(cols[0], cols[1]) + (top & 0xFFFF)
        y1 = pair_cols(cols[2], cols[3]) + (top >> 16) + (y0 >> 16)
        assert y0 <= M32 and y1 <= M32
        c = (y1 >> 16) + (1 if (y0 | y1) & 0xFFFF else 0)
        assert c < 1 << 16
        yb, cs, cin = c << 16, 0, 0
        yb, cs, cin = add_columns(t, 0, cols[4:16], yb, cs, cin)
        for k in range(1, 8):
            yb, cs, cin = add_columns(t, 3 + 4 * (k - 1), cols[16 * k:16 * k + 16], yb, cs, cin)
        yb, cs, cin = add_columns(t, 31, cols[128:132], yb, cs, cin)
        got = words_to_int(t) + (((yb >> 16) + cs + cin) << 1024)
        # plain integers: the columns at positions 124.., T's top limb at 124..127,
        # the part below position 128 rounded up to a whole unit of position 128
        low = sum((w - BIAS) << (8 * c) for c, w in enumerate(cols[:4])) + top
        high = sum((w - BIAS) << (8 * (c - 4)) for c, w in enumerate(cols[4:], start=4))
        want = words_to_int(t_hi) + high + -(-low // (1 << 32))
        assert got == want
