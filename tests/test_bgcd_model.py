"""Word-level model of the batch-GCD reformulation, checked against the definition.

The GPU scan does not form prod_{j != i} n_j.  Per modulus it reduces block
products word by word (q = t_0 n' mod 2^32, t = (t + q n) / 2^32, the next word
entering at the top of an L+1-word window), multiplies the residues into a
running product with Montgomery multiplications, and takes gcd with n_i.  This
model replays those word steps in Python integers for small limb counts and
checks (1) the window stays within L+2 words and ends at most n, (2) the
reduction equals P * 2^(-32 M) mod n, (3) the resulting gcds equal
gcd(n_i, prod of the others) for every modulus, including duplicates, shared
factors, short moduli and ragged blocks.
"""
import math
import random

import pytest

W32 = 1 << 32


def _words(x, n):
    return [(x >> (32 * i)) & (W32 - 1) for i in range(n)]


def _val(ws):
    return sum(w << (32 * i) for i, w in enumerate(ws))


def _reduce_step(t, n_val, np_, L):
    q = (t[0] * np_) % W32
    v = _val(t) + q * n_val
    assert v % W32 == 0
    v //= W32
    assert v < (1 << (32 * (L + 2)))
    return _words(v, L + 2)


def _redc_long(T, n_val, np_, L):
    M = len(T)
    t = T[:L] + [0, 0]
    for s in range(M):
        t = _reduce_step(t, n_val, np_, L)
        x = T[s + L] if s + L < M else 0
        t = _words(_val(t) + (x << (32 * (L - 1))), L + 2)
        assert t[L + 1] == 0
    w = _val(t)
    assert w <= n_val
    return w - n_val if w == n_val else w


def _cios(a, b, n_val, np_, L):
    t = [0] * (L + 2)
    A = _words(a, L)
    for i in range(L):
        t = _words(_val(t) + _words(b, L)[i] * _val(A), L + 2)
        t = _reduce_step(t, n_val, np_, L)
    w = _val(t)
    assert w < 2 * n_val
    return w - n_val if w >= n_val else w


def _scan(mods, L, blk):
    k = len(mods)
    R = 1 << (32 * L)
    blocks = [mods[c:c + blk] for c in range(0, k, blk)]
    bprod = [math.prod(b) for b in blocks]
    out = []
    for i, n in enumerate(mods):
        np_ = (-pow(n, -1, W32)) % W32
        acc = 1
        w = i // 32
        for sb in range(-(-k // 32)):
            if sb == w:
                for j in range(32 * sb, min(k, 32 * sb + 32)):
                    if j != i:
                        acc = _cios(mods[j], acc, n, np_, L)
            else:
                for c in range(32 * sb // blk, min(len(blocks), (32 * sb + 32) // blk)):
                    M = len(blocks[c]) * L
                    r = _redc_long(_words(bprod[c], M), n, np_, L)
                    assert r == bprod[c] * pow(R, -len(blocks[c]), n) % n
                    acc = _cios(r, acc, n, np_, L)
        out.append(math.gcd(n, acc))
    return out


@pytest.mark.parametrize("L,k,blk", [(2, 1, 8), (2, 17, 8), (2, 40, 16), (4, 70, 32), (4, 33, 16)])
def test_scan_model_equals_definition(L, k, blk):
    rng = random.Random(L * 1000 + k)
    mods = [rng.getrandbits(32 * L) | 1 | (1 << (32 * L - 1)) for _ in range(k)]
    if k > 3:
        mods[2] = mods[0]                                   # duplicate
        p = rng.getrandbits(16 * L) | 1
        mods[1] = p * (rng.getrandbits(16 * L - 1) | 1)     # shares p with the next
        if k > 20:
            mods[20] = p * (rng.getrandbits(16 * L - 1) | 1)
    mods[-1] = (mods[-1] >> 40) | 1                         # short modulus
    got = _scan(mods, L, blk)
    want = [math.gcd(n, math.prod(mods[:i] + mods[i + 1:])) for i, n in enumerate(mods)]
    assert got == want
