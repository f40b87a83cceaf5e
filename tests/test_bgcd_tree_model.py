"""CPU model of the product/remainder-tree batch GCD kernels (csrc/bgcd_tree.cu).

The GPU path computes g_i = gcd(n_i, prod_{j != i} n_j) for many moduli at
once (the weak-key scan of the paper's introduction) with a product tree and a
remainder tree instead of a scan over all pairs.  This file restates, in
Python integers, the exact steps and word sizes the kernels take, and checks
them against math.gcd on small sets, so that the bounds the kernels rely on
(no conditional subtraction in the tree, one extra word of slack, the Newton
steps, the transform indexing) are pinned before the GPU runs them:

  * product tree X_t (node of 2^t moduli, s_t = L 2^t words), padding leaves 1;
  * Y_t = X_t^2, mu_t = -Y_t^-1 mod 2^(32*2s_t): by Newton from one word at
    the top level of the remainder tree (the root's children), below it from
    the parent: mu_a = Y_b mu_parent mod 2^(32*2s_t), one product;
  * Montgomery remainder tree Z_t = (Z_{t+1} + q Y_t) / 2^(32*2s_t),
    q = Z_{t+1} mu_t mod 2^(32*2s_t), Z_T = X_T, with no subtraction
    (Z_t < (T - t + 1) Y_t, stored in 2 s_t + 1 words);
  * leaves: word-serial Montgomery reduction of the node's Z modulo n_i^2,
    one conditional subtraction, exact division by n_i, gcd with n_i;
  * products by three-prime number-theoretic transforms of 32-bit words
    (decimation in frequency forward, in time inverse, nested twiddle table
    tw[len + j] = w_(2len)^j), recombined by Garner's method, with an addend
    and an output slice.
"""
import math
import random

import pytest

W = 32
MASK = (1 << W) - 1
PRIMES = (2013265921, 3221225473, 3489660929)   # 15*2^27+1, 3*2^30+1, 13*2^28+1


def words(x, n):
    return [(x >> (W * k)) & MASK for k in range(n)]


def value(ws):
    return sum(w << (W * k) for k, w in enumerate(ws))


def neg_inv32(n0):
    inv = n0
    for _ in range(4):
        inv = (inv * (2 - n0 * inv)) & MASK
    return (-inv) & MASK


def neg_inverse(y, nw, seed_mu=None, seed_w=1):
    """mu = -y^-1 mod 2^(32 nw) by Newton doublings: with y mu = -1 + 2^(32w) (H)
    (low w words all ones), mu_hi = H mu + mu mod 2^(32w)."""
    if seed_mu is None:
        mu, w = neg_inv32(y & MASK), 1
    else:
        mu, w = seed_mu, seed_w
    while w < nw:
        prod = (y % (1 << (W * 2 * w))) * mu
        assert prod % (1 << (W * w)) == (1 << (W * w)) - 1
        h = (prod >> (W * w)) % (1 << (W * w))
        hi = (h * mu + mu) % (1 << (W * w))
        mu, w = mu + (hi << (W * w)), 2 * w
    assert (y * mu + 1) % (1 << (W * nw)) == 0
    return mu


def valid(n):
    return n % 2 == 1 and n >= 3


def tree_gcds(mods, L, t0=2):
    count = len(mods)
    K = 1
    while K < max(count, 2):
        K *= 2
    T = K.bit_length() - 1
    t0 = min(t0, T)
    leaves = [m if (i < count and valid(m)) else 1 for i, m in enumerate(list(mods) + [1] * (K - count))]
    X = [leaves]
    for t in range(T):
        X.append([X[t][2 * v] * X[t][2 * v + 1] for v in range(K >> (t + 1))])
        s = L << (t + 1)
        assert all(x < 1 << (W * s) for x in X[t + 1])
    Z = [X[T][0]]
    mu_parent = None
    for t in range(T - 1, t0 - 1, -1):
        s = L << t
        k = 2 * s
        Y = [x * x for x in X[t]]
        if t == T - 1:
            mu_t = [neg_inverse(y, k) for y in Y]              # Newton from one word, top level only
        else:
            # from the parent: mu_parent = -(Y_a Y_b)^-1, so Y_b mu_parent = -Y_a^-1
            mu_t = [Y[v ^ 1] * (mu_parent[v >> 1] % (1 << (W * k))) % (1 << (W * k)) for v in range(K >> t)]
        for v, y in enumerate(Y):
            assert (y * mu_t[v] + 1) % (1 << (W * k)) == 0
        mu_parent = mu_t
        Zt = []
        for v in range(K >> t):
            zp = Z[v // 2]
            y = Y[v]
            q = (zp % (1 << (W * k))) * mu_t[v] % (1 << (W * k))
            tot = zp + q * y
            assert tot % (1 << (W * k)) == 0
            # the low half sums to 0 or 2^(32k): its carry is "low half of zp nonzero"
            assert ((zp % (1 << (W * k)) + (q * y) % (1 << (W * k))) >> (W * k)) == (zp % (1 << (W * k)) != 0)
            z = tot >> (W * k)
            assert z < (T - t + 1) * y and z < 1 << (W * (k + 1))
            Zt.append(z)
        Z = Zt
    out = []
    s0 = L << t0
    for i in range(count):
        n = mods[i]
        if not valid(n):
            out.append((0, -1))
            continue
        z = Z[i >> t0]
        M = 2 * s0 + 1
        N = n * n
        k = 2 * L
        npr = neg_inv32(N & MASK)
        t = z % (1 << (W * k))
        for step in range(M):
            q = (t & MASK) * npr & MASK
            t = (t + q * N) >> W
            nxt = k + step
            if nxt < M:
                t += ((z >> (W * nxt)) & MASK) << (W * (k - 1))
        assert t <= N
        if t >= N:
            t -= N
        assert t == z * pow(2, -W * M, N) % N
        assert t % n == 0
        # exact division, word by word from the bottom
        inv = (-neg_inv32(n & MASK)) & MASK
        u, r = 0, t
        for j in range(L):
            d = ((r >> (W * j)) & MASK) * inv & MASK
            r -= (d * n) << (W * j)
            u += d << (W * j)
        assert r == 0 and u == t // n and u < n
        g = math.gcd(n, u)
        out.append((g, 0 if g == 1 else (2 if g == n else 1)))
    return out


def brute(mods):
    res = []
    for i, n in enumerate(mods):
        if not valid(n):
            res.append((0, -1))
            continue
        p = 1
        for j, m in enumerate(mods):
            if j != i and valid(m):
                p *= m
        g = math.gcd(n, p)
        res.append((g, 0 if g == 1 else (2 if g == n else 1)))
    return res


def rand_prime(rng, bits):
    while True:
        c = rng.getrandbits(bits) | (1 << (bits - 1)) | 1
        if all(pow(a, c - 1, c) == 1 for a in (2, 3, 5, 7, 11, 13)):
            return c


@pytest.mark.parametrize("count,t0", [(2, 2), (3, 1), (5, 2), (8, 2), (13, 3), (33, 2), (64, 0)])
def test_tree_matches_brute_force(count, t0):
    rng = random.Random(count * 31 + t0)
    L = 2
    primes = [rand_prime(rng, 32) for _ in range(2 * count)]
    mods = [primes[2 * i] * primes[2 * i + 1] for i in range(count)]
    if count >= 3:
        mods[1] = primes[0] * primes[5]          # shares p0 with n0
    if count >= 5:
        mods[4] = mods[2]                        # duplicate
        mods[3] = 6                              # invalid (even)
    if count >= 8:
        mods[7] = 1                              # invalid (< 3)
        mods[6] = primes[1] * primes[12 % (2 * count)]
    assert tree_gcds(mods, L, t0) == brute(mods)


def test_tree_leading_zero_limbs_and_single_valid():
    rng = random.Random(5)
    small = [rand_prime(rng, 20) * rand_prime(rng, 20) for _ in range(6)]
    small[2] = small[0]
    assert tree_gcds(small, 4, 2) == brute(small)
    assert tree_gcds([small[0], 4], 4, 2) == brute([small[0], 4])


# ---------------------------------------------------------------- transform model

def prime_consts(p):
    R = 1 << W
    e2 = 0
    while (p - 1) % (1 << (e2 + 1)) == 0:
        e2 += 1
    odd = (p - 1) >> e2
    factors = {2} | {f for f in range(3, 50, 2) if odd % f == 0 and all(f % g for g in range(3, f, 2))}
    g = next(g for g in range(2, 100) if all(pow(g, (p - 1) // f, p) != 1 for f in factors))
    return {"p": p, "R": R % p, "g": g, "e2": e2, "pinv": pow(p, -1, R)}


def mmul(a, b, c):
    p, pinv = c["p"], c["pinv"]
    t = a * b
    m = (t & MASK) * pinv & MASK
    th, mh = t >> W, (m * p) >> W
    r = th - mh
    return r + p if r < 0 else r


def tables(c, nmax):
    p, R = c["p"], 1 << W
    root = pow(c["g"], (p - 1) // nmax, p)
    iroot = pow(root, -1, p)
    tw, itw = [0] * nmax, [0] * nmax
    length = 1
    while length < nmax:
        for j in range(length):
            e = j * (nmax // (2 * length))
            tw[length + j] = pow(root, e, p) * R % p
            itw[length + j] = pow(iroot, e, p) * R % p
        length *= 2
    return tw, itw


def dif(a, n, c, tw):
    p = c["p"]
    length = n // 2
    while length >= 1:
        for blk in range(0, len(a), 2 * length):
            for j in range(length):
                u, v = a[blk + j], a[blk + j + length]
                a[blk + j] = (u + v) % p
                a[blk + j + length] = mmul((u - v) % p, tw[length + j], c)
        length //= 2


def dit(a, n, c, itw):
    p = c["p"]
    length = 1
    while length < n:
        for blk in range(0, len(a), 2 * length):
            for j in range(length):
                u, v = a[blk + j], mmul(a[blk + j + length], itw[length + j], c)
                a[blk + j] = (u + v) % p
                a[blk + j + length] = (u - v) % p
        length *= 2


def garner(r):
    p1, p2, p3 = PRIMES
    v1 = r[0]
    v2 = (r[1] - v1) * pow(p1, -1, p2) % p2
    v3 = (r[2] - v1 - p1 * v2) * pow(p1 * p2, -1, p3) % p3
    return v1 + p1 * v2 + p1 * p2 * v3


def ntt_bmul(A, B, na, nb, D=None, lo=0, hi=None, nmax=64):
    """Batched A_i * B_i + D_i, words [lo, hi), through the transform path."""
    cnt = len(A)
    n = 1
    while n < na + nb:
        n *= 2
    assert n <= nmax
    cs = [prime_consts(p) for p in PRIMES]
    res = []
    for k, c in enumerate(cs):
        p = c["p"]
        tw, itw = tables(c, nmax)
        fa = [0] * (cnt * n)
        fb = [0] * (cnt * n)
        for i in range(cnt):
            aw = words(A[i], na)
            bw = words(B[i], nb)
            for j in range(na):
                fa[i * n + j] = aw[j] % p
            for j in range(nb):
                fb[i * n + j] = bw[j] % p
        dif(fa, n, c, tw)
        dif(fb, n, c, tw)
        fa = [mmul(x, y, c) for x, y in zip(fa, fb)]
        dit(fa, n, c, itw)
        scale = pow(n, -1, p) * pow(1 << W, 2, p) % p
        res.append([mmul(x, scale, c) for x in fa])
    out = []
    for i in range(cnt):
        total = sum(garner([res[k][i * n + j] for k in range(3)]) << (W * j) for j in range(n))
        if D is not None:
            total += D[i]
        h = hi if hi is not None else n + 2
        out.append((total >> (W * lo)) % (1 << (W * (h - lo))))
    return out


@pytest.mark.parametrize("na,nb,cnt", [(3, 5, 3), (8, 8, 2), (16, 7, 2), (32, 32, 1)])
def test_transform_product(na, nb, cnt):
    rng = random.Random(na * 100 + nb)
    A = [rng.getrandbits(W * na) for _ in range(cnt)]
    B = [rng.getrandbits(W * nb) for _ in range(cnt)]
    A[0] = (1 << (W * na)) - 1                     # all-ones words: the largest columns
    B[0] = (1 << (W * nb)) - 1
    got = ntt_bmul(A, B, na, nb)
    assert got == [a * b for a, b in zip(A, B)]


def test_transform_addend_slice():
    """The remainder step's shape: an addend one word longer than the product,
    the upper half plus one word kept."""
    rng = random.Random(9)
    na, nb = 8, 8
    A = [rng.getrandbits(W * na) for _ in range(2)]
    B = [rng.getrandbits(W * nb) for _ in range(2)]
    D = [rng.getrandbits(W * (na + nb + 1)) for _ in range(2)]
    lo, hi = 8, 17
    got = ntt_bmul(A, B, na, nb, D=D, lo=lo, hi=hi)
    want = [((a * b + d) >> (W * lo)) % (1 << (W * (hi - lo))) for a, b, d in zip(A, B, D)]
    assert got == want


def test_column_bound_fits_three_primes():
    """The largest product the tree forms has operands of 2^26 words: every
    convolution column is below 2^26 * 2^64, under the primes' product; each
    prime has a root of unity of order 2^27 (the longest transform)."""
    M = PRIMES[0] * PRIMES[1] * PRIMES[2]
    assert (1 << 26) * ((1 << 32) - 1) ** 2 < M
    for p in PRIMES:
        assert (p - 1) % (1 << 27) == 0
    assert PRIMES[0] < PRIMES[1] < PRIMES[2] < 1 << 32
    assert PRIMES[0] * PRIMES[1] < 1 << 64


def tile_rounds(a, c, tw, itw, other=None):
    """The shared-memory kernels' grouping on one 4096-word tile: 512 threads,
    thread t holds words b + k q (b = (t // q) 8q + t % q) for q = 512, 64, 8,
    1 and runs the three stages at distances 4q, 2q, q; with ``other`` the
    forward rounds are followed by the product and the inverse rounds."""
    p = c["p"]
    a = list(a)

    def groups(q):
        for t in range(512):
            b = (t // q) * 8 * q + t % q
            yield t % q, [b + k * q for k in range(8)]

    def bf(i, j, w, inverse):
        u, v = a[i], a[j]
        if inverse:
            v = mmul(v, w, c)
            a[i], a[j] = (u + v) % p, (u - v) % p
        else:
            a[i], a[j] = (u + v) % p, mmul((u - v) % p, w, c)

    for q in (512, 64, 8, 1):
        for jp, ix in groups(q):
            for k in range(4):
                bf(ix[k], ix[k + 4], tw[4 * q + jp + k * q], False)
            for k, w in ((0, tw[2 * q + jp]), (1, tw[2 * q + jp + q]), (4, tw[2 * q + jp]), (5, tw[2 * q + jp + q])):
                bf(ix[k], ix[k + 2], w, False)
            for k in range(0, 8, 2):
                bf(ix[k], ix[k + 1], tw[q + jp], False)
    if other is None:
        return a
    a = [mmul(x, y, c) for x, y in zip(a, other)]
    for q in (1, 8, 64, 512):
        for jp, ix in groups(q):
            for k in range(0, 8, 2):
                bf(ix[k], ix[k + 1], itw[q + jp], True)
            for k, w in ((0, itw[2 * q + jp]), (1, itw[2 * q + jp + q]), (4, itw[2 * q + jp]), (5, itw[2 * q + jp + q])):
                bf(ix[k], ix[k + 2], w, True)
            for k in range(4):
                bf(ix[k], ix[k + 4], itw[4 * q + jp + k * q], True)
    return a


def test_tile_rounds_equal_radix2_stages():
    """Three stages per exchange on the 512-thread grouping equal the twelve
    radix-2 stages (forward; and forward, product, inverse)."""
    rng = random.Random(77)
    c = prime_consts(PRIMES[1])
    tw, itw = tables(c, 4096)
    x = [rng.randrange(c["p"]) for _ in range(4096)]
    y = [rng.randrange(c["p"]) for _ in range(4096)]
    ref = list(x)
    dif(ref, 4096, c, tw)
    assert tile_rounds(x, c, tw, itw) == ref
    yr = list(y)
    dif(yr, 4096, c, tw)
    prod = [mmul(u, v, c) for u, v in zip(ref, yr)]
    dit(prod, 4096, c, itw)
    assert tile_rounds(x, c, tw, itw, yr) == prod


def pass16(a, h, c, tws, inverse):
    """One global pass of four stages (distances 8h .. h forward, h .. 8h
    inverse) on 16-word groups b + m h, b = 16h * block + j: at distance d h
    word m pairs with m + d when m & d is clear, twiddle [d h + j + (m mod d) h]."""
    p = c["p"]
    a = list(a)
    order = (1, 2, 4, 8) if inverse else (8, 4, 2, 1)
    for blk in range(len(a) // (16 * h)):
        for j in range(h):
            b = blk * 16 * h + j
            x = [a[b + m * h] for m in range(16)]
            for d in order:
                for m in range(16):
                    if m & d:
                        continue
                    w = tws[d * h + j + (m & (d - 1)) * h]
                    u, v = x[m], x[m + d]
                    if inverse:
                        v = mmul(v, w, c)
                        x[m], x[m + d] = (u + v) % p, (u - v) % p
                    else:
                        x[m], x[m + d] = (u + v) % p, mmul((u - v) % p, w, c)
            for m in range(16):
                a[b + m * h] = x[m]
    return a


def test_radix16_pass_equals_four_stages():
    """The four top stages of a length-2^11 transform as one pass equal the
    radix-2 stages, forward and inverse."""
    rng = random.Random(78)
    c = prime_consts(PRIMES[2])
    n = 1 << 11
    tw, itw = tables(c, n)
    x = [rng.randrange(c["p"]) for _ in range(2 * n)]          # two transforms back to back
    p = c["p"]
    ref = list(x)
    length = n // 2
    while length >= n // 16:                                  # stages n/2 .. n/16
        for blk in range(0, len(ref), 2 * length):
            for j in range(length):
                u, v = ref[blk + j], ref[blk + j + length]
                ref[blk + j] = (u + v) % p
                ref[blk + j + length] = mmul((u - v) % p, tw[length + j], c)
        length //= 2
    assert pass16(x, n // 16, c, tw, False) == ref
    back = list(ref)
    length = n // 16
    while length < n:
        for blk in range(0, len(back), 2 * length):
            for j in range(length):
                u, v = back[blk + j], mmul(back[blk + j + length], itw[length + j], c)
                back[blk + j] = (u + v) % p
                back[blk + j + length] = (u - v) % p
        length *= 2
    assert pass16(ref, n // 16, c, itw, True) == back


def test_uncarried_square_would_pass_the_primes_range():
    """Why a node's square is carried into 32-bit words before its transform is
    kept for later products: the pointwise square of X^ stands for the
    uncarried coefficients of X*X (up to s 2^64 for s-word X), and their
    product with a k = 2s-word operand has columns up to 2s * s 2^64 * 2^32,
    beyond p1 p2 p3 already for s = 4 (so Garner's recombination would wrap);
    with carried words the columns stay below 2s 2^64."""
    M = PRIMES[0] * PRIMES[1] * PRIMES[2]
    for s in (4, 1024, 1 << 20):
        assert 2 * s * (s * (1 << 64)) * (1 << 32) > M
    assert 2 * (1 << 25) * (1 << 64) < M


# ---------------------------------------------------------------- carry scan model

CARRY_WORDS, CARRY_THREADS = 16, 256
CARRY_BLOCK = CARRY_WORDS * CARRY_THREADS


def lookahead_in(g, p, cin, bits):
    """Carry into each of `bits` positions and out of the top, for generate
    bits g and propagate bits p (disjoint): the bits of (a + g + cin) ^ a ^ g
    with a = g | p, as the kernels compute them with one addition."""
    a = g | p
    s = a + g + cin
    return (s ^ a ^ g) & ((1 << bits) - 1), (s >> bits) & 1


def carry_kernels(cols, addend, lo, hi):
    """The three carry kernels on one product: columns cols[j] (integers below
    2^96 as the recombination gives them), an addend (list of words), words
    [lo, hi) of sum_j cols[j] 2^(32 j) + addend returned."""
    n = len(cols)

    def word_sum(c):
        v = addend[c] if c < len(addend) else 0
        if 0 <= c < n:
            v += cols[c] & MASK
        if 0 <= c - 1 < n:
            v += (cols[c - 1] >> 32) & MASK
        if 0 <= c - 2 < n:
            v += cols[c - 2] >> 64
        return v

    nb = -(-hi // CARRY_BLOCK)
    # pass 1: per thread, words before inter-word carries and its masks
    words, masks = {}, {}
    for b in range(nb):
        for t in range(CARRY_THREADS):
            c0 = b * CARRY_BLOCK + t * CARRY_WORDS
            g = p = 0
            if c0 < hi:
                prev = (word_sum(c0 - 1) >> 32) if c0 >= 1 else 0
                for m in range(CARRY_WORDS):
                    s = word_sum(c0 + m)
                    v = (s & MASK) + prev
                    prev = s >> 32
                    assert prev <= 3 and v < (1 << 32) + 3
                    words[c0 + m] = v & MASK
                    g |= (v >> 32) << m
                    p |= (1 if v == MASK else 0) << m
            masks[b, t] = (g, p)

    def run_gp(g, p):
        a = g | p
        c0 = ((a + g) >> CARRY_WORDS) & 1
        c1 = ((a + g + 1) >> CARRY_WORDS) & 1
        return c0, c1 & (1 - c0)

    def block_carries(b, cin_block):
        """carry into each thread's run: lanes by one addition per warp, warps by one per block"""
        G = [run_gp(*masks[b, t])[0] for t in range(CARRY_THREADS)]
        P = [run_gp(*masks[b, t])[1] for t in range(CARRY_THREADS)]
        wg, wp, lane_bits = [], [], []
        for w in range(CARRY_THREADS // 32):
            gm = sum(G[32 * w + l] << l for l in range(32))
            pm = sum(P[32 * w + l] << l for l in range(32))
            a = gm | pm
            g0 = (a + gm) >> 32
            g1 = (a + gm + 1) >> 32
            wg.append(g0)
            wp.append(g1 & (1 - g0))
            lane_bits.append((gm, pm))
        bgm = sum(x << i for i, x in enumerate(wg))
        bpm = sum(x << i for i, x in enumerate(wp))
        nw = CARRY_THREADS // 32
        blk_g = ((bgm | bpm) + bgm) >> nw & 1
        blk_p = (((bgm | bpm) + bgm + 1) >> nw & 1) & (1 - blk_g)
        warp_in, _ = lookahead_in(bgm, bpm, cin_block, nw)
        into = []
        for w in range(nw):
            gm, pm = lane_bits[w]
            lane_in, _ = lookahead_in(gm, pm, (warp_in >> w) & 1, 32)
            into += [(lane_in >> l) & 1 for l in range(32)]
        return blk_g, blk_p, into

    # pass 2: the product's block carries, 32 blocks per step
    flags = [block_carries(b, 0)[:2] for b in range(nb)]
    cin_blocks, cin = [], 0
    for base in range(0, nb, 32):
        gm = sum(flags[b][0] << (b - base) for b in range(base, min(nb, base + 32)))
        pm = sum(flags[b][1] << (b - base) for b in range(base, min(nb, base + 32)))
        into, cin = lookahead_in(gm, pm, cin, 32)
        cin_blocks += [(into >> (b - base)) & 1 for b in range(base, min(nb, base + 32))]
    # pass 3: increments
    out = dict(words)
    for b in range(nb):
        _, _, tin = block_carries(b, cin_blocks[b])
        for t in range(CARRY_THREADS):
            g, p = masks[b, t]
            wi, _ = lookahead_in(g, p, tin[t], CARRY_WORDS)
            for m in range(CARRY_WORDS):
                c = b * CARRY_BLOCK + t * CARRY_WORDS + m
                if (wi >> m) & 1 and c in out:
                    out[c] = (out[c] + 1) & MASK
    return [out.get(c, 0) for c in range(lo, hi)]


@pytest.mark.parametrize("case", ["random", "ones", "ripple"])
def test_carry_kernels_equal_integer_sums(case):
    """The carry passes on columns below 2^96 (the recombination's range), with
    an addend and an output slice, equal the integer sum: random columns;
    columns that make long runs of all-ones words across thread, warp and
    block boundaries; a single carry rippling through 2.5 blocks."""
    rng = random.Random(hash(case) & 0xffff)
    n = 2 * CARRY_BLOCK + 1500
    if case == "random":
        cols = [rng.getrandbits(90) for _ in range(n)]
        addend = [rng.getrandbits(32) for _ in range(n + 1)]
    elif case == "ones":
        cols = [MASK if rng.random() < 0.97 else rng.getrandbits(33) for _ in range(n)]
        addend = [0] * (n + 1)
    else:
        cols = [MASK] * n
        cols[0] = MASK
        addend = [1]
    total = sum(c << (32 * j) for j, c in enumerate(cols)) + sum(a << (32 * j) for j, a in enumerate(addend))
    lo, hi = 37, n + 2
    got = carry_kernels(cols, addend, lo, hi)
    assert got == words(total >> (32 * lo), hi - lo)


def school_carry(cols, addend, lo, hi, threads=128):
    """The schoolbook kernel's carries for one product per CTA: thread t takes
    the run of r = ceil(hi / threads) words from t r, its generate/propagate
    bits combine within each warp and across the warps by one addition each."""
    n = len(cols)

    def word_sum(c):
        v = addend[c] if c < len(addend) else 0
        if 0 <= c < n:
            v += cols[c] & MASK
        if 0 <= c - 1 < n:
            v += (cols[c - 1] >> 32) & MASK
        if 0 <= c - 2 < n:
            v += cols[c - 2] >> 64
        return v

    r = -(-hi // threads)
    assert r <= 32
    runs = []
    for t in range(threads):
        c0, c1 = t * r, min(t * r + r, hi)
        prev = (word_sum(c0 - 1) >> 32) if 1 <= c0 <= hi else 0
        g = p = 0
        for c in range(c0, c1):
            s = word_sum(c)
            v = (s & MASK) + prev
            prev = s >> 32
            g |= (v >> 32) << (c - c0)
            p |= (1 if v == MASK else 0) << (c - c0)
        a = g | p
        G = ((a + g) >> r) & 1
        P = (((a + g + 1) >> r) & 1) & (1 - G)
        runs.append((c0, c1, g, p, G, P))
    nw = threads // 32
    warp_gp = []
    for w in range(nw):
        gm = sum(runs[32 * w + l][4] << l for l in range(32))
        pm = sum(runs[32 * w + l][5] << l for l in range(32))
        a = gm | pm
        g0 = (a + gm) >> 32
        warp_gp.append((g0, ((a + gm + 1) >> 32) & (1 - g0), gm, pm))
    bgm = sum(x[0] << i for i, x in enumerate(warp_gp))
    bpm = sum(x[1] << i for i, x in enumerate(warp_gp))
    warp_in, _ = lookahead_in(bgm, bpm, 0, nw)
    out = {}
    for w in range(nw):
        _, _, gm, pm = warp_gp[w]
        lane_in, _ = lookahead_in(gm, pm, (warp_in >> w) & 1, 32)
        for l in range(32):
            c0, c1, g, p, _, _ = runs[32 * w + l]
            into, _ = lookahead_in(g, p, (lane_in >> l) & 1, r)
            prev = (word_sum(c0 - 1) >> 32) if 1 <= c0 <= hi else 0
            for c in range(c0, c1):
                s = word_sum(c)
                out[c] = ((s & MASK) + prev + ((into >> (c - c0)) & 1)) & MASK
                prev = s >> 32
    return [out[c] for c in range(lo, hi)]


@pytest.mark.parametrize("nc,hi", [(130, 130), (512, 512), (1024, 1025), (2048, 2049)])
def test_school_carry_equals_integer_sums(nc, hi):
    """Schoolbook column sums (below 2^74 for products of up to 1024 words),
    random and all-ones heavy, with an addend one word longer than the product
    (the remainder step's shape), against the integer sum."""
    rng = random.Random(nc)
    for ones in (False, True):
        cols = [(MASK if ones and rng.random() < 0.95 else rng.getrandbits(74)) for _ in range(nc)]
        addend = [rng.getrandbits(32) for _ in range(hi)]
        total = sum(c << (32 * j) for j, c in enumerate(cols)) + sum(a << (32 * j) for j, a in enumerate(addend))
        got = school_carry(cols, addend, 3, hi)
        assert got == words(total >> 96, hi - 3)
