"""Pins of the CPU oracle to facts that do not come from the oracle itself.

Sources of truth used here:
  - values the paper prints (Fig. 4 trace, Fig. 2 key, Sec. 2 toy key/packets);
  - brute force (repeated multiplication, Fig. 4) on small exponents;
  - Python's built-in arbitrary-precision integers (``pow``, ``divmod``,
    ``*``) -- an independent implementation, used only as a reference;
  - closed forms and invariants: 0^x, 1^x, (n-1)^x, Fermat's little theorem,
    multiplicativity, decrypt(encrypt(m)) = m, CRT = plain definition.
"""
import random

import numpy as np
import pytest

import oracle
import workloads
from conftest import read_golden


def test_fig4_trace(oracle_lib):
    g = read_golden("fig4_naive_trace.txt")
    assert oracle.naive_trace(g["g"], g["e"], g["m"]) == g["trace"]
    for method in ("l2r", "r2l", "naive"):
        assert oracle.modexp(g["g"], g["e"], g["m"], method) == 445
    for k in range(1, 7):
        assert oracle.modexp(g["g"], g["e"], g["m"], "kary", k=k) == 445
        assert oracle.modexp(g["g"], g["e"], g["m"], "sliding", k=k) == 445


def test_fig2_key_roundtrip_every_message(oracle_lib):
    k = read_golden("fig2_key.txt")
    assert k["p"] * k["q"] == k["n"] and (k["p"] - 1) * (k["q"] - 1) == k["phi"]
    assert (k["e"] * k["d"]) % k["phi"] == 1
    for m in range(k["n"]):
        c = oracle.modexp(m, k["e"], k["n"])
        assert oracle.modexp(c, k["d"], k["n"]) == m
        assert oracle.crt_decrypt(c, k["d"], k["p"], k["q"]) == m


def test_toy_key_as_printed_and_corrected(oracle_lib):
    t = read_golden("toy_key.txt")
    n, e, d = t["n"], t["e"], t["d"]
    phi = (t["p"] - 1) * (t["q"] - 1)
    assert t["p"] * t["q"] == n
    # the printed pair is not an RSA inverse: e*d mod phi(n) = 267, not 1 (Sec. 2 example)
    assert (e * d) % phi == 267
    d_fix = workloads.TOY_D_CORRECTED
    assert (e * d_fix) % phi == 1
    packets = t["packets"]
    cts = [oracle.modexp(m, e, n) for m in packets]
    # brute-force pin: 130 / 136 repeated multiplications
    assert cts == [oracle.modexp(m, e, n, "naive") for m in packets]
    assert [oracle.modexp(c, d_fix, n) for c in cts] == packets
    roundtrip_printed = [oracle.modexp(c, d, n) for c in cts]
    assert roundtrip_printed != packets
    assert roundtrip_printed == [oracle.modexp(c, d, n, "naive") for c in cts]


def test_brute_force_small_exponents(oracle_lib):
    rng = random.Random(1)
    for _ in range(300):
        nl = rng.choice([1, 2, 3])
        m = rng.getrandbits(32 * nl) | 1
        if m < 3:
            continue
        g = rng.randrange(m)
        e = rng.randrange(0, 300)
        want = oracle.modexp(g, e, m, "naive")
        for method in ("l2r", "r2l"):
            assert oracle.modexp(g, e, m, method) == want
        assert want == pow(g, e, m)


@pytest.mark.parametrize("nlimbs", [1, 2, 3, 7, 16, 32, 48, 64, 128])
def test_against_python_pow(oracle_lib, nlimbs):
    rng = random.Random(nlimbs)
    reps = 6 if nlimbs >= 64 else 20
    for _ in range(reps):
        m = rng.getrandbits(32 * nlimbs) | 1 | (1 << (32 * nlimbs - 1))
        g = rng.randrange(m)
        e = rng.getrandbits(rng.choice([1, 17, 64, 32 * nlimbs if nlimbs <= 16 else 256]))
        assert oracle.modexp(g, e, m) == pow(g, e, m)


def test_methods_agree_tiny(oracle_lib):
    rng = random.Random(7)
    for _ in range(400):
        m = rng.randrange(3, 1 << 40) | 1
        g = rng.randrange(m)
        e = rng.randrange(1, 1 << 20)
        ref = pow(g, e, m)
        assert oracle.modexp(g, e, m, "l2r") == ref
        assert oracle.modexp(g, e, m, "r2l") == ref
        k = rng.randrange(1, 7)
        assert oracle.modexp(g, e, m, "kary", k=k) == ref
        assert oracle.modexp(g, e, m, "sliding", k=k) == ref


def test_mul_and_divmod_against_python(oracle_lib):
    rng = random.Random(3)
    special = [0, 1, 2, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFE, 0xFFFFFFFF]
    for _ in range(3000):
        nu, nv = rng.randrange(1, 9), rng.randrange(1, 6)
        if rng.random() < 0.6:
            limbs_u = [rng.choice(special) for _ in range(nu)]
            limbs_v = [rng.choice(special) for _ in range(nv)]
            u = sum(x << (32 * i) for i, x in enumerate(limbs_u))
            v = sum(x << (32 * i) for i, x in enumerate(limbs_v))
        else:
            u, v = rng.getrandbits(32 * nu), rng.getrandbits(32 * nv)
        if v == 0:
            continue
        assert oracle.mul(u, v) == u * v
        assert oracle.divmod_(u, v) == divmod(u, v)


def test_divmod_add_back_cases(oracle_lib):
    """Inputs where the two-limb quotient estimate is still one too large
    (Algorithm D step D6): u = q*v + r with the top limbs chosen so the
    estimate from u's top two limbs over v's top limb overshoots."""
    rng = random.Random(11)
    hits = 0
    for _ in range(4000):
        vtop = 0x80000000 | rng.getrandbits(16)
        v = (vtop << 64) | (0xFFFFFFFF << 32) | rng.getrandbits(32)
        q = rng.getrandbits(32)
        r = rng.randrange(v)
        u = q * v + r
        assert oracle.divmod_(u, v) == (q, r)
        # estimate from the top limbs of u against v's top two limbs
        top = u >> 64
        qhat = min(top // vtop, 0xFFFFFFFF)
        if qhat > q + 1:
            hits += 1
    assert hits >= 0  # the equality above is the pin; hits only reports coverage


def test_closed_forms(oracle_lib):
    rng = random.Random(5)
    for _ in range(60):
        nl = rng.choice([1, 4, 32])
        n = rng.getrandbits(32 * nl) | 1 | (1 << (32 * nl - 1))
        x = rng.getrandbits(64) | 1
        assert oracle.modexp(0, x, n) == 0
        assert oracle.modexp(1, x, n) == 1
        assert oracle.modexp(n - 1, x, n) == n - 1           # x odd
        assert oracle.modexp(n - 1, x + 1, n) == 1            # even exponent
        g = rng.randrange(n)
        assert oracle.modexp(g, 1, n) == g
        assert oracle.modexp(g, 0, n) == 1


def test_fermat_on_generated_primes(oracle_lib):
    st = workloads.Stream(workloads.stream_key(9, "fermat"))
    for bits in (64, 128, 512):
        p = workloads.gen_prime(bits, st, mr_rounds=20)
        for _ in range(5):
            a = 2 + st.below(p - 3)
            assert oracle.modexp(a, p - 1, p) == 1


def test_multiplicativity(oracle_lib):
    rng = random.Random(13)
    for nl in (2, 16):
        n = rng.getrandbits(32 * nl) | 1 | (1 << (32 * nl - 1))
        for _ in range(10):
            a, b = rng.randrange(n), rng.randrange(n)
            e = rng.getrandbits(64)
            lhs = oracle.modexp((a * b) % n, e, n)
            rhs = (oracle.modexp(a, e, n) * oracle.modexp(b, e, n)) % n
            assert lhs == rhs


def test_crt_equals_plain_and_roundtrip(oracle_lib):
    for bits in (128, 256, 1024):
        key = workloads.gen_key(bits, seed=21, index=bits, mr_rounds=20)
        msgs = workloads.messages_below(key.n, 12, 21, ("crt", bits))
        for m in workloads.rows_to_ints(msgs):
            c = oracle.modexp(m, key.e, key.n)
            mp = oracle.modexp(c, key.d, key.n)
            assert mp == m
            assert oracle.crt_decrypt(c, key.d, key.p, key.q) == m
        # c = 0 mod p and c = 0 mod q edge cases
        for c in (key.p, key.q, 2 * key.p % key.n, 0, 1, key.n - 1):
            assert oracle.crt_decrypt(c, key.d, key.p, key.q) == pow(c, key.d, key.n)


def test_batch_driver_matches_scalar(oracle_lib):
    key = workloads.gen_key(512, seed=4, index=0, mr_rounds=20)
    msgs = workloads.messages_below(key.n, 37, 4, "batch")
    out_plain = oracle.modexp_batch(msgs, key.d, key.n, threads=3)
    out_crt = oracle.crt_batch(msgs, key.d, key.p, key.q, threads=5)
    ints = workloads.rows_to_ints(msgs)
    want = [pow(m, key.d, key.n) for m in ints]
    assert workloads.rows_to_ints(out_plain) == want
    assert workloads.rows_to_ints(out_crt) == want


# ------------------------------------------------------------------ Miller-Rabin (key generation, Fig. 1)

def _trial_division_prime(n):
    if n < 2:
        return False
    f = 2
    while f * f <= n:
        if n % f == 0:
            return False
        f += 1
    return True


def test_miller_rabin_matches_trial_division_small(oracle_lib):
    """Bases 2, 3, 5, 7 decide primality exactly below 3 215 031 751."""
    for n in range(5, 6000, 2):
        bases = [b for b in (2, 3, 5, 7) if b <= n - 2]
        assert oracle.miller_rabin(n, bases) == int(_trial_division_prime(n)), n


def test_miller_rabin_strong_pseudoprimes_and_carmichael(oracle_lib):
    # 2047 = 23 * 89 is the smallest strong pseudoprime to base 2: base 2 passes, base 3 does not
    assert oracle.miller_rabin(2047, [2]) == 1
    assert oracle.miller_rabin(2047, [3]) == 0
    # Carmichael numbers fool the Fermat test for every coprime base but not Miller-Rabin base 2
    for n in (561, 1105, 1729, 2465, 2821, 6601, 8911):
        assert oracle.miller_rabin(n, [2]) == 0, n
    # F5 = 2^32 + 1 = 641 * 6700417 and 2^67 - 1 = 193707721 * 761838257287 are composite
    assert oracle.miller_rabin((1 << 32) + 1, [3]) == 0
    assert 193707721 * 761838257287 == (1 << 67) - 1
    assert oracle.miller_rabin((1 << 67) - 1, [3, 5]) == 0
    # but 2^p - 1 (p prime) always passes base 2: 2^p = 1 (mod n); a strong-pseudoprime pin
    assert oracle.miller_rabin((1 << 67) - 1, [2]) == 1
    # even and tiny inputs are rejected
    assert oracle.miller_rabin(10, [3]) == -1 and oracle.miller_rabin(3, [2]) == -1


def test_miller_rabin_mersenne_primes(oracle_lib):
    """2^127 - 1, 2^521 - 1 and 2^607 - 1 are prime: every base passes."""
    rng = np.random.default_rng(11)
    for p in (127, 521, 607):
        n = (1 << p) - 1
        bases = [2 + int.from_bytes(rng.bytes(p // 8 + 1), "little") % (n - 3) for _ in range(6)]
        assert oracle.miller_rabin(n, bases) == 1, p
    # and a product of two of them is not
    n = ((1 << 127) - 1) * ((1 << 521) - 1)
    assert oracle.miller_rabin(n, [2, 3]) == 0


# ------------------------------------------------------------------ batch GCD (weak-key detection)

def _ints_rows(vals, L):
    return workloads.ints_to_rows(vals, L)


def test_batch_gcd_constructed_sharing(oracle_lib):
    """Planted shared primes (21-bit primes and Mersenne primes, a duplicate, a
    prime square, invalid entries holding primes of valid moduli): every g_i
    equals the value read off the known factorisations."""
    import bgcd_cases
    values, _, want, flags = bgcd_cases.constructed_case()
    L = 8                                                  # 2^127-1 squared-scale moduli fit 256 bits
    assert max(values).bit_length() <= 32 * L
    g, f = oracle.batch_gcd(_ints_rows(values, L), threads=3)
    assert workloads.rows_to_ints(g) == want
    assert f.tolist() == flags
    assert sorted(set(flags)) == [-1, 0, 1, 2]


def test_batch_gcd_brute_force_tiny(oracle_lib):
    """Tiny moduli: the largest common divisor of n_i and the exact product of
    the others, found by scanning every candidate divisor."""
    import bgcd_cases
    for mods in bgcd_cases.brute_cases():
        want, flags = bgcd_cases.brute_case(mods)
        g, f = oracle.batch_gcd(_ints_rows(mods, 1), threads=2)
        assert workloads.rows_to_ints(g) == want, mods
        assert f.tolist() == flags, mods


def test_batch_gcd_special_cases(oracle_lib):
    # one modulus: the product of the others is empty (1), so g = 1
    g, f = oracle.batch_gcd(_ints_rows([MERSENNE_127 := (1 << 127) - 1], 4))
    assert workloads.rows_to_ints(g) == [1] and f.tolist() == [0]
    # every other modulus invalid: still g = 1
    g, f = oracle.batch_gcd(_ints_rows([MERSENNE_127, 0, 2, 1, 1 << 100], 4))
    assert workloads.rows_to_ints(g) == [1, 0, 0, 0, 0] and f.tolist() == [0, -1, -1, -1, -1]
    # selected rows come back in the order asked for
    vals = [15, 21, 35, 143]
    g, f = oracle.batch_gcd(_ints_rows(vals, 1), rows=[3, 0])
    assert workloads.rows_to_ints(g) == [1, 15] and f.tolist() == [0, 2]
