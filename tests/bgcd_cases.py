"""Batch-GCD cases whose answers come from their construction, not from a gcd.

g_i = gcd(n_i, prod_{j != i, n_j valid} n_j); a modulus is valid when it is
odd and at least 3.  When the prime factorisation of every modulus is known,
g_i = prod_p p^min(v_p(n_i), v_p(prod of the others)), read off exponent
counts.  For tiny moduli the answer is found by brute force: the largest d
dividing both n_i and the exact product of the others.
"""
from __future__ import annotations

import math
import random
from collections import Counter

# 2^p - 1 is prime for these p (Mersenne primes, known independently of any test here)
MERSENNE = [(1 << p) - 1 for p in (61, 89, 107, 127)]


def trial_prime(n: int) -> bool:
    if n < 2:
        return False
    f = 2
    while f * f <= n:
        if n % f == 0:
            return False
        f += 1
    return True


def primes_from(lo: int, count: int) -> list[int]:
    out, n = [], lo | 1
    while len(out) < count:
        if trial_prime(n):
            out.append(n)
        n += 2
    return out


def valid(n: int) -> bool:
    return n % 2 == 1 and n >= 3


def flag_of(n: int, g: int) -> int:
    if not valid(n):
        return -1
    return 0 if g == 1 else (2 if g == n else 1)


def expected_from_factors(factors: list[list[int]], values: list[int]) -> list[int]:
    """factors[i]: the prime factors of values[i] with multiplicity ([] for an
    invalid value, whose factors never count)."""
    counts = [Counter(f) if valid(v) else Counter() for f, v in zip(factors, values)]
    total = Counter()
    for c in counts:
        total.update(c)
    out = []
    for c, v in zip(counts, values):
        if not valid(v):
            out.append(0)
            continue
        g = 1
        for p, e in c.items():
            g *= p ** min(e, total[p] - e)
        out.append(g)
    return out


def constructed_case(seed: int = 12):
    """Moduli from 21-bit primes (trial division) and Mersenne primes, with
    planted sharing: one shared prime, both primes shared with different
    moduli, a duplicate, a shared Mersenne prime, a prime square that shares
    with two moduli, and invalid entries (even, 1, 0) that hold primes of valid
    moduli and must not reveal them.  Returns (values, factors, g, flags)."""
    rng = random.Random(seed)
    pool = primes_from(1 << 20, 80)
    rng.shuffle(pool)
    facs = [[pool.pop(), pool.pop()] for _ in range(16)]
    facs.append([facs[0][0], pool.pop()])                 # shares one prime with modulus 0
    facs.append([facs[1][0], facs[2][1]])                 # both primes shared, with moduli 1 and 2
    facs.append(list(facs[3]))                            # duplicate of modulus 3
    facs.append([MERSENNE[0], MERSENNE[3]])               # 2^127 - 1 shared with the next
    facs.append([MERSENNE[1], MERSENNE[3]])
    facs.append([MERSENNE[2], pool.pop()])
    sq = pool.pop()
    facs.append([sq, sq])                                 # p^2, p in two more moduli: g = p^2
    facs.append([sq, pool.pop()])
    facs.append([sq, pool.pop()])
    q = pool.pop()
    facs.append([q, q, pool.pop()])                       # q^2 r with q once elsewhere: g = q
    facs.append([q, pool.pop()])
    values = [math.prod(f) for f in facs]
    # invalid entries carrying primes of moduli 4 and 5 (excluded: 4 and 5 stay coprime)
    values += [2 * facs[4][0], 1, 0, 4 * facs[5][1]]
    facs += [[2, facs[4][0]], [], [], [2, 2, facs[5][1]]]
    order = list(range(len(values)))
    rng.shuffle(order)
    values = [values[k] for k in order]
    facs = [facs[k] for k in order]
    g = expected_from_factors(facs, values)
    return values, facs, g, [flag_of(v, x) for v, x in zip(values, g)]


def brute_case(mods: list[int]):
    """(g, flags) by brute force on tiny moduli."""
    gs = []
    for i, n in enumerate(mods):
        if not valid(n):
            gs.append(0)
            continue
        P = math.prod(m for j, m in enumerate(mods) if j != i and valid(m))
        gs.append(max(d for d in range(1, n + 1) if n % d == 0 and P % d == 0))
    return gs, [flag_of(n, x) for n, x in zip(mods, gs)]


def brute_cases(seed: int = 3, trials: int = 40):
    rng = random.Random(seed)
    yield [3, 9, 15, 2, 5]                                # 3 is the smallest valid modulus
    yield [27, 9, 3]
    yield [7]
    for _ in range(trials):
        k = rng.randrange(1, 9)
        yield [rng.choice([0, 1, 2, 3]) if rng.random() < 0.15 else rng.randrange(3, 400) for _ in range(k)]
