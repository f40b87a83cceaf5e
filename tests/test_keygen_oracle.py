"""The benchmark keys pass the oracle's own primality test.

The input generators (workloads.py) must not import the oracle, so their key
recipe runs its own Miller-Rabin with Python's built-in modular power (40
rounds after a sieve by the primes below 2^16; key generation, Fig. 1).  This
test re-checks what that recipe produced with the oracle's Miller-Rabin
(binary modexp and the test's definition), 40 seeded bases per prime, and the
key relations of Fig. 1 (n = pq of exactly the stated size, e d = 1 mod phi).
"""
import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle
import workloads


def _bases(p, rounds, tag):
    st = workloads.Stream(workloads.stream_key(workloads.DEFAULT_SEED, "mr-check", tag))
    return [2 + st.below(p - 3) for _ in range(rounds)]


def _check_key(key, rounds=40):
    assert key.p * key.q == key.n and key.n.bit_length() == key.bits
    assert key.p.bit_length() == key.q.bit_length() == key.bits // 2 and key.p > key.q
    phi = (key.p - 1) * (key.q - 1)
    assert (key.e * key.d) % phi == 1 and math.gcd(key.e, phi) == 1
    for which, prime in (("p", key.p), ("q", key.q)):
        assert oracle.miller_rabin(prime, _bases(prime, rounds, (key.bits, which, key.n % 1000003))) == 1
    # and the oracle calls n itself composite
    assert oracle.miller_rabin(key.n, _bases(key.n, 4, (key.bits, "n"))) == 0


def test_benchmark_keys_pass_the_oracle_miller_rabin():
    keys = [workloads.rsa_single(2048, 1)[0], workloads.rsa_single(4096, 1)[0]]
    with ThreadPoolExecutor(max_workers=2) as ex:
        list(ex.map(_check_key, keys))


def test_ragged_keys_pass_the_oracle_miller_rabin():
    rb_keys = workloads.gen_keys(workloads.ragged_key_specs(256, workloads.DEFAULT_SEED), workloads.DEFAULT_SEED)
    # one key of each size present in the mix (the first of each), 40 rounds per prime
    picked = {}
    for k in rb_keys:
        picked.setdefault(k.bits, k)
    assert sorted(picked) == [1024, 2048, 3072, 4096]
    with ThreadPoolExecutor(max_workers=4) as ex:
        list(ex.map(_check_key, picked.values()))
    sizes = np.array([k.bits for k in rb_keys])
    assert len(set(k.n for k in rb_keys)) == 256 and set(sizes.tolist()) <= {1024, 2048, 3072, 4096}
