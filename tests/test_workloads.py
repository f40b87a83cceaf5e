"""The seeded input generators (shared by both sides of every parity test).

SplitMix64 is pinned to its published reference outputs; the batch-GCD
moduli, random halves and messages are checked for the structure the
workloads promise.
"""
import math

import numpy as np

import workloads


def test_splitmix64_reference_vector():
    """Steele, Lea and Flood's SplitMix64 from state 1234567: the first five
    outputs of the reference generator."""
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
            16408922859458223821]
    key = 1234567
    scalar = [workloads._mix64((key + (i + 1) * workloads.GAMMA) & workloads.MASK64) for i in range(5)]
    assert scalar == want
    assert workloads.draws(key, 0, 5).tolist() == want
    st = workloads.Stream(key)
    assert [st.u64() for _ in range(5)] == want
    # counter form: any window of the stream without generating what precedes it
    assert workloads.draws_at(key, np.array([4, 0], dtype=np.uint64)).tolist() == [want[4], want[0]]


def test_random_odd_halves_shape():
    vals = workloads.random_odd_halves(64, 1024, 7, "t")
    assert len(set(vals)) == 64
    for v in vals:
        assert v % 2 == 1 and v.bit_length() == 1024 and (v >> 1022) == 3
    assert vals == workloads.random_odd_halves(64, 1024, 7, "t")          # seeded
    assert vals != workloads.random_odd_halves(64, 1024, 8, "t")


def test_weak_key_moduli_structure():
    rows, pairs = workloads.weak_key_moduli(count=300, bits=2048, seed=11, shared=5)
    assert rows.shape == (300, 64) and rows.dtype == np.uint32
    vals = workloads.rows_to_ints(rows)
    assert all(v % 2 == 1 and v.bit_length() == 2048 for v in vals)
    assert len(pairs) == 5 and len({x for p in pairs for x in p}) == 10
    for i, j in pairs:
        g = math.gcd(vals[i], vals[j])
        assert g.bit_length() >= 1023                                     # the planted 1024-bit factor
    again, pairs2 = workloads.weak_key_moduli(count=300, bits=2048, seed=11, shared=5)
    assert np.array_equal(rows, again) and pairs == pairs2


def test_messages_below_modulus():
    n = (1 << 2047) + 12345
    rows = workloads.messages_below(n, 500, 3, "t")
    vals = workloads.rows_to_ints(rows)
    assert all(0 <= v < n for v in vals)
    assert max(vals).bit_length() == 2048 or max(vals) > n // 2           # spans the range
    assert np.array_equal(rows, workloads.messages_below(n, 500, 3, "t"))
