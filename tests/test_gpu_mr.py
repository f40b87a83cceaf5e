"""GPU: batch Miller-Rabin (key generation) against the oracle's Miller-Rabin.

Candidates at 512, 1024 and 2048 bits (the last: RSA-4096 key generation): primes from seeded key generation, products of
two primes (RSA moduli of the half size), squares of primes, seeded random odd
numbers (almost all composite), Mersenne numbers below the size (2^127 - 1 and
2^521 - 1 prime, 2^67 - 1 composite but a strong probable prime to base 2),
small Carmichael numbers and 2047 in full-width rows, and invalid candidates
(even, below 5).  The verdict of every candidate must equal the oracle's with
the same bases.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def ctx(torch_cuda):
    from paper_1407_1465_gb300 import RsaContext, build
    build.build()
    c = RsaContext(0, mem_budget_bytes=4 << 30)
    yield c
    c.close()


def _candidates(bits):
    L = bits // 32
    rng = np.random.default_rng(bits)
    full = workloads.gen_keys([(2 * bits, 0), (2 * bits, 1)], workloads.DEFAULT_SEED)
    half = workloads.gen_keys([(bits, 0), (bits, 1)], workloads.DEFAULT_SEED)
    primes = [k.p for k in full] + [k.q for k in full]
    cands = list(primes)
    cands += [k.n for k in half] + [k.p * k.p for k in half]
    cands += [int.from_bytes(rng.bytes(bits // 8), "little") | 1 | (1 << (bits - 1)) for _ in range(40)]
    cands += [(1 << 127) - 1, (1 << 67) - 1, 2047, 561, 1729, 8911]
    if bits >= 1024:
        cands.append((1 << 521) - 1)
    if bits >= 2048:
        cands.append((1 << 1279) - 1)               # a Mersenne prime
    cands += [10, 3, 1 << 40]                        # invalid: even or below 5
    return cands


@pytest.mark.parametrize("bits", [512, 1024, 2048])
def test_mr_batch_matches_oracle(torch_cuda, ctx, bits):
    L = bits // 32
    cands = _candidates(bits)
    rounds = 3
    rng = np.random.default_rng(bits + 1)
    bases = []
    for n in cands:
        row = []
        for r in range(rounds):
            if n < 5:
                row.append(2)
            elif n in (2047, (1 << 67) - 1) and r == 0:
                row.append(2)                          # the strong-pseudoprime base
            else:
                row.append(2 + int.from_bytes(rng.bytes(bits // 8 + 1), "little") % (n - 3))
        bases.append(row)
    crow = workloads.ints_to_rows(cands, L)
    brow = np.stack([workloads.ints_to_rows(r, L) for r in bases])
    want = np.array([oracle.miller_rabin(int(n), b) if n % 2 and n >= 5 else -1 for n, b in zip(cands, bases)],
                    dtype=np.int32)
    t = torch_cuda
    v = ctx.miller_rabin(bits, t.from_numpy(crow.view(np.int32)).cuda(), t.from_numpy(brow.view(np.int32)).cuda())
    t.cuda.synchronize()
    got = v.cpu().numpy()
    assert np.array_equal(got, want)
    # the generated primes pass, their products fail, the invalid rows are flagged
    assert (got[:4] == 1).all() and (got[4:6] == 0).all() and (got[-3:] == -1).all()
    # base 2 alone: 2047 and 2^67 - 1 pass (strong pseudoprimes), base 3 exposes them
    for n in (2047, (1 << 67) - 1):
        for b, expect in ((2, 1), (3, 0)):
            c1 = t.from_numpy(workloads.ints_to_rows([n], L).view(np.int32)).cuda()
            b1 = t.from_numpy(workloads.ints_to_rows([b], L).reshape(1, 1, L).view(np.int32)).cuda()
            r = ctx.miller_rabin(bits, c1, b1)
            t.cuda.synchronize()
            assert int(r.cpu()[0]) == expect == oracle.miller_rabin(n, [b])
