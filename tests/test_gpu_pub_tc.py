"""GPU parity of the RSA-2048 public exponent on the tensor cores.

A 2048-bit modulus has the shape of an RSA-4096 prime, so x^e mod n runs the
two-round tensor-core Montgomery products of the RSA-4096 CRT path (binary
method, Fig. 5, over the key's e).  Exact comparison with the oracle, element by
element: counts that leave partial tiles of 128 and CTAs with one tile, the
exponent 65537, a 100-bit and a 2047-bit exponent, edge messages (0, 1, 2,
n - 1) and messages >= n (RSA_ERR_RANGE, zeroed rows); the automatic choice
(the tensor cores from 4096 operations, the CUDA-core kernel below), told apart
by the bounded MMA waits, which only the tensor-core path has: with a zero poll
budget its operations report RSA_ERR_TIMEOUT.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

PUB = 0
TC, CIOS = 3, 1
RSA_ERR_RANGE, RSA_ERR_TIMEOUT = -3, -6


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


@pytest.fixture(scope="module")
def key():
    return workloads.gen_keys([(2048, 0)], workloads.DEFAULT_SEED)[0]


def run(torch, ctx, kid, rows, variant):
    ctx.set_tuning(2048, PUB, variant=variant)
    try:
        rows = np.ascontiguousarray(rows, dtype=np.uint32)
        t = torch.from_numpy(rows.view(np.int32)).cuda()
        out = torch.empty_like(t)
        st = torch.full((rows.shape[0],), 99, dtype=torch.int32, device="cuda")
        ctx.modexp_key(kid, PUB, t, out, st)
        torch.cuda.synchronize()
        return out.cpu().numpy().view(np.uint32).reshape(rows.shape), st.cpu().numpy()
    finally:
        ctx.set_tuning(2048, PUB, reset=True)


@pytest.mark.parametrize("count", [1, 77, 129, 300, 1000])
def test_pub_tc_parity_e65537(torch_cuda, ctx, key, count):
    kid = ctx.keyload(2048, key.n, key.e)
    try:
        rows = workloads.messages_below(key.n, count, 7, ("pub-tc", count))
        got, st = run(torch_cuda, ctx, kid, rows, TC)
        assert (st == 0).all()
        assert np.array_equal(got, oracle.modexp_batch(rows, key.e, key.n))
    finally:
        ctx.keyunload(kid)


@pytest.mark.parametrize("ebits", [100, 2047])
def test_pub_tc_long_exponents(torch_cuda, ctx, key, ebits):
    rng = np.random.default_rng(ebits)
    e = int.from_bytes(rng.bytes((ebits + 7) // 8), "little") % (1 << ebits) | (1 << (ebits - 1)) | 1
    kid = ctx.keyload(2048, key.n, e)
    try:
        rows = workloads.messages_below(key.n, 150, 9, ("pub-tc-long", ebits))
        got, st = run(torch_cuda, ctx, kid, rows, TC)
        assert (st == 0).all()
        assert np.array_equal(got, oracle.modexp_batch(rows, e, key.n))
    finally:
        ctx.keyunload(kid)


def test_pub_tc_edge_messages(torch_cuda, ctx, key):
    kid = ctx.keyload(2048, key.n, key.e, key.d, key.p, key.q)
    try:
        good = [0, 1, 2, key.n - 1, key.p, 3 * key.q]
        bad = [key.n, key.n + 1, (1 << 2048) - 1]
        rows = workloads.ints_to_rows(good + bad, 64)
        got, st = run(torch_cuda, ctx, kid, rows, TC)
        assert list(st) == [0] * len(good) + [RSA_ERR_RANGE] * len(bad)
        assert np.array_equal(got[:len(good)], oracle.modexp_batch(rows[:len(good)], key.e, key.n))
        assert not got[len(good):].any()
    finally:
        ctx.keyunload(kid)


def test_pub_tc_automatic_choice_and_timeout(torch_cuda, ctx, key, monkeypatch):
    """From 4096 operations the automatic choice runs the tensor-core kernel
    (every status RSA_ERR_TIMEOUT under a zero poll budget, rows zeroed),
    below it the CUDA-core kernel (unaffected by the budget); both equal the
    oracle on sampled rows and each other on every row; the context keeps
    working after the timeouts."""
    kid = ctx.keyload(2048, key.n, key.e)
    try:
        big = workloads.messages_below(key.n, 4096 + 37, 11, ("pub-tc-auto",))
        small = big[:4000]
        auto_big, st = run(torch_cuda, ctx, kid, big, 0)
        assert (st == 0).all()
        cios_big, st = run(torch_cuda, ctx, kid, big, CIOS)
        assert (st == 0).all() and np.array_equal(auto_big, cios_big)
        idx = [0, 127, 128, 4095, 4096, 4096 + 36]
        assert np.array_equal(auto_big[idx], oracle.modexp_batch(big[idx], key.e, key.n))
        monkeypatch.setenv("RSAGPU_TC_WAIT_POLLS", "0")
        got, st = run(torch_cuda, ctx, kid, big, 0)
        assert (st == RSA_ERR_TIMEOUT).all() and not got.any()
        got, st = run(torch_cuda, ctx, kid, small, 0)
        assert (st == 0).all() and np.array_equal(got, cios_big[:4000])
        monkeypatch.delenv("RSAGPU_TC_WAIT_POLLS")
        got, st = run(torch_cuda, ctx, kid, big, 0)
        assert (st == 0).all() and np.array_equal(got, cios_big)
    finally:
        ctx.keyunload(kid)
