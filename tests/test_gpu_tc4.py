"""GPU parity of the RSA-3072/4096 tensor-core CRT path (variant 3 at 3072 and
4096 bits) against the oracle.

The Montgomery reduction modulo each 1536- or 2048-bit prime runs on the
tensor cores in two rounds of half the prime size (crt_tc4.cu).  Exact comparison, element by
element, at windows 3 and 4 for counts that leave ragged tiles of 128
operations and CTAs with one tile; edge messages (0, 1, n-1, p, q, multiples
of p, q) and messages >= n, which must come back as RSA_ERR_RANGE with zeroed
rows; the bounded MMA waits; and the 16384-ciphertext workload (sampled rows
against the oracle, every row against the four-lane CUDA-core path).
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

PUB, CRT = 0, 1
TC = 3


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
    c = RsaContext(0, mem_budget_bytes=8 << 30)
    yield c
    c.close()


@pytest.fixture(scope="module", params=[3072, 4096])
def key(request):
    return workloads.gen_keys([(request.param, 0)], workloads.DEFAULT_SEED)[0]


@pytest.fixture(scope="module")
def kid(ctx, key):
    k = ctx.keyload(key.bits, key.n, key.e, key.d, key.p, key.q)
    yield k
    ctx.keyunload(k)


def run(torch, ctx, bits, kid, rows, variant, window=0, tpo=0):
    ctx.set_tuning(bits, CRT, variant=variant, window=window, threads_per_op=tpo)
    try:
        rows = np.ascontiguousarray(rows, dtype=np.uint32)
        t = torch.from_numpy(rows.view(np.int32)).cuda()
        out = torch.empty_like(t)
        st = torch.full((rows.shape[0],), 99, dtype=torch.int32, device="cuda")
        ctx.modexp_key(kid, CRT, t, out, st)
        torch.cuda.synchronize()
        return out.cpu().numpy().view(np.uint32).reshape(rows.shape), st.cpu().numpy()
    finally:
        ctx.set_tuning(bits, CRT, reset=True)


@pytest.mark.parametrize("window", [3, 4])
@pytest.mark.parametrize("count", [1, 77, 129, 300])
def test_tc4_crt_parity(torch_cuda, ctx, key, kid, count, window):
    rows = workloads.messages_below(key.n, count, 5, ("tc4", key.bits, count, window))
    got, st = run(torch_cuda, ctx, key.bits, kid, rows, TC, window)
    assert (st == 0).all()
    assert np.array_equal(got, oracle.crt_batch(rows, key.d, key.p, key.q))


def test_tc4_edge_messages(torch_cuda, ctx, key, kid):
    n, p, q = key.n, key.p, key.q
    half = key.bits // 2
    good = [0, 1, 2, 3, n - 1, n - 2, p, q, 2 * p, 3 * q, p * 5 % n, (1 << (key.bits - 1)), n // 2, (1 << 32) - 1,
            (1 << half) - 1, 1 << half]
    bad = [n, n + 1, (1 << key.bits) - 1]
    rows = workloads.ints_to_rows(good + bad, key.limbs)
    got, st = run(torch_cuda, ctx, key.bits, kid, rows, TC, 3)
    ng = len(good)
    assert (st[:ng] == 0).all() and (st[ng:] == -3).all()
    assert np.array_equal(got[:ng], oracle.crt_batch(rows[:ng], key.d, key.p, key.q))
    assert not got[ng:].any()


def test_tc4_full_workload(torch_cuda, ctx, key, kid):
    """16384 ciphertexts (the RSA-4096 benchmark batch at 4096 bits): every row
    equals the four-lane CUDA-core path's, sampled rows the oracle's."""
    k2, rows = workloads.rsa_single(key.bits, 16384)
    assert k2.n == key.n
    got, st = run(torch_cuda, ctx, key.bits, kid, rows, TC, 3)
    assert (st == 0).all()
    ref, st2 = run(torch_cuda, ctx, key.bits, kid, rows, 1, 5, 4)
    assert (st2 == 0).all() and np.array_equal(got, ref)
    idx = np.arange(0, rows.shape[0], 2731)
    assert np.array_equal(got[idx], oracle.crt_batch(rows[idx], key.d, key.p, key.q))


def test_tc4_wait_timeout_reports_status(torch_cuda, ctx, key, kid, monkeypatch):
    """With a poll budget of 0 every MMA wait gives up at once: each operation
    comes back as RSA_ERR_TIMEOUT with a zeroed row, and the context works
    normally afterwards."""
    rows = workloads.messages_below(key.n, 150, 41, ("tc4_timeout", key.bits))
    monkeypatch.setenv("RSAGPU_TC_WAIT_POLLS", "0")
    got, st = run(torch_cuda, ctx, key.bits, kid, rows, TC, 3)
    assert (st == -6).all() and not got.any()
    monkeypatch.delenv("RSAGPU_TC_WAIT_POLLS")
    got, st = run(torch_cuda, ctx, key.bits, kid, rows[:40], TC, 3)
    assert (st == 0).all()
    assert np.array_equal(got, oracle.crt_batch(rows[:40], key.d, key.p, key.q))
