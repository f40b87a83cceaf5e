"""GPU parity of the tensor-core CRT path (variant 3, RSA-2048) against the oracle.

Exact comparison, element by element, for counts that leave ragged tiles of
128 operations and CTAs with fewer than three tiles; edge messages (0, 1,
n-1, p, q, multiples of p, and messages >= n that must be rejected); the
full 65536-message benchmark workload (sampled rows against the oracle, every
row against the CUDA-core CRT path and through encrypt(decrypt(c)) = c).
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


@pytest.fixture(scope="module")
def keys():
    ks = workloads.gen_keys([(2048, 0), (2048, 1), (4096, 0)], workloads.DEFAULT_SEED)
    return ks


def run(torch, ctx, kid, kind, rows, variant, window=0):
    ctx.set_tuning(2048, kind, variant=variant, window=window)
    try:
        rows = np.ascontiguousarray(rows, dtype=np.uint32)
        t = torch.from_numpy(rows.view(np.int32)).cuda()
        out = torch.empty_like(t)
        st = torch.full((rows.shape[0],), 99, dtype=torch.int32, device="cuda")
        ctx.modexp_key(kid, kind, t, out, st)
        torch.cuda.synchronize()
        return out.cpu().numpy().view(np.uint32).reshape(rows.shape), st.cpu().numpy()
    finally:
        ctx.set_tuning(2048, kind, reset=True)


@pytest.mark.parametrize("window", [3, 4])
@pytest.mark.parametrize("count", [1, 77, 128, 129, 513, 1000])
def test_tc_crt_parity(torch_cuda, ctx, keys, count, window):
    key = keys[0]
    kid = ctx.keyload(2048, key.n, key.e, key.d, key.p, key.q)
    rows = workloads.messages_below(key.n, count, 31, ("tc", count))
    got, st = run(torch_cuda, ctx, kid, CRT, rows, TC, window)
    assert (st == 0).all()
    assert np.array_equal(got, oracle.crt_batch(rows, key.d, key.p, key.q))
    ctx.keyunload(kid)


def test_tc_edge_messages(torch_cuda, ctx, keys):
    for key in keys[:2]:
        kid = ctx.keyload(2048, key.n, key.e, key.d, key.p, key.q)
        n, L = key.n, key.limbs
        vals = [0, 1, 2, n - 1, n - 2, key.p, key.q, 2 * key.p, key.q * 7 % n, key.p - 1, key.q + 1,
                (1 << 2047), (1 << 2047) - 1, n // 2, (1 << 1024) - 1, 1 << 1024, (1 << 32) - 1]
        bad = [n, n + 1, (1 << 2048) - 1]
        rows = np.concatenate([workloads.ints_to_rows(vals, L), workloads.ints_to_rows(bad, L)])
        got, st = run(torch_cuda, ctx, kid, CRT, rows, TC, 3 if key is keys[1] else 4)
        ng = len(vals)
        assert (st[:ng] == 0).all() and (st[ng:] == -3).all()
        assert np.array_equal(got[:ng], oracle.crt_batch(rows[:ng], key.d, key.p, key.q))
        assert not got[ng:].any()
        ctx.keyunload(kid)


def test_tc_full_rsa2048_workload(torch_cuda, ctx, keys):
    """65536 messages: several tiles per tile slot, the benchmark's launch."""
    key = keys[0]
    kid = ctx.keyload(2048, key.n, key.e, key.d, key.p, key.q)
    rows = workloads.messages_below(key.n, 65536, workloads.DEFAULT_SEED, ("single", 2048))
    dec, st = run(torch_cuda, ctx, kid, CRT, rows, TC)
    assert (st == 0).all()
    rng = np.random.default_rng(3)
    idx = np.sort(rng.choice(rows.shape[0], 192, replace=False))
    idx = np.concatenate([[0, 127, 128, 383, 384, rows.shape[0] - 1], idx])
    assert np.array_equal(dec[idx], oracle.crt_batch(rows[idx], key.d, key.p, key.q))
    ref, st2 = run(torch_cuda, ctx, kid, CRT, rows, 1)          # CUDA-core CIOS path, every row
    assert (st2 == 0).all() and np.array_equal(dec, ref)
    enc, st3 = run(torch_cuda, ctx, kid, PUB, dec, 0)           # encrypt(decrypt(c)) = c, every row
    assert (st3 == 0).all() and np.array_equal(enc, rows)
    ctx.keyunload(kid)


def test_tc_rejects_other_sizes(torch_cuda, ctx, keys):
    """The tensor-core path serves 2048-, 3072- and 4096-bit CRT; 1024-bit keys are refused."""
    from paper_1407_1465_gb300 import RsaError
    key = workloads.gen_keys([(1024, 0)], workloads.DEFAULT_SEED)[0]
    kid = ctx.keyload(1024, key.n, key.e, key.d, key.p, key.q)
    rows = workloads.messages_below(key.n, 4, 9, ("tc1024",))
    ctx.set_tuning(1024, CRT, variant=TC)
    try:
        t = torch_cuda.from_numpy(rows.view(np.int32)).cuda()
        with pytest.raises(RsaError) as ei:
            ctx.modexp_key(kid, CRT, t, torch_cuda.empty_like(t))
        assert ei.value.code == -7
    finally:
        ctx.set_tuning(1024, CRT, reset=True)
        ctx.keyunload(kid)


def test_tc_wait_timeout_reports_status(torch_cuda, ctx, keys, monkeypatch):
    """The kernel's waits on MMA completion are bounded.  With a poll budget of
    0 every wait gives up at once: each operation must come back as
    RSA_ERR_TIMEOUT (-6) with a zeroed row, the launch must end by itself, and
    the context must work normally afterwards."""
    key = keys[0]
    kid = ctx.keyload(2048, key.n, key.e, key.d, key.p, key.q)
    rows = workloads.messages_below(key.n, 300, 41, ("tc_timeout",))
    monkeypatch.setenv("RSAGPU_TC_WAIT_POLLS", "0")
    got, st = run(torch_cuda, ctx, kid, CRT, rows, TC)
    assert (st == -6).all() and not got.any()
    monkeypatch.delenv("RSAGPU_TC_WAIT_POLLS")
    got, st = run(torch_cuda, ctx, kid, CRT, rows, TC)
    assert (st == 0).all()
    assert np.array_equal(got, oracle.crt_batch(rows, key.d, key.p, key.q))
    ctx.keyunload(kid)
