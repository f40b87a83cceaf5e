"""GPU parity of the tree form of the batch GCD (product and remainder trees,
products by three-prime number-theoretic transforms) against the oracle.

Exact comparison of every g_i and flag with oracle_batch_gcd_row: planted
sharing read off known factorisations, random odd moduli (many small common
factors) at counts that leave the trees ragged (padding leaves) and that
reach the transform path (products above 1024 words), invalid, short and
duplicate moduli, every leaf level of the remainder tree, the tree against
the scan over all rows at 6000 moduli, 2^17- and 2^20-modulus RSA-2048-shaped
scans (planted pairs, divisibility of every result, sampled rows against the
oracle; 2^20 is the size limit), the automatic choice and the host-buffer
form, and the errors.
"""
import numpy as np
import pytest

import bgcd_cases
import oracle
import workloads

pytestmark = pytest.mark.gpu

SCAN, TREE = 1, 2


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
    c = RsaContext(0, mem_budget_bytes=12 << 30)
    yield c
    c.close()


def gpu_gcd(torch, ctx, nbits, rows, method=TREE):
    rows = np.ascontiguousarray(rows, dtype=np.uint32)
    t = torch.from_numpy(rows.view(np.int32)).cuda()
    g, f = ctx.batch_gcd(nbits, t, method=method)
    torch.cuda.synchronize()
    return g.cpu().numpy().view(np.uint32).reshape(rows.shape), f.cpu().numpy()


def _random_odd(count, nbits, seed):
    vals = workloads.random_odd_halves(count, nbits, seed, ("tree", count))
    return workloads.ints_to_rows(vals, nbits // 32)


@pytest.mark.parametrize("nbits", [512, 1024, 2048])
def test_tree_constructed_sharing(torch_cuda, ctx, nbits):
    values, _, want, flags = bgcd_cases.constructed_case(seed=nbits)
    rows = workloads.ints_to_rows(values, nbits // 32)
    g, f = gpu_gcd(torch_cuda, ctx, nbits, rows)
    assert workloads.rows_to_ints(g) == want
    assert f.tolist() == flags


@pytest.mark.parametrize("nbits,count", [(512, 2), (512, 3), (512, 17), (512, 300), (1024, 33), (1024, 257),
                                         (1024, 1000), (2048, 2), (2048, 5), (2048, 100), (2048, 513)])
def test_tree_random_odd_matches_oracle(torch_cuda, ctx, nbits, count):
    rows = _random_odd(count, nbits, 5)
    g, f = gpu_gcd(torch_cuda, ctx, nbits, rows)
    og, of = oracle.batch_gcd(rows)
    assert np.array_equal(g, og)
    assert np.array_equal(f, of)


def test_tree_invalid_and_short_moduli(torch_cuda, ctx):
    rows = _random_odd(70, 1024, 9)
    vals = workloads.rows_to_ints(rows)
    vals[3] = 0
    vals[10] = 1
    p12 = vals[12] >> 600 | 1
    vals[12] = p12 * (vals[13] >> 600 | 1)
    vals[11] = 2 * p12 * (vals[14] >> 600 | 1)   # even: left out although it holds p12
    vals[20] = 3
    vals[21] = 9
    vals[30] = vals[31] >> 500 | 1               # leading zero limbs
    vals[40] = vals[41]                          # duplicate
    vals[69] = (1 << 1024) - 1                   # all-ones limbs
    rows = workloads.ints_to_rows(vals, 32)
    g, f = gpu_gcd(torch_cuda, ctx, 1024, rows)
    og, of = oracle.batch_gcd(rows)
    assert np.array_equal(g, og) and np.array_equal(f, of)
    assert f[3] == -1 and f[10] == -1 and f[11] == -1 and not g[3].any()
    assert f[40] == 2 and f[41] == 2 and f[20] != 0


@pytest.mark.parametrize("t0", ["0", "1", "3", "6"])
def test_tree_leaf_levels(torch_cuda, ctx, monkeypatch, t0):
    """The remainder tree stopped at every level (nodes of 1 .. 64 moduli)
    before the per-modulus reduction."""
    monkeypatch.setenv("RSAGPU_GCD_TREE_T0", t0)
    for nbits, count in ((2048, 300), (512, 5)):
        rows = _random_odd(count, nbits, 11)
        g, f = gpu_gcd(torch_cuda, ctx, nbits, rows)
        og, of = oracle.batch_gcd(rows)
        assert np.array_equal(g, og) and np.array_equal(f, of)


def test_tree_equals_scan(torch_cuda, ctx):
    """6000 1024-bit moduli: the tree's rows equal the scan's on every row (two
    independent GPU forms) and the oracle's on sampled rows."""
    rows = _random_odd(6000, 1024, 17)
    g, f = gpu_gcd(torch_cuda, ctx, 1024, rows, TREE)
    sg, sf = gpu_gcd(torch_cuda, ctx, 1024, rows, SCAN)
    assert np.array_equal(g, sg) and np.array_equal(f, sf)
    idx = [0, 1, 63, 64, 4095, 4096, 5999]
    og, of = oracle.batch_gcd(rows, rows=idx)
    assert np.array_equal(g[idx], og) and np.array_equal(f[idx], of)


def test_tree_large_weak_key_scan(torch_cuda, ctx):
    """131072 RSA-2048-shaped moduli (the tree's benchmark size): planted pairs
    are found, every g_i divides n_i and matches its flag, sampled rows equal
    the oracle's."""
    count = 1 << 17
    rows, pairs = workloads.weak_key_moduli(count)
    g, f = gpu_gcd(torch_cuda, ctx, 2048, rows)
    vals = workloads.rows_to_ints(rows)
    gs = workloads.rows_to_ints(g)
    for i, j in pairs:
        assert f[i] >= 1 and f[j] >= 1 and gs[i] > 1
    for k in range(count):
        assert gs[k] >= 1 and vals[k] % gs[k] == 0
        assert (f[k] == 0) == (gs[k] == 1) and (f[k] == 2) == (gs[k] == vals[k])
    rng = np.random.default_rng(4)
    idx = sorted(set(rng.choice(count, 6, replace=False).tolist()) | {0, count - 1, pairs[0][0], pairs[0][1]})
    og, of = oracle.batch_gcd(rows, rows=idx)
    assert np.array_equal(g[idx], og) and np.array_equal(f[idx], of)


def test_tree_largest_size(torch_cuda):
    """2^20 RSA-2048-shaped moduli, the tree's limit (2^26 modulus words:
    transforms of 2^27 words, the first prime's 2-adic order): planted pairs
    found, every g_i divides n_i and matches its flag, sampled rows equal the
    oracle's."""
    from paper_1407_1465_gb300 import RsaContext, rsa_batch_gcd_tree_bytes
    count = 1 << 20
    c = RsaContext(0, mem_budget_bytes=rsa_batch_gcd_tree_bytes(2048, count) + (2 << 30))
    try:
        rows, pairs = workloads.weak_key_moduli(count)
        g, f = gpu_gcd(torch_cuda, c, 2048, rows)
    finally:
        c.close()
    vals = workloads.rows_to_ints(rows)
    gs = workloads.rows_to_ints(g)
    for i, j in pairs:
        assert f[i] >= 1 and f[j] >= 1 and gs[i] > 1
    for k in range(count):
        assert gs[k] >= 1 and vals[k] % gs[k] == 0
        assert (f[k] == 0) == (gs[k] == 1) and (f[k] == 2) == (gs[k] == vals[k])
    idx = sorted({0, 1, count // 2, count - 1, pairs[0][0], pairs[0][1], pairs[-1][0], 777777})
    og, of = oracle.batch_gcd(rows, rows=idx)
    assert np.array_equal(g[idx], og) and np.array_equal(f[idx], of)


def test_tree_auto_choice_and_host_form(torch_cuda, ctx):
    """RSA_GCD_AUTO takes the tree from 2^18 modulus words (4096 2048-bit
    moduli, 16384 512-bit) when it fits the budget; the host-buffer form
    follows the same choice and equals both device forms."""
    from paper_1407_1465_gb300 import RsaContext, rsa_batch_gcd_method, rsa_batch_gcd_tree_bytes
    assert rsa_batch_gcd_method(ctx.handle, 2048, 4096) == TREE
    assert rsa_batch_gcd_method(ctx.handle, 2048, 4095) == SCAN
    assert rsa_batch_gcd_method(ctx.handle, 512, 16384) == TREE
    assert rsa_batch_gcd_method(ctx.handle, 512, 16383) == SCAN
    assert rsa_batch_gcd_method(ctx.handle, 512, 1) == SCAN
    small = RsaContext(0, mem_budget_bytes=rsa_batch_gcd_tree_bytes(2048, 32768) // 2)
    try:
        assert rsa_batch_gcd_method(small.handle, 2048, 32768) == SCAN
    finally:
        small.close()
    rows = _random_odd(33000, 512, 23)
    hg, hf = ctx.batch_gcd_host(512, rows)
    tg, tf = gpu_gcd(torch_cuda, ctx, 512, rows, TREE)
    sg, sf = gpu_gcd(torch_cuda, ctx, 512, rows, SCAN)
    assert np.array_equal(hg, tg) and np.array_equal(hf, tf)
    assert np.array_equal(tg, sg) and np.array_equal(tf, sf)
    idx = [0, 16383, 16384, 32767, 32999]
    og, of = oracle.batch_gcd(rows, rows=idx)
    assert np.array_equal(tg[idx], og) and np.array_equal(tf[idx], of)


def test_tree_degenerate_sets(torch_cuda, ctx):
    """One modulus (the product of the others is empty: g = 1, flag 0), only
    invalid moduli (every flag -1, zero rows), one valid among invalid ones."""
    n = 1000003 * 1000033
    for nbits in (512, 2048):
        L = nbits // 32
        for vals, want_g, want_f in (([n], [1], [0]), ([0, 1, 2, 4, 10], [0] * 5, [-1] * 5),
                                     ([6, n, 1000003 * 2], [0, 1, 0], [-1, 0, -1])):
            rows = workloads.ints_to_rows(vals, L)
            g, f = gpu_gcd(torch_cuda, ctx, nbits, rows)
            assert workloads.rows_to_ints(g) == want_g and f.tolist() == want_f
            og, of = oracle.batch_gcd(rows)
            assert np.array_equal(g, og) and np.array_equal(f, of)


def test_tree_errors(torch_cuda, ctx):
    from paper_1407_1465_gb300 import RsaError, rsa_batch_gcd_ex, rsa_batch_gcd_tree_bytes
    t = torch_cuda.zeros((4, 64), dtype=torch_cuda.int32, device="cuda")
    fl = torch_cuda.zeros(4, dtype=torch_cuda.int32, device="cuda")
    with pytest.raises(RsaError) as ei:
        rsa_batch_gcd_ex(ctx.handle, 2048, 4, t, None, fl, 7)
    assert ei.value.code == -1
    with pytest.raises(RsaError) as ei:
        rsa_batch_gcd_ex(ctx.handle, 2048, (1 << 20) + 1, t, None, fl, TREE)
    assert ei.value.code == -1
    with pytest.raises(RsaError) as ei:
        rsa_batch_gcd_tree_bytes(2048, (1 << 20) + 1)
    assert ei.value.code == -1
    assert rsa_batch_gcd_tree_bytes(2048, 1 << 20) > rsa_batch_gcd_tree_bytes(2048, 1 << 17)
    rsa_batch_gcd_ex(ctx.handle, 2048, 0, t, None, fl, TREE)       # empty: nothing to do
    g, f = gpu_gcd(torch_cuda, ctx, 2048, workloads.ints_to_rows([15, 21], 64))
    assert workloads.rows_to_ints(g) == [3, 3] and f.tolist() == [1, 1]
