"""GPU parity of the batch GCD (weak-key detection), scan form, against the oracle.

Exact comparison of every g_i and flag: planted sharing read off known
factorisations (small moduli in wide limb slots, leading zero limbs), real
RSA moduli with planted shared primes, random odd moduli (many small common
factors) at counts that leave ragged warps, blocks and parts, invalid moduli,
each block size and occupancy variant, and the 16384-modulus RSA-2048
benchmark workload (sampled rows against the oracle, planted pairs and
divisibility of every result).
"""
import numpy as np
import pytest

import bgcd_cases
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
    c = RsaContext(0, mem_budget_bytes=8 << 30)
    yield c
    c.close()


def gpu_gcd(torch, ctx, nbits, rows):
    """The scan form (RSA_GCD_SCAN); the tree form has its own tests."""
    rows = np.ascontiguousarray(rows, dtype=np.uint32)
    t = torch.from_numpy(rows.view(np.int32)).cuda()
    g, f = ctx.batch_gcd(nbits, t, method=1)
    torch.cuda.synchronize()
    return g.cpu().numpy().view(np.uint32).reshape(rows.shape), f.cpu().numpy()


@pytest.mark.parametrize("nbits", [512, 1024, 2048])
def test_bgcd_constructed_sharing(torch_cuda, ctx, nbits):
    values, _, want, flags = bgcd_cases.constructed_case(seed=nbits)
    rows = workloads.ints_to_rows(values, nbits // 32)
    g, f = gpu_gcd(torch_cuda, ctx, nbits, rows)
    assert workloads.rows_to_ints(g) == want
    assert f.tolist() == flags


def test_bgcd_rsa_moduli_planted_primes(torch_cuda, ctx):
    """Real 1024- and 2048-bit RSA moduli (Miller-Rabin primes); moduli 40..
    reuse primes of earlier keys."""
    for bits, nkeys in ((1024, 48), (2048, 24)):
        keys = workloads.gen_keys([(bits, i) for i in range(nkeys)], 777, mr_rounds=8)
        facs = [[k.p, k.q] for k in keys]
        facs += [[keys[0].p, keys[1].q], [keys[2].p, keys[3].p], [keys[4].p, keys[4].q]]
        values = [a * b for a, b in facs]
        want = bgcd_cases.expected_from_factors(facs, values)
        rows = workloads.ints_to_rows(values, bits // 32)
        g, f = gpu_gcd(torch_cuda, ctx, bits, rows)
        assert workloads.rows_to_ints(g) == want
        assert f.tolist() == [bgcd_cases.flag_of(v, x) for v, x in zip(values, want)]
        assert (f[5:nkeys] == 0).all()


def _random_odd(count, nbits, seed):
    vals = workloads.random_odd_halves(count, nbits, seed, ("gpu", count))
    return workloads.ints_to_rows(vals, nbits // 32)


@pytest.mark.parametrize("nbits,count", [(512, 1), (512, 2), (512, 15), (512, 17), (512, 300),
                                         (1024, 16), (1024, 31), (1024, 33), (1024, 257), (1024, 1000),
                                         (2048, 32), (2048, 100), (2048, 513)])
def test_bgcd_random_odd_matches_oracle(torch_cuda, ctx, nbits, count):
    rows = _random_odd(count, nbits, 5)
    g, f = gpu_gcd(torch_cuda, ctx, nbits, rows)
    og, of = oracle.batch_gcd(rows)
    assert np.array_equal(g, og)
    assert np.array_equal(f, of)
    if count >= 100:
        assert (of == 1).any() or (of == 2).any()   # small common factors appear


def test_bgcd_invalid_and_short_moduli(torch_cuda, ctx):
    rows = _random_odd(70, 1024, 9)
    vals = workloads.rows_to_ints(rows)
    vals[3] = 0
    vals[10] = 1
    p12 = vals[12] >> 600 | 1                    # modulus 12 = p12 * r; an even entry holds p12
    vals[12] = p12 * (vals[13] >> 600 | 1)
    vals[11] = 2 * p12 * (vals[14] >> 600 | 1)
    vals[20] = 3
    vals[21] = 9
    vals[30] = vals[31] >> 500 | 1               # short modulus, leading zero limbs
    vals[40] = vals[41]                          # duplicate
    rows = workloads.ints_to_rows(vals, 32)
    g, f = gpu_gcd(torch_cuda, ctx, 1024, rows)
    og, of = oracle.batch_gcd(rows)
    assert np.array_equal(g, og) and np.array_equal(f, of)
    assert f[3] == -1 and f[10] == -1 and f[11] == -1 and not g[3].any()
    assert f[40] == 2 and f[41] == 2 and f[20] != 0


@pytest.mark.parametrize("block,minb", [("8", "3"), ("32", "3"), ("16", "2"), ("32", "2"), ("8", "2")])
def test_bgcd_block_sizes_agree(torch_cuda, ctx, monkeypatch, block, minb):
    """Every block size and both register variants."""
    monkeypatch.setenv("RSAGPU_GCD_BLOCK", block)
    monkeypatch.setenv("RSAGPU_GCD_MINB", minb)
    rows = _random_odd(450, 2048, 13)
    g, f = gpu_gcd(torch_cuda, ctx, 2048, rows)
    og, of = oracle.batch_gcd(rows)
    assert np.array_equal(g, og) and np.array_equal(f, of)


def test_bgcd_errors(torch_cuda, ctx):
    from paper_1407_1465_gb300 import RsaError, rsa_batch_gcd
    t = torch_cuda.zeros((4, 64), dtype=torch_cuda.int32, device="cuda")
    fl = torch_cuda.zeros(4, dtype=torch_cuda.int32, device="cuda")
    with pytest.raises(RsaError) as ei:
        rsa_batch_gcd(ctx.handle, 4096, 4, t, None, fl)
    assert ei.value.code == -7
    with pytest.raises(RsaError) as ei:
        rsa_batch_gcd(ctx.handle, 2048, 4, t, None, None)
    assert ei.value.code == -1
    with pytest.raises(RsaError) as ei:
        rsa_batch_gcd(ctx.handle, 2048, 3, t.view(-1)[1:].reshape(-1)[:3 * 64], None, fl)
    assert ei.value.code == -1
    rsa_batch_gcd(ctx.handle, 2048, 0, t, None, fl)           # empty batch: nothing to do


def test_bgcd_full_weak_key_workload(torch_cuda, ctx):
    """16384 RSA-2048-shaped moduli, the benchmark's launch: planted pairs are
    found, every g_i divides n_i and (for flags 1) is a proper factor, sampled
    rows equal the oracle's."""
    rows, pairs = workloads.weak_key_moduli()
    g, f = gpu_gcd(torch_cuda, ctx, 2048, rows)
    vals = workloads.rows_to_ints(rows)
    gs = workloads.rows_to_ints(g)
    for i, j in pairs:
        assert f[i] >= 1 and f[j] >= 1
        assert gs[i] % 2 == 1 and gs[i] > 1
    for k in range(len(vals)):
        assert gs[k] >= 1 and vals[k] % gs[k] == 0
        assert (f[k] == 0) == (gs[k] == 1) and (f[k] == 2) == (gs[k] == vals[k])
    rng = np.random.default_rng(8)
    idx = sorted(set(rng.choice(len(vals), 20, replace=False).tolist()) | {0, 31, 32, len(vals) - 1}
                 | {pairs[0][0], pairs[0][1]})
    og, of = oracle.batch_gcd(rows, rows=idx)
    assert np.array_equal(g[idx], og) and np.array_equal(f[idx], of)


def test_bgcd_host_buffers(torch_cuda, ctx):
    """rsa_batch_gcd_host: host moduli in, host gcds and flags out, equal to the
    device form and to the oracle; either output may be left out."""
    from paper_1407_1465_gb300 import rsa_batch_gcd_host
    rows = _random_odd(333, 1024, 21)
    g = np.zeros_like(rows)
    f = np.zeros(rows.shape[0], dtype=np.int32)
    rsa_batch_gcd_host(ctx.handle, 1024, rows.shape[0], rows, g, f)
    og, of = oracle.batch_gcd(rows)
    assert np.array_equal(g, og) and np.array_equal(f, of)
    f2 = np.full(rows.shape[0], 99, dtype=np.int32)
    rsa_batch_gcd_host(ctx.handle, 1024, rows.shape[0], rows, None, f2)
    assert np.array_equal(f2, of)
    dg, df = gpu_gcd(torch_cuda, ctx, 1024, rows)
    assert np.array_equal(dg, g) and np.array_equal(df, f)
    hg, hf = ctx.batch_gcd_host(1024, rows)                  # the context method
    assert np.array_equal(hg, g) and np.array_equal(hf, f)
