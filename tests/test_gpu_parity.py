"""GPU parity: the CUDA path against the CPU oracle, element by element.

Every comparison is exact (the result of a modular exponentiation in [0, n)
is unique).  Inputs are seeded and synthetic (workloads.py); expected values
come from the oracle only.  Sizes: a few tiles with a ragged tail for every
key size and exponent kind, plus the full benchmark workloads (65536 RSA-2048
and 16384 RSA-4096 messages) checked on sampled rows against the oracle and
on every row through the invariant encrypt(decrypt(c)) = c.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

PUB, CRT, PLAIN = 0, 1, 2


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
    specs = [(1024, 0), (2048, 0), (3072, 0), (4096, 0)]
    ks = workloads.gen_keys(specs, workloads.DEFAULT_SEED)
    return {k.bits: k for k in ks}


@pytest.fixture(scope="module")
def kids(ctx, keys):
    return {b: ctx.keyload(b, k.n, k.e, k.d, k.p, k.q) for b, k in keys.items()}


def run(torch, ctx, kid, kind, rows):
    rows = np.ascontiguousarray(rows, dtype=np.uint32)
    t = torch.from_numpy(rows.view(np.int32)).cuda()
    out = torch.empty_like(t)
    st = torch.full((rows.shape[0],), 99, dtype=torch.int32, device="cuda")
    ctx.modexp_key(kid, kind, t, out, st)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32).reshape(rows.shape), st.cpu().numpy()


def expect(key, kind, rows, threads=0):
    if kind == PUB:
        return oracle.modexp_batch(rows, key.e, key.n, threads=threads)
    if kind == CRT:
        return oracle.crt_batch(rows, key.d, key.p, key.q, threads=threads)
    return oracle.modexp_batch(rows, key.d, key.n, threads=threads)


# ------------------------------------------------------------------ single-limb (paper's toy key)

def test_toy_key_4096_packets(torch_cuda, ctx):
    t = workloads
    kid = ctx.keyload(32, t.TOY_N, t.TOY_E, t.TOY_D, t.TOY_P, t.TOY_Q)
    packets = t.toy_packets(4096).reshape(-1, 1)
    enc, st = run(torch_cuda, ctx, kid, PUB, packets)
    assert (st == 0).all()
    want_enc = np.array([[oracle.modexp(int(m), t.TOY_E, t.TOY_N)] for m in packets[:, 0]], dtype=np.uint32)
    assert np.array_equal(enc, want_enc)
    for kind in (PLAIN, CRT):
        dec, st = run(torch_cuda, ctx, kid, kind, enc)
        want = np.array([[oracle.modexp(int(c), t.TOY_D, t.TOY_N)] for c in enc[:, 0]], dtype=np.uint32)
        assert np.array_equal(dec, want)
    # the printed d does not invert e; the corrected one round-trips the paper's packets
    kid2 = ctx.keyload(32, t.TOY_N, t.TOY_E, t.TOY_D_CORRECTED, t.TOY_P, t.TOY_Q)
    pk = np.array(t.PAPER_PACKETS, dtype=np.uint32).reshape(-1, 1)
    c, _ = run(torch_cuda, ctx, kid2, PUB, pk)
    for kind in (PLAIN, CRT):
        back, _ = run(torch_cuda, ctx, kid2, kind, c)
        assert np.array_equal(back, pk)


# ------------------------------------------------------------------ multi-limb, small counts

@pytest.mark.parametrize("bits", [1024, 2048, 3072, 4096])
@pytest.mark.parametrize("count", [1, 32, 77])
def test_crt_parity(torch_cuda, ctx, keys, kids, bits, count):
    key = keys[bits]
    rows = workloads.messages_below(key.n, count, 5, ("crt", bits, count))
    got, st = run(torch_cuda, ctx, kids[bits], CRT, rows)
    assert (st == 0).all()
    assert np.array_equal(got, expect(key, CRT, rows))
    if count == 77 and bits <= 2048:   # also against the plain definition c^d mod n
        plain = oracle.modexp_batch(rows[:16], key.d, key.n)
        assert np.array_equal(got[:16], plain)


@pytest.mark.parametrize("bits", [1024, 2048, 3072, 4096])
@pytest.mark.parametrize("kind", [PUB, PLAIN])
def test_full_modulus_parity(torch_cuda, ctx, keys, kids, bits, kind):
    key = keys[bits]
    rows = workloads.messages_below(key.n, 45, 6, ("full", bits, kind))
    got, st = run(torch_cuda, ctx, kids[bits], kind, rows)
    assert (st == 0).all()
    assert np.array_equal(got, expect(key, kind, rows))


def _edge_rows(key):
    n, L = key.n, key.limbs
    vals = [0, 1, 2, 3, n - 1, n - 2, key.p, key.q, 2 * key.p, key.p * 5 % n, key.q * 7 % n,
            (1 << (key.bits - 1)), (1 << (key.bits - 1)) - 1, n // 2, (1 << 32) - 1]
    bad = [n, n + 1, (1 << key.bits) - 1]
    return workloads.ints_to_rows(vals, L), workloads.ints_to_rows(bad, L)


@pytest.mark.parametrize("bits", [1024, 2048, 4096])
def test_edge_messages(torch_cuda, ctx, keys, kids, bits):
    key = keys[bits]
    good, bad = _edge_rows(key)
    rows = np.concatenate([good, bad])
    kinds = [CRT, PUB] + ([PLAIN] if bits <= 2048 else [])
    for kind in kinds:
        got, st = run(torch_cuda, ctx, kids[bits], kind, rows)
        ng = good.shape[0]
        assert (st[:ng] == 0).all() and (st[ng:] == -3).all()
        assert np.array_equal(got[:ng], expect(key, kind, good))
        assert not got[ng:].any()


def test_window_and_launch_shapes(torch_cuda, ctx, keys, kids):
    key = keys[2048]
    rows = workloads.messages_below(key.n, 200, 8, "shapes")
    want = expect(key, CRT, rows)
    try:
        for variant in (1, 2):
            for w in (3, 4, 5, 6):
                for warps, cps in ((2, 0), (4, 1), (8, 0)):
                    ctx.set_tuning(2048, CRT, window=w, warps_per_cta=warps, ctas_per_sm=cps, variant=variant)
                    got, _ = run(torch_cuda, ctx, kids[2048], CRT, rows)
                    assert np.array_equal(got, want), (variant, w, warps, cps)
        # the separated squaring on 1024-bit keys too (16-limb halves), and for the plain exponent
        key1 = keys[1024]
        rows1 = workloads.messages_below(key1.n, 70, 8, "shapes1024")
        for kind in (CRT, PLAIN):
            ctx.set_tuning(1024, kind, variant=2)
            got, _ = run(torch_cuda, ctx, kids[1024], kind, rows1)
            assert np.array_equal(got, expect(key1, kind, rows1)), kind
            ctx.set_tuning(1024, kind, reset=True)
    finally:
        ctx.set_tuning(2048, CRT, reset=True)


def test_in_place_and_host_api(torch_cuda, ctx, keys, kids):
    key = keys[2048]
    rows = workloads.messages_below(key.n, 70, 9, "inplace")
    want = expect(key, CRT, rows)
    t = torch_cuda.from_numpy(rows.view(np.int32)).cuda()
    ctx.modexp_key(kids[2048], CRT, t, t)
    torch_cuda.cuda.synchronize()
    assert np.array_equal(t.cpu().numpy().view(np.uint32), want)
    st = np.zeros(70, dtype=np.int32)
    out = ctx.modexp_key_host(kids[2048], CRT, rows, status=st)
    assert np.array_equal(out, want) and (st == 0).all()


def test_errors_are_status_codes(torch_cuda, ctx, keys):
    from paper_1407_1465_gb300 import RsaError
    key = keys[1024]
    pub_only = ctx.keyload(1024, key.n, key.e)
    rows = workloads.messages_below(key.n, 4, 1, "err")
    t = torch_cuda.from_numpy(rows.view(np.int32)).cuda()
    for kind in (CRT, PLAIN):
        with pytest.raises(RsaError) as ei:
            ctx.modexp_key(pub_only, kind, t)
        assert ei.value.code == -2
    with pytest.raises(RsaError) as ei:
        ctx.modexp_key(9999, PUB, t)
    assert ei.value.code == -2
    with pytest.raises(RsaError):
        ctx.modexp_key(pub_only, 7, t)
    ctx.keyunload(pub_only)


# ------------------------------------------------------------------ full benchmark sizes

def test_full_rsa2048_workload(torch_cuda, ctx, keys, kids):
    """65536 RSA-2048 messages under the default launch shape."""
    key = keys[2048]
    rows = workloads.messages_below(key.n, 65536, workloads.DEFAULT_SEED, ("single", 2048))
    dec, st = run(torch_cuda, ctx, kids[2048], CRT, rows)
    assert (st == 0).all()
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(rows.shape[0], 192, replace=False))
    idx = np.concatenate([[0, 31, 32, rows.shape[0] - 1], idx])
    assert np.array_equal(dec[idx], expect(key, CRT, rows[idx]))
    enc, st = run(torch_cuda, ctx, kids[2048], PUB, dec)    # encrypt(decrypt(c)) = c, every row
    assert (st == 0).all() and np.array_equal(enc, rows)


def test_full_rsa4096_workload(torch_cuda, ctx, keys, kids):
    key = keys[4096]
    rows = workloads.messages_below(key.n, 16384, workloads.DEFAULT_SEED, ("single", 4096))
    dec, st = run(torch_cuda, ctx, kids[4096], CRT, rows)
    assert (st == 0).all()
    rng = np.random.default_rng(2)
    idx = np.sort(rng.choice(rows.shape[0], 48, replace=False))
    idx = np.concatenate([[0, rows.shape[0] - 1], idx])
    assert np.array_equal(dec[idx], expect(key, CRT, rows[idx]))
    back = oracle.modexp_batch(dec, key.e, key.n)            # every row, through the oracle
    assert np.array_equal(back, rows)


def test_autotune_installs_a_working_shape(torch_cuda, ctx, keys, kids, tmp_path):
    from paper_1407_1465_gb300 import rsa_autotune
    key = keys[2048]
    cache = str(tmp_path / "tune.txt")
    best = rsa_autotune(ctx.handle, kids[2048], CRT, 4096, cache)
    assert best["ms"] > 0 and 3 <= best["window"] <= 6 and best["warps_per_cta"] in (2, 4, 8)
    assert ctx.get_tuning(2048, CRT)["window"] == best["window"]
    again = rsa_autotune(ctx.handle, kids[2048], CRT, 4096, cache)     # served from the cache file
    assert again["ms"] == pytest.approx(best["ms"], rel=1e-9)
    assert {k: again[k] for k in again if k != "ms"} == {k: best[k] for k in best if k != "ms"}
    rows = workloads.messages_below(key.n, 100, 12, "tuned")
    got, st = run(torch_cuda, ctx, kids[2048], CRT, rows)
    assert (st == 0).all() and np.array_equal(got, expect(key, CRT, rows))
    ctx.set_tuning(2048, CRT, reset=True)


@pytest.mark.parametrize("tpo", [2, 4])
@pytest.mark.parametrize("bits", [2048, 3072, 4096])
def test_lanes_per_operation_crt(torch_cuda, ctx, keys, kids, bits, tpo):
    """One operation spread over 2 or 4 lanes (warp-shuffle carries) gives the
    same results; counts leave a ragged last tile."""
    key = keys[bits]
    good, bad = _edge_rows(key)
    rows = np.concatenate([workloads.messages_below(key.n, 45, 21, ("tpo", bits, tpo)), good, bad])
    ng = rows.shape[0] - bad.shape[0]
    want = expect(key, CRT, rows[:ng])
    try:
        for w in ((4, 5) if bits == 2048 else (4, 5, 6)):
            ctx.set_tuning(bits, CRT, window=w, threads_per_op=tpo)
            got, st = run(torch_cuda, ctx, kids[bits], CRT, rows)
            assert (st[:ng] == 0).all() and (st[ng:] == -3).all()
            assert np.array_equal(got[:ng], want), (bits, tpo, w)
            assert not got[ng:].any()
    finally:
        ctx.set_tuning(bits, CRT, reset=True)


@pytest.mark.parametrize("tpo", [2, 4])
@pytest.mark.parametrize("bits", [2048, 3072, 4096])
def test_lanes_per_operation_public(torch_cuda, ctx, keys, kids, bits, tpo):
    key = keys[bits]
    good, bad = _edge_rows(key)
    rows = np.concatenate([workloads.messages_below(key.n, 37, 22, ("tpo-pub", bits, tpo)), good, bad])
    ng = rows.shape[0] - bad.shape[0]
    try:
        ctx.set_tuning(bits, PUB, threads_per_op=tpo)
        got, st = run(torch_cuda, ctx, kids[bits], PUB, rows)
        assert (st[:ng] == 0).all() and (st[ng:] == -3).all()
        assert np.array_equal(got[:ng], expect(key, PUB, rows[:ng]))
        assert not got[ng:].any()
    finally:
        ctx.set_tuning(bits, PUB, reset=True)


@pytest.mark.parametrize("bits", [1024, 2048])
def test_public_sliding_window_long_exponents(torch_cuda, ctx, keys, bits):
    """Long public exponents: the sliding-window method (Fig. 7, windows 4..6)
    and the binary method (Fig. 5) both equal the oracle; short windows and an
    exponent whose top window is shorter than w are covered by the exponent set."""
    key = keys[bits]
    rng = np.random.default_rng(bits + 17)
    exps = [(1 << (bits - 1)) | int.from_bytes(rng.bytes(bits // 8), "little") % (1 << (bits - 1)) | 1,
            (1 << 200) + 1, 3, 0b1000000000000000000000000000000000000000000000000000000000000000000000101]
    rows = workloads.messages_below(key.n, 45, 61, ("slide", bits))
    for e in exps:
        kid = ctx.keyload(bits, key.n, e)
        want = oracle.modexp_batch(rows, e, key.n)
        try:
            for variant, window in ((1, 0), (2, 4), (2, 5), (2, 6), (0, 0)):
                ctx.set_tuning(bits, PUB, variant=variant, window=window)
                got, st = run(torch_cuda, ctx, kid, PUB, rows)
                assert (st == 0).all()
                assert np.array_equal(got, want), (e.bit_length(), variant, window)
        finally:
            ctx.set_tuning(bits, PUB, reset=True)
            ctx.keyunload(kid)
