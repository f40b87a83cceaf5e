"""Ragged multi-key batches (rsa_modexp_batch) against the oracle.

Mixed key sizes (single-limb, 1024-4096 bits), all exponent kinds, shuffled
order and a packed message buffer addressed by per-operation limb offsets;
every result is compared with the oracle, with the same operation run alone
through rsa_modexp_key, and invalid operations must come back as status codes
without disturbing the others.  The full ragged workload (256 keys, 200000
operations) is checked on sampled operations.
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


def expect_one(key, kind, row):
    m = workloads.limbs_to_int(row)
    n_limbs = row.size
    if kind == PUB:
        v = oracle.modexp(m, key.e, key.n)
    elif kind == CRT and n_limbs > 1:
        v = oracle.crt_decrypt(m, key.d, key.p, key.q)
    else:
        v = oracle.modexp(m, key.d, key.n)
    return workloads.int_to_limbs(v, n_limbs)


class ToyKey:
    bits, n, e, d, p, q = 32, workloads.TOY_N, workloads.TOY_E, workloads.TOY_D, workloads.TOY_P, workloads.TOY_Q


def build_mix(keys, kids, count, seed):
    """A shuffled mix of operations over the given keys; returns device-ready arrays."""
    st = workloads.Stream(workloads.stream_key(seed, "mix"))
    ops = []
    for i in range(count):
        k = st.below(len(keys))
        key = keys[k]
        kinds = [PUB, CRT, PLAIN]
        kind = kinds[st.below(len(kinds))]
        if key.bits == 32:
            row = np.array([st.below(key.n)], dtype=np.uint32)
        else:
            row = workloads.messages_below(key.n, 1, seed, ("mix", i))[0]
        ops.append((k, kind, row))
    sizes = [max(4, r.size) if r.size > 1 else 1 for _, _, r in ops]
    offsets, pos = [], 0
    for s in sizes:
        pos = (pos + 3) // 4 * 4 if s > 1 else pos
        offsets.append(pos)
        pos += s
    packed = np.zeros(pos + 4, dtype=np.uint32)
    for (k, kind, row), off in zip(ops, offsets):
        packed[off:off + row.size] = row
    key_ids = np.array([kids[k] for k, _, _ in ops], dtype=np.int32)
    sels = np.array([kind for _, kind, _ in ops], dtype=np.uint8)
    return ops, key_ids, sels, np.array(offsets, dtype=np.uint64), packed


def run_batch(torch, ctx, key_ids, sels, offsets, packed):
    dev = "cuda"
    k = torch.from_numpy(key_ids).to(dev)
    s = torch.from_numpy(sels).to(dev)
    o = torch.from_numpy(offsets.view(np.int64)).to(dev)
    m = torch.from_numpy(packed.view(np.int32)).to(dev)
    out = torch.full_like(m, -1)
    st = torch.full((key_ids.size,), 99, dtype=torch.int32, device=dev)
    ctx.modexp_batch(k, s, o, m, out, st)
    rc = ctx.sync()
    return out.cpu().numpy().view(np.uint32), st.cpu().numpy(), rc


@pytest.fixture(scope="module")
def mixed_keys(ctx):
    ks = workloads.gen_keys([(1024, 0), (2048, 0), (3072, 0), (4096, 0)], workloads.DEFAULT_SEED)
    keys = [ToyKey()] + ks
    kids = [ctx.keyload(k.bits, k.n, k.e, k.d, k.p, k.q) for k in keys]
    return keys, kids


@pytest.mark.parametrize("wide", ["100", "100/16", "0"])
@pytest.mark.parametrize("count", [1, 63, 700])
def test_ragged_mix_matches_oracle(torch_cuda, ctx, mixed_keys, monkeypatch, count, wide):
    """Small batches run 2048/4096-bit CRT with 4/8 lanes per operation
    (RSAGPU_RAGGED_WIDE_PCT=100, the default; "100/16": 4096-bit CRT on 16
    lanes); 0 forces one/four lanes."""
    pct, _, lanes = wide.partition("/")
    monkeypatch.setenv("RSAGPU_RAGGED_WIDE_PCT", pct)
    monkeypatch.setenv("RSAGPU_RAGGED_LANES_4096", lanes or "8")
    keys, kids = mixed_keys
    ops, key_ids, sels, offsets, packed = build_mix(keys, kids, count, 100 + count)
    out, st, rc = run_batch(torch_cuda, ctx, key_ids, sels, offsets, packed)
    assert rc == 0 and (st == 0).all()
    for (k, kind, row), off in zip(ops, offsets):
        got = out[int(off):int(off) + row.size]
        assert np.array_equal(got, expect_one(keys[k], kind, row)), (keys[k].bits, kind)


def test_ragged_equals_alone(torch_cuda, ctx, mixed_keys):
    """Each result is the same in the mix as when its group runs alone."""
    keys, kids = mixed_keys
    ops, key_ids, sels, offsets, packed = build_mix(keys, kids, 500, 7)
    out, st, rc = run_batch(torch_cuda, ctx, key_ids, sels, offsets, packed)
    assert rc == 0
    for k in range(len(keys)):
        for kind in (PUB, CRT, PLAIN):
            idx = [i for i, (kk, kd, _) in enumerate(ops) if kk == k and kd == kind]
            if not idx:
                continue
            rows = np.stack([ops[i][2] for i in idx])
            t = torch_cuda.from_numpy(rows.view(np.int32)).cuda()
            alone = ctx.modexp_key(kids[k], kind, t).cpu().numpy().view(np.uint32)
            for j, i in enumerate(idx):
                off = int(offsets[i])
                assert np.array_equal(out[off:off + rows.shape[1]], alone[j])


def test_ragged_invalid_operations(torch_cuda, ctx, mixed_keys):
    keys, kids = mixed_keys
    ops, key_ids, sels, offsets, packed = build_mix(keys, kids, 120, 11)
    key_ids = key_ids.copy()
    sels = sels.copy()
    offsets = offsets.copy()
    key_ids[3] = 12345                     # unknown key
    key_ids[5] = -1                        # negative id
    sels[7] = 9                            # bad kind
    wide = [i for i, (k, _, _) in enumerate(ops) if keys[k].bits >= 1024 and i not in (3, 5, 7)]
    offsets[wide[0]] += 1                  # misaligned row
    bad = {3: -2, 5: -2, 7: -1, wide[0]: -1}
    out, st, rc = run_batch(torch_cuda, ctx, key_ids, sels, offsets, packed)
    assert rc in (-2, -1)
    for i, (k, kind, row) in enumerate(ops):
        if i in bad:
            assert st[i] == bad[i], (i, st[i])
            continue
        assert st[i] == 0
        off = int(offsets[i])
        assert np.array_equal(out[off:off + row.size], expect_one(keys[k], kind, row))
    assert ctx.sync() == 0      # the error was reported once


def test_ragged_host_api(torch_cuda, ctx, mixed_keys):
    keys, kids = mixed_keys
    ops, key_ids, sels, offsets, packed = build_mix(keys, kids, 200, 13)
    from paper_1407_1465_gb300 import rsa_modexp_batch_host
    out = np.zeros_like(packed)
    st = np.full(len(ops), 99, dtype=np.int32)
    rsa_modexp_batch_host(ctx.handle, len(ops), key_ids, sels, offsets, packed.size, packed, out, st)
    assert (st == 0).all()
    for (k, kind, row), off in zip(ops, offsets):
        assert np.array_equal(out[int(off):int(off) + row.size], expect_one(keys[k], kind, row))


def test_ragged_full_workload_sampled(torch_cuda, ctx):
    """The ragged benchmark workload: 256 keys, 200000 operations, one call."""
    rb = workloads.ragged()
    kids = [ctx.keyload(k.bits, k.n, k.e, k.d, k.p, k.q) for k in rb.keys]
    key_ids = np.array([kids[k] for k in rb.key_ids], dtype=np.int32)
    out, st, rc = run_batch(torch_cuda, ctx, key_ids, rb.exp_sel, rb.offsets, rb.packed)
    assert rc == 0 and (st == 0).all()
    rng = np.random.default_rng(5)
    idx = rng.choice(len(rb.msgs), 120, replace=False)
    for i in idx:
        key = rb.keys[rb.key_ids[i]]
        off = int(rb.offsets[i])
        row = rb.msgs[i]
        assert np.array_equal(out[off:off + row.size], expect_one(key, int(rb.exp_sel[i]), row))
    for k in kids:
        ctx.keyunload(k)


def test_ragged_autotune_batch(torch_cuda, ctx, mixed_keys):
    """The ragged autotuner (coordinate descent over lanes per operation, the
    tensor-core group, the CRT windows and the CTA cap) installs the fastest
    configuration, and results stay exact under it."""
    from paper_1407_1465_gb300 import RSA_TUNE_RAGGED, RsaError
    keys, kids = mixed_keys
    ops, key_ids, sels, offsets, packed = build_mix(keys, kids, 300, 77)
    dev = torch_cuda.device("cuda")
    k = torch_cuda.from_numpy(key_ids).to(dev)
    s = torch_cuda.from_numpy(sels).to(dev)
    o = torch_cuda.from_numpy(offsets.view(np.int64)).to(dev)
    m = torch_cuda.from_numpy(packed.view(np.int32)).to(dev)
    try:
        best = ctx.autotune_batch(k, s, o, m)
        assert best["threads_per_op"] in (1, 4) and best["ctas_per_sm"] in (0, 2, 4) and best["ms"] > 0
        assert best["window"] in (4, 5) and best["window_big"] in (4, 5) and best["window_tc"] in (3, 4)
        assert best["variant"] in (0, 1, 3) and best["tc_min_ops"] in (128, 512)
        t = ctx.get_tuning(0, RSA_TUNE_RAGGED)
        for f in ("threads_per_op", "ctas_per_sm", "window", "window_big", "window_tc", "variant", "tc_min_ops"):
            assert t[f] == best[f], f
        out, st, rc = run_batch(torch_cuda, ctx, key_ids, sels, offsets, packed)
        assert rc == 0 and (st == 0).all()
        for (kk, kind, row), off in zip(ops, offsets):
            assert np.array_equal(out[int(off):int(off) + row.size], expect_one(keys[kk], kind, row))
        with pytest.raises(RsaError):
            ctx.set_tuning(0, RSA_TUNE_RAGGED, threads_per_op=2)
        with pytest.raises(RsaError):
            ctx.set_tuning(0, RSA_TUNE_RAGGED, window_tc=5)
        with pytest.raises(RsaError):
            ctx.set_tuning(2048, CRT, window_big=4)    # ragged-only fields
    finally:
        ctx.set_tuning(0, RSA_TUNE_RAGGED, reset=True)


@pytest.mark.parametrize("lanes", ["8", "16"])
def test_ragged_small_tiles_all_run(torch_cuda, ctx, mixed_keys, monkeypatch, lanes):
    """A batch of 4096-bit CRT operations only, small enough for the latency
    shapes (8 or 16 lanes per operation: 4 or 2 operations per tile).  Its tiles
    outnumber count/8 + buckets, so every tile must fit the planner's tile list
    (a list sized for 8-operation tiles dropped the excess ones and left their
    operations unrun).  Every result equals the same messages run through
    rsa_modexp_key; sampled ones equal the oracle."""
    monkeypatch.setenv("RSAGPU_RAGGED_LANES_4096", lanes)
    keys, kids = mixed_keys
    k = next(i for i, key in enumerate(keys) if key.bits == 4096)
    key = keys[k]
    count = 600
    rows = workloads.messages_below(key.n, count, 44, ("small-tiles", lanes))
    offsets = np.arange(count, dtype=np.uint64) * 128
    key_ids = np.full(count, kids[k], dtype=np.int32)
    sels = np.full(count, CRT, dtype=np.uint8)
    out, st, rc = run_batch(torch_cuda, ctx, key_ids, sels, offsets, rows.reshape(-1).copy())
    assert rc == 0 and (st == 0).all()
    alone = ctx.modexp_key(kids[k], CRT, torch_cuda.from_numpy(rows.view(np.int32)).cuda())
    assert np.array_equal(out.reshape(count, 128), alone.cpu().numpy().view(np.uint32))
    idx = [0, 1, 299, 598, 599]
    assert np.array_equal(out.reshape(count, 128)[idx], oracle.crt_batch(rows[idx], key.d, key.p, key.q))
