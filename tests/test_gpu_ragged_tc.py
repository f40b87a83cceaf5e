"""Ragged batches with the tensor-core groups (2048-, 3072- and 4096-bit CRT on
tcgen05 MMAs).

A CRT bucket (one key) of at least tc_min_ops operations sends all its
operations to its size's tensor-core group, in tiles of 128 (the last one
possibly partial), up to four tiles of one key per CTA at 2048 bits and two at
3072/4096 bits; smaller buckets run on the CUDA cores.  The mix here has a
2048-bit bucket of five tiles plus 37 operations (two chunks: four tiles, then
one whole and one partial), one of exactly two tiles, one below a tile, a
3072-bit bucket of two tiles plus 10, a 4096-bit bucket of three tiles plus 5
(two chunks, the second ending in a partial tile), public operations on the
same keys and 1024-bit CRT, shuffled; edge messages and out-of-range messages
sit inside tensor-core tiles.  Every result is compared with the oracle, and with the same
batch run with the group off and with a 512-operation threshold.  The bounded
MMA waits of the group report RSA_ERR_TIMEOUT when their poll budget is zero.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

PUB, CRT = 0, 1
RSA_ERR_RANGE, RSA_ERR_TIMEOUT = -3, -6
# (key index, kind, count) over the keys 2048 x 3, 1024, 3072, 4096: 5 tiles + 37, exactly 2 tiles, 100
# (below a tile); 3072: 2 tiles + 10; 4096: 3 tiles + 5
PLAN = [(0, CRT, 5 * 128 + 37), (1, CRT, 2 * 128), (2, CRT, 100), (0, PUB, 40), (1, PUB, 25), (3, CRT, 90),
        (4, CRT, 2 * 128 + 10), (5, CRT, 3 * 128 + 5), (5, PUB, 12)]


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
def mix(ctx):
    keys = workloads.gen_keys([(2048, 0), (2048, 1), (2048, 2), (1024, 0), (3072, 0), (4096, 0)],
                              workloads.DEFAULT_SEED)
    kids = [ctx.keyload(k.bits, k.n, k.e, k.d, k.p, k.q) for k in keys]
    ops = []
    for k, kind, n in PLAN:
        key = keys[k]
        rows = workloads.messages_below(key.n, n, 3, ("tc-mix", k, kind))
        if k in (0, 4, 5) and kind == CRT:
            edge = [0, 1, 2, key.n - 1, key.p, key.q, 3 * key.p, key.q * 5 % key.n]
            rows[:len(edge)] = workloads.ints_to_rows(edge, key.limbs)
            bad = [key.n, key.n + 7, (1 << key.bits) - 1]
            rows[len(edge):len(edge) + len(bad)] = workloads.ints_to_rows(bad, key.limbs)
        ops += [(k, kind, rows[i]) for i in range(n)]
    perm = np.random.default_rng(11).permutation(len(ops))
    ops = [ops[i] for i in perm]
    offsets, pos = [], 0
    for _, _, row in ops:
        offsets.append(pos)
        pos += row.size
    packed = np.zeros(pos, dtype=np.uint32)
    for (_, _, row), off in zip(ops, offsets):
        packed[off:off + row.size] = row
    key_ids = np.array([kids[k] for k, _, _ in ops], dtype=np.int32)
    sels = np.array([kind for _, kind, _ in ops], dtype=np.uint8)
    # expected values: the oracle per (key, kind) group
    want = [None] * len(ops)
    status = np.zeros(len(ops), dtype=np.int32)
    for k, key in enumerate(keys):
        for kind in (PUB, CRT):
            idx = [i for i, (kk, kd, _) in enumerate(ops) if kk == k and kd == kind]
            if not idx:
                continue
            rows = np.stack([ops[i][2] for i in idx])
            vals = [workloads.limbs_to_int(r) for r in rows]
            ok = np.array([v < key.n for v in vals])
            res = np.zeros_like(rows)
            if ok.any():
                good = rows[ok]
                res[ok] = (oracle.crt_batch(good, key.d, key.p, key.q) if kind == CRT
                           else oracle.modexp_batch(good, key.e, key.n))
            for j, i in enumerate(idx):
                want[i] = res[j]
                status[i] = 0 if ok[j] else RSA_ERR_RANGE
    return keys, ops, key_ids, sels, np.array(offsets, dtype=np.uint64), packed, want, status


def _run(torch, ctx, key_ids, sels, offsets, packed):
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


@pytest.mark.parametrize("setting", [dict(variant=3, window_tc=3), dict(variant=3, window_tc=4),
                                     dict(variant=3, tc_min_ops=512), dict(variant=1)])
def test_ragged_tensor_core_group_matches_oracle(torch_cuda, ctx, mix, setting):
    from paper_1407_1465_gb300 import RSA_TUNE_RAGGED
    keys, ops, key_ids, sels, offsets, packed, want, status = mix
    try:
        ctx.set_tuning(0, RSA_TUNE_RAGGED, threads_per_op=1, **setting)
        before = ctx.stats()["kernel_launches"]
        out, st, rc = _run(torch_cuda, ctx, key_ids, sels, offsets, packed)
        assert ctx.stats()["kernel_launches"] > before
        assert rc == 0
        assert np.array_equal(st, status)
        for i, ((k, kind, row), off) in enumerate(zip(ops, offsets)):
            assert np.array_equal(out[int(off):int(off) + row.size], want[i]), (i, keys[k].bits, kind, setting)
    finally:
        ctx.set_tuning(0, RSA_TUNE_RAGGED, reset=True)


def test_ragged_tensor_core_wait_timeout(torch_cuda, ctx, mix, monkeypatch):
    """A zero poll budget makes every MMA wait of the group give up: its
    operations report RSA_ERR_TIMEOUT with zeroed rows, rsa_sync reports it,
    the other operations are unaffected and the context keeps working."""
    from paper_1407_1465_gb300 import RSA_TUNE_RAGGED
    keys, ops, key_ids, sels, offsets, packed, want, status = mix
    try:
        ctx.set_tuning(0, RSA_TUNE_RAGGED, threads_per_op=1, variant=3)
        monkeypatch.setenv("RSAGPU_TC_WAIT_POLLS", "0")
        out, st, rc = _run(torch_cuda, ctx, key_ids, sels, offsets, packed)
        monkeypatch.delenv("RSAGPU_TC_WAIT_POLLS")
        assert rc == RSA_ERR_TIMEOUT
        timed = st == RSA_ERR_TIMEOUT
        # every operation of the CRT buckets of at least 128 at 2048/3072/4096 bits ran on the tensor cores
        on_tc = sum(n for k, kind, n in PLAN if kind == CRT and keys[k].bits >= 2048 and n >= 128)
        assert on_tc == (5 * 128 + 37) + 2 * 128 + (2 * 128 + 10) + (3 * 128 + 5)
        assert timed.sum() == on_tc
        for i, ((k, kind, row), off) in enumerate(zip(ops, offsets)):
            got = out[int(off):int(off) + row.size]
            if timed[i]:
                assert not got.any()
            else:
                assert st[i] == status[i] and np.array_equal(got, want[i])
        out, st, rc = _run(torch_cuda, ctx, key_ids, sels, offsets, packed)
        assert rc == 0 and np.array_equal(st, status)
    finally:
        ctx.set_tuning(0, RSA_TUNE_RAGGED, reset=True)
