"""The request loop (rsa_server_*): staggered arrivals of mixed requests.

Requests over several keys, sizes and exponent kinds arrive spread over time;
the loop batches whatever has arrived while earlier batches are still on the
GPU.  Every request's result must equal the oracle's and the result of the
same messages run alone through rsa_modexp_key; a request larger than the
memory budget allows is refused at submit.
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


def test_serving_mixed_arrivals(torch_cuda):
    from paper_1407_1465_gb300 import (RsaContext, RsaError, build, rsa_server_drain, rsa_server_get_stats,
                                       rsa_server_poll, rsa_server_start, rsa_server_stop, rsa_server_submit)
    build.build()
    keys = workloads.gen_keys([(1024, 0), (2048, 0), (3072, 0), (4096, 0)], workloads.DEFAULT_SEED)
    ctx = RsaContext(0, mem_budget_bytes=8 << 30)
    try:
        kids = [ctx.keyload(k.bits, k.n, k.e, k.d, k.p, k.q) for k in keys]
        rsa_server_start(ctx.handle, max_inflight_batches=3, batch_window_us=300, mem_budget_bytes=64 << 20)
        st = workloads.Stream(workloads.stream_key(3, "serve"))
        reqs = []
        for r in range(90):
            k = st.below(len(keys))
            kinds = [PUB, CRT] + ([PLAIN] if keys[k].bits <= 2048 else [])
            kind = kinds[st.below(len(kinds))]
            count = 1 + st.below(64)
            msgs = workloads.messages_below(keys[k].n, count, 3, ("serve", r))
            out = np.zeros_like(msgs)
            status = np.full(count, 99, dtype=np.int32)
            arrive = 1_000_000 + r * 400_000          # one request every 0.4 ms, starting at 1 ms
            t = rsa_server_submit(ctx.handle, kids[k], kind, msgs, out, status, arrive_ns=arrive)
            reqs.append((t, k, kind, msgs, out, status))
        rsa_server_drain(ctx.handle, timeout_ms=120000)
        stats = rsa_server_get_stats(ctx.handle)
        assert stats["completed"] == len(reqs) and stats["batches"] >= 2
        assert stats["p99_us"] >= stats["p50_us"] > 0
        for t, k, kind, msgs, out, status in reqs:
            assert rsa_server_poll(ctx.handle, t) == 1
            assert (status == 0).all()
            key = keys[k]
            if kind == PUB:
                want = oracle.modexp_batch(msgs, key.e, key.n)
            elif kind == CRT:
                want = oracle.crt_batch(msgs, key.d, key.p, key.q)
            else:
                want = oracle.modexp_batch(msgs, key.d, key.n)
            assert np.array_equal(out, want)
            alone = ctx.modexp_key(kids[k], kind, torch_cuda.from_numpy(msgs.view(np.int32)).cuda())
            assert np.array_equal(alone.cpu().numpy().view(np.uint32), out)
        # a request bigger than one batch's share of the budget is refused
        big = workloads.messages_below(keys[3].n, 60000, 4, "big")
        with pytest.raises(RsaError) as ei:
            rsa_server_submit(ctx.handle, kids[3], CRT, big, np.zeros_like(big))
        assert ei.value.code == -4
        rsa_server_stop(ctx.handle)
    finally:
        ctx.close()
