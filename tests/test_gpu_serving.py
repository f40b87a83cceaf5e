"""The request loop (rsa_server_*): staggered arrivals of mixed requests.

Requests over several keys, sizes and exponent kinds arrive spread over time;
the loop batches whatever has arrived while earlier batches are still on the
GPU.  Every request's result must equal the oracle's and the result of the
same messages run alone through rsa_modexp_key.  Admission is by bytes in
flight: requests larger than a slot's share of the budget are served (waiting
for room when the batches in flight hold it), and only a request larger than
the whole budget is refused at submit.
"""
import threading
import time

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


@pytest.mark.parametrize("mix_sizes", [False, True])
def test_serving_mixed_arrivals(torch_cuda, mix_sizes):
    """One modulus size per batch (the default) and batches that take every size
    (RSA_SERVER_MIX_SIZES) give the same, exact results."""
    from paper_1407_1465_gb300 import (RsaContext, RsaError, build, rsa_server_drain, rsa_server_get_stats,
                                       rsa_server_poll, rsa_server_start, rsa_server_stop, rsa_server_submit)
    build.build()
    keys = workloads.gen_keys([(1024, 0), (2048, 0), (3072, 0), (4096, 0)], workloads.DEFAULT_SEED)
    ctx = RsaContext(0, mem_budget_bytes=8 << 30)
    try:
        kids = [ctx.keyload(k.bits, k.n, k.e, k.d, k.p, k.q) for k in keys]
        rsa_server_start(ctx.handle, max_inflight_batches=3, batch_window_us=300, mem_budget_bytes=64 << 20,
                         mix_sizes=mix_sizes)
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
        # a request bigger than the whole budget (65000 x 4096-bit rows: ~68 MB
        # of rows, results and metadata against 64 MiB) is refused
        big = np.zeros((65000, 128), dtype=np.uint32)
        with pytest.raises(RsaError) as ei:
            rsa_server_submit(ctx.handle, kids[3], CRT, big, np.zeros_like(big))
        assert ei.value.code == -4
        rsa_server_stop(ctx.handle)
    finally:
        ctx.close()



def test_serving_admission_by_bytes_in_flight(torch_cuda):
    """Two requests that each take more than half of the budget (and far more
    than a slot's share) are both served: the second waits until the first's
    batch gives its bytes back; the arena never holds more than the budget."""
    from paper_1407_1465_gb300 import (RsaContext, build, rsa_server_drain, rsa_server_get_stats, rsa_server_poll,
                                       rsa_server_start, rsa_server_stop, rsa_server_submit)
    build.build()
    key = workloads.gen_keys([(2048, 0)], workloads.DEFAULT_SEED)[0]
    budget = 40 << 20
    ctx = RsaContext(0, mem_budget_bytes=6 << 30)
    try:
        kid = ctx.keyload(key.bits, key.n, key.e, key.d, key.p, key.q)
        rsa_server_start(ctx.handle, max_inflight_batches=4, batch_window_us=100, mem_budget_bytes=budget)
        reqs = []
        # 40000 rows: 40000 x (8 x 64 + 17) bytes and alignment, 21 160 192 bytes of the arena
        for r, count in enumerate([40000, 40000, 5, 17]):
            msgs = workloads.messages_below(key.n, count, 8, ("admit", r))
            out = np.zeros_like(msgs)
            status = np.full(count, 99, dtype=np.int32)
            reqs.append((rsa_server_submit(ctx.handle, kid, PUB, msgs, out, status), msgs, out, status))
        rsa_server_drain(ctx.handle, timeout_ms=120000)
        st = rsa_server_get_stats(ctx.handle)
        assert st["completed"] == 4 and st["rejected"] == 0
        assert 21_160_192 <= st["peak_bytes"] <= budget
        for t, msgs, out, status in reqs:
            assert rsa_server_poll(ctx.handle, t) == 1 and (status == 0).all()
            alone = ctx.modexp_key(kid, PUB, torch_cuda.from_numpy(msgs.view(np.int32)).cuda())
            assert np.array_equal(alone.cpu().numpy().view(np.uint32), out)
            idx = np.arange(0, len(msgs), max(1, len(msgs) // 64))
            assert np.array_equal(out[idx], oracle.modexp_batch(msgs[idx], key.e, key.n))
        rsa_server_stop(ctx.handle)
    finally:
        ctx.close()


def test_serving_failure_paths(torch_cuda):
    """A request whose arrival time never comes (a dropped doorbell) keeps the
    drain from finishing: rsa_server_drain returns RSA_ERR_TIMEOUT, and
    rsa_server_stop cancels it promptly with RSA_ERR_TIMEOUT in its status.
    A submitting thread that dies half way leaves what it queued to be served
    correctly; a request under an unknown key is refused at submit."""
    from paper_1407_1465_gb300 import (RsaContext, RsaError, build, rsa_server_clock, rsa_server_drain,
                                       rsa_server_poll, rsa_server_start, rsa_server_stop, rsa_server_submit)
    build.build()
    key = workloads.gen_keys([(2048, 0)], workloads.DEFAULT_SEED)[0]
    ctx = RsaContext(0, mem_budget_bytes=4 << 30)
    try:
        kid = ctx.keyload(key.bits, key.n, key.e, key.d, key.p, key.q)
        rsa_server_start(ctx.handle, max_inflight_batches=4, batch_window_us=100, mem_budget_bytes=64 << 20)
        done = []
        died = []

        def producer():
            try:
                for r in range(10):
                    if r == 5:
                        raise RuntimeError("producer died")
                    msgs = workloads.messages_below(key.n, 7 + r, 5, ("fail", r))
                    out = np.zeros_like(msgs)
                    t = rsa_server_submit(ctx.handle, kid, CRT, msgs, out)
                    done.append((t, msgs, out))
            except RuntimeError as exc:
                died.append(exc)

        th = threading.Thread(target=producer)
        th.start()
        th.join()
        assert died and len(done) == 5
        far_msgs = workloads.messages_below(key.n, 3, 6, "far")
        far_out = np.zeros_like(far_msgs)
        far_status = np.full(3, 99, dtype=np.int32)
        rsa_server_submit(ctx.handle, kid, CRT, far_msgs, far_out, far_status,
                          arrive_ns=rsa_server_clock(ctx.handle) + 3600 * 10**9)
        with pytest.raises(RsaError) as ei:
            rsa_server_drain(ctx.handle, timeout_ms=2000)
        assert ei.value.code == -6
        for t, msgs, out in done:
            assert rsa_server_poll(ctx.handle, t) == 1
            assert np.array_equal(out, oracle.crt_batch(msgs, key.d, key.p, key.q))
        with pytest.raises(RsaError) as ei:
            rsa_server_submit(ctx.handle, 999, CRT, far_msgs, np.zeros_like(far_msgs))
        assert ei.value.code == -2
        t0 = time.monotonic()
        rsa_server_stop(ctx.handle)
        assert time.monotonic() - t0 < 5.0
        assert (far_status == -6).all() and not far_out.any()
    finally:
        ctx.close()


def test_serving_restart_returns_memory(torch_cuda):
    """Stopping the loop gives its slots' buffers back to the context's budget,
    so the loop can be started again in the same context."""
    from paper_1407_1465_gb300 import RsaContext, build, rsa_server_start, rsa_server_stop
    build.build()
    ctx = RsaContext(0, mem_budget_bytes=5 << 30)
    try:
        base = ctx.stats()["bytes_resident"]
        for _ in range(3):
            rsa_server_start(ctx.handle, max_inflight_batches=4, batch_window_us=100, mem_budget_bytes=64 << 20)
            assert ctx.stats()["bytes_resident"] > base
            rsa_server_stop(ctx.handle)
            assert ctx.stats()["bytes_resident"] == base
    finally:
        ctx.close()


def test_serving_concurrent_submitters(torch_cuda):
    """Four host threads submit at once (the binding releases the GIL, so the
    submits overlap); every request completes with the oracle's result."""
    from paper_1407_1465_gb300 import (RsaContext, build, rsa_server_drain, rsa_server_poll, rsa_server_start,
                                       rsa_server_stop, rsa_server_submit)
    build.build()
    keys = workloads.gen_keys([(1024, 0), (2048, 0)], workloads.DEFAULT_SEED)
    ctx = RsaContext(0, mem_budget_bytes=4 << 30)
    try:
        kids = [ctx.keyload(k.bits, k.n, k.e, k.d, k.p, k.q) for k in keys]
        rsa_server_start(ctx.handle, max_inflight_batches=4, batch_window_us=100, mem_budget_bytes=64 << 20)
        done = [[] for _ in range(4)]
        errors = []

        def submitter(tid):
            try:
                for r in range(25):
                    k = (tid + r) % 2
                    kind = CRT if r % 3 else PUB
                    msgs = workloads.messages_below(keys[k].n, 1 + (r * 7 + tid) % 20, tid, ("conc", r))
                    out = np.zeros_like(msgs)
                    t = rsa_server_submit(ctx.handle, kids[k], kind, msgs, out)
                    done[tid].append((t, k, kind, msgs, out))
            except Exception as exc:   # reported below, not swallowed
                errors.append(exc)

        threads = [threading.Thread(target=submitter, args=(i,)) for i in range(4)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        assert not errors
        rsa_server_drain(ctx.handle, timeout_ms=120000)
        tickets = set()
        for lst in done:
            for t, k, kind, msgs, out in lst:
                assert t not in tickets
                tickets.add(t)
                assert rsa_server_poll(ctx.handle, t) == 1
                key = keys[k]
                want = (oracle.crt_batch(msgs, key.d, key.p, key.q) if kind == CRT
                        else oracle.modexp_batch(msgs, key.e, key.n))
                assert np.array_equal(out, want)
        assert len(tickets) == 100
        rsa_server_stop(ctx.handle)
    finally:
        ctx.close()
