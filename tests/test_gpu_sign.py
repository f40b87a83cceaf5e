"""GPU: signing and verification on the exponentiation kernels (Sec. 3.2-3.3
primitives with the roles of d and e swapped), against the oracle.

Signatures must equal rep^d mod n exactly; verification must accept every
genuine signature and reject tampered signatures, wrong representatives and
out-of-range signatures, per operation.
"""
import numpy as np
import pytest

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
    c = RsaContext(0, mem_budget_bytes=4 << 30)
    yield c
    c.close()


def dev(torch, rows):
    return torch.from_numpy(np.ascontiguousarray(rows, dtype=np.uint32).view(np.int32)).cuda()


def host(t, shape):
    return t.cpu().numpy().view(np.uint32).reshape(shape)


@pytest.mark.parametrize("bits", [1024, 2048, 3072, 4096])
def test_sign_then_verify(torch_cuda, ctx, bits):
    key = workloads.gen_keys([(bits, 3)], workloads.DEFAULT_SEED)[0]
    kid = ctx.keyload(bits, key.n, key.e, key.d, key.p, key.q)
    reps = workloads.messages_below(key.n, 70, 51, ("sign", bits))
    sigs = ctx.sign(kid, dev(torch_cuda, reps))
    torch_cuda.cuda.synchronize()
    got = host(sigs, reps.shape)
    want = oracle.crt_batch(reps, key.d, key.p, key.q)
    assert np.array_equal(got, want)
    assert np.array_equal(oracle.modexp_batch(got[:8], key.e, key.n), reps[:8])
    # verification: genuine, tampered, wrong representative, out of range
    bad_sig = got.copy()
    bad_sig[1, 0] ^= 1
    bad_sig[2, key.limbs // 2] ^= 0x80000000
    bad_rep = reps.copy()
    bad_rep[3, 0] ^= 1
    bad_sig[4] = workloads.ints_to_rows([key.n + 1], key.limbs)[0]
    st = ctx.verify(kid, dev(torch_cuda, bad_sig), dev(torch_cuda, bad_rep))
    torch_cuda.cuda.synchronize()
    st = st.cpu().numpy()
    expect = np.zeros(reps.shape[0], dtype=np.int32)
    expect[[1, 2, 3]] = -8
    expect[4] = -3
    assert np.array_equal(st, expect)
    ctx.keyunload(kid)


def test_sign_without_crt_and_rejections(torch_cuda, ctx):
    from paper_1407_1465_gb300 import RsaError
    key = workloads.gen_keys([(2048, 4)], workloads.DEFAULT_SEED)[0]
    kid = ctx.keyload(2048, key.n, key.e, key.d)               # d, no p, q: plain exponent
    reps = workloads.messages_below(key.n, 33, 52, ("sign-plain",))
    bad = workloads.ints_to_rows([key.n], key.limbs)
    rows = np.concatenate([reps, bad])
    st = torch_cuda.full((rows.shape[0],), 99, dtype=torch_cuda.int32, device="cuda")
    sigs = ctx.sign(kid, dev(torch_cuda, rows), status=st)
    torch_cuda.cuda.synchronize()
    got = host(sigs, rows.shape)
    assert np.array_equal(got[:33], oracle.modexp_batch(reps, key.d, key.n))
    assert not got[33:].any()
    assert np.array_equal(st.cpu().numpy(), np.array([0] * 33 + [-3], dtype=np.int32))
    pub = ctx.keyload(2048, key.n, key.e)                      # public only: cannot sign
    with pytest.raises(RsaError) as ei:
        ctx.sign(pub, dev(torch_cuda, reps))
    assert ei.value.code == -2
    st = ctx.verify(pub, sigs[:33], dev(torch_cuda, reps))     # but verifies
    torch_cuda.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    ctx.keyunload(pub)
    ctx.keyunload(kid)


def test_toy_key_signatures(torch_cuda, ctx):
    """The paper's Fig. 2 key (n = 187, e = 7, d = 23): every representative below n."""
    t = workloads
    kid = ctx.keyload(32, 187, 7, 23, 11, 17)
    reps = np.arange(187, dtype=np.uint32).reshape(-1, 1)
    sigs = ctx.sign(kid, dev(torch_cuda, reps))
    torch_cuda.cuda.synchronize()
    got = host(sigs, reps.shape)
    assert np.array_equal(got[:, 0], np.array([oracle.modexp(int(m), 23, 187) for m in range(187)], dtype=np.uint32))
    st = ctx.verify(kid, sigs, dev(torch_cuda, reps))
    torch_cuda.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    ctx.keyunload(kid)
