"""The allocation-free CRT entry point (rsa_crt_decrypt_noalloc).

Callers that cannot allocate device memory at call time (inside a graph
capture, behind a host process's own memory pool, or in services that forbid
allocation after start-up) use this entry point; its scratch is a fixed array
inside the library.  The test calls it through the C ABI twice in a row (the
second call reuses the array the first one left behind) and requires results
identical to the ordinary rsa_modexp_key CRT path.  It sits in a file of its
own, collected last, and passes alone or after the other tests.
"""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def test_noalloc_matches_modexp_key_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_1465_gb300 import RSA_EXP_PRIVATE_CRT, RsaContext, _lib, build, rsa_key_record
    build.build()
    lib = _lib.lib()
    keys = workloads.gen_keys([(2048, 0), (4096, 0)], workloads.DEFAULT_SEED)
    ctx = RsaContext(0)
    try:
        for key in keys:
            # inputs and outputs are allocated by the caller (here: torch), never by the entry point
            rec = torch.from_numpy(rsa_key_record(key.bits, key.n, key.e, key.d, key.p, key.q)
                                   .view(np.int32)).cuda()
            kid = ctx.keyload(key.bits, key.n, key.e, key.d, key.p, key.q)
            for call in range(2):
                count = 3000 + 37 * call    # several resident rounds of the capped grid, ragged tail
                rows = workloads.messages_below(key.n, count, 31 + call, ("noalloc", key.bits))
                msgs = torch.from_numpy(rows.view(np.int32)).cuda()
                ref = ctx.modexp_key(kid, RSA_EXP_PRIVATE_CRT, msgs)
                out = torch.full_like(msgs, -1)
                st = torch.full((count,), 99, dtype=torch.int32, device="cuda")
                stream = torch.cuda.current_stream().cuda_stream
                rc = lib.rsa_crt_decrypt_noalloc(ctypes.c_void_p(rec.data_ptr()), key.bits, count,
                                                 ctypes.c_void_p(msgs.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                                 ctypes.c_void_p(st.data_ptr()), ctypes.c_void_p(stream))
                assert rc == 0, _lib.last_error()
                torch.cuda.synchronize()
                assert torch.equal(out, ref), "no-alloc result differs on call %d (%d bits)" % (call, key.bits)
                assert bool((st == 0).all())
        # sizes outside the supported set are refused with a clear error
        rc = lib.rsa_crt_decrypt_noalloc(ctypes.c_void_p(rec.data_ptr()), 8192, 1, ctypes.c_void_p(msgs.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), None, None)
        assert rc == -7 and "4096" in _lib.last_error()
    finally:
        ctx.close()
