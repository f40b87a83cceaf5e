"""The allocation-free CRT entry point (rsa_crt_decrypt_noalloc).

Callers that cannot allocate device memory at call time (inside a graph
capture, behind a host process's own memory pool, or in services that forbid
allocation after start-up) use this entry point; its scratch is a fixed array
inside the library.  The test calls it through the C ABI twice in a row per key
size (the second call reuses the array the first one left behind) and requires
results identical to the ordinary rsa_modexp_key CRT path, with sampled rows
also checked against the oracle.  It sits in a file of its own, collected last,
and passes alone or after the other tests.

The counts are chosen above what one round of the scratch-capped grid holds:
the array keeps 2 * 16 * H * 128 bytes of window tables per warp pair (H limbs
per prime, window 4), so 32 MiB caps the grid at 512 / 256 / 170 / 128 warp
pairs for 1024 / 2048 / 3072 / 4096-bit keys, i.e. 16384 / 8192 / 5440 / 4096
operations per round.  Counts past those make every warp pair take a second
tile and reuse its table slot.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 32 << 20
WINDOW = 4
# operations per key size: past one round of the capped grid, with a ragged tail
COUNTS = {1024: 16384 + 901, 2048: 8192 + 411, 3072: 5440 + 167, 4096: 4096 + 403}


def _ops_per_round(bits):
    H = bits // 64
    return SCRATCH_BYTES // (2 * (1 << WINDOW) * H * 128) * 32


def test_counts_exceed_one_round_of_the_capped_grid():
    for bits, count in COUNTS.items():
        assert count > _ops_per_round(bits), bits


def test_noalloc_matches_modexp_key_and_oracle_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_1465_gb300 import RSA_EXP_PRIVATE_CRT, RsaContext, _lib, build, rsa_key_record
    build.build()
    lib = _lib.lib()
    keys = workloads.gen_keys([(1024, 0), (2048, 0), (3072, 0), (4096, 0)], workloads.DEFAULT_SEED)
    ctx = RsaContext(0)
    try:
        for key in keys:
            # inputs and outputs are allocated by the caller (here: torch), never by the entry point
            rec = torch.from_numpy(rsa_key_record(key.bits, key.n, key.e, key.d, key.p, key.q)
                                   .view(np.int32)).cuda()
            kid = ctx.keyload(key.bits, key.n, key.e, key.d, key.p, key.q)
            for call in range(2):
                count = COUNTS[key.bits] - 29 * call
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
                # rows of the first tile, of the second round of the capped grid and of the tail
                r1 = _ops_per_round(key.bits)
                idx = sorted({0, 31, r1 - 1, r1, r1 + 33, count - 1})
                got = out.cpu().numpy().view(np.uint32)[idx]
                want = oracle.crt_batch(rows[idx], key.d, key.p, key.q)
                assert np.array_equal(got, want), "no-alloc rows differ from the oracle (%d bits)" % key.bits
        # sizes outside the supported set are refused with a clear error
        rc = lib.rsa_crt_decrypt_noalloc(ctypes.c_void_p(rec.data_ptr()), 8192, 1, ctypes.c_void_p(msgs.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), None, None)
        assert rc == -7 and "4096" in _lib.last_error()
    finally:
        ctx.close()
