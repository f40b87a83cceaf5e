"""Host-side checks of the C ABI (no GPU compute).

- the library builds, loads and exports every function include/rsa_gb300.h declares;
- the host key precomputation (rsa_key_record) matches Python integers;
- the algorithmic work model (rsa_products_per_op) matches its closed form;
- argument validation errors come back as status codes.
"""
import os
import re

import numpy as np
import pytest

import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rsa_gb300.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1407_1465_gb300 import build, _lib
    build.build()
    return _lib.lib()


def declared_functions():
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rsa_[a-z_0-9]+)\s*\(", text)))


def test_header_symbols_exported(lib):
    names = declared_functions()
    assert "rsa_modexp_batch" in names and "rsa_keyload" in names
    for name in names:
        assert hasattr(lib, name), "symbol %s declared but not exported" % name


def test_binding_covers_header():
    from paper_1407_1465_gb300 import _lib
    bound = {s[0] for s in _lib.SIGNATURES}
    for name in declared_functions():
        assert name in bound, "no ctypes signature for %s" % name


def _layout(L):
    """Word offsets of the key record (mirrors keyrec.h)."""
    H = L // 2
    off = {"n": 16, "r2n": 16 + L, "onen": 16 + 2 * L, "unitL": 16 + 3 * L, "e": 16 + 4 * L,
           "d": 16 + 5 * L + 4, "p": 16 + 6 * L + 8}
    names = ["p", "q", "r2p", "r3p", "r2q", "r3q", "onep", "oneq", "qinv", "unitH"]
    for i, nm in enumerate(names):
        off[nm] = off["p"] + i * H
    off["dp"] = off["p"] + 10 * H
    off["dq"] = off["dp"] + H + 4
    off["total"] = off["dq"] + H + 4
    return off


def _get(rec, off, n):
    return workloads.limbs_to_int(rec[off:off + n])


@pytest.mark.parametrize("bits", [1024, 2048, 3072, 4096])
def test_key_record_matches_python(lib, bits):
    from paper_1407_1465_gb300 import rsa_key_record
    key = workloads.gen_key(bits, seed=77, index=bits, mr_rounds=8)
    rec = rsa_key_record(bits, key.n, key.e, key.d, key.p, key.q)
    L, H = bits // 32, bits // 64
    lay = _layout(L)
    assert rec.size == lay["total"]
    hdr = rec[:16]
    assert hdr[0] == bits and hdr[1] == L and hdr[2] == H and hdr[3] == 3
    assert (int(hdr[4]) * key.n) % 2**32 == 2**32 - 1      # n' = -n^-1 mod 2^32
    assert (int(hdr[5]) * key.p) % 2**32 == 2**32 - 1
    assert (int(hdr[6]) * key.q) % 2**32 == 2**32 - 1
    assert hdr[7] == key.e.bit_length() and hdr[8] == key.d.bit_length()
    R, Rh = 1 << (32 * L), 1 << (32 * H)
    assert _get(rec, lay["n"], L) == key.n
    assert _get(rec, lay["r2n"], L) == R * R % key.n
    assert _get(rec, lay["onen"], L) == R % key.n
    assert _get(rec, lay["unitL"], L) == 1
    assert _get(rec, lay["e"], L + 4) == key.e
    assert _get(rec, lay["d"], L + 4) == key.d
    p, q = key.p, key.q
    assert _get(rec, lay["p"], H) == p and _get(rec, lay["q"], H) == q
    assert _get(rec, lay["r2p"], H) == Rh * Rh % p and _get(rec, lay["r3p"], H) == Rh ** 3 % p
    assert _get(rec, lay["r2q"], H) == Rh * Rh % q and _get(rec, lay["r3q"], H) == Rh ** 3 % q
    assert _get(rec, lay["onep"], H) == Rh % p and _get(rec, lay["oneq"], H) == Rh % q
    assert _get(rec, lay["qinv"], H) == pow(q, -1, p)
    assert _get(rec, lay["dp"], H + 4) == key.d % (p - 1)
    assert _get(rec, lay["dq"], H + 4) == key.d % (q - 1)


def test_key_record_toy_and_public_only(lib):
    from paper_1407_1465_gb300 import rsa_key_record
    rec = rsa_key_record(32, 17947, 131, 137, 137, 131)
    assert rec[16] == 17947 and rec[0] == 32 and rec[3] == 3
    # single-limb keys keep p, q, dp, dq, qinv in the header
    assert list(rec[9:14]) == [137, 131, 137 % 136, 137 % 130, pow(131, -1, 137)]
    key = workloads.gen_key(1024, seed=5, index=3, mr_rounds=8)
    rec = rsa_key_record(1024, key.n, key.e)
    assert rec[3] == 0  # neither d nor CRT


def test_key_record_validation(lib):
    from paper_1407_1465_gb300 import RsaError, rsa_key_record
    key = workloads.gen_key(1024, seed=5, index=4, mr_rounds=8)
    cases = [
        dict(nbits=512, n=key.p, e=key.e),                        # size
        dict(nbits=1024, n=key.n - 1, e=key.e),                   # even modulus
        dict(nbits=1024, n=key.n, e=0),                           # zero exponent
        dict(nbits=1024, n=key.n, e=key.e, d=key.d, p=key.p, q=key.q + 2),  # p*q != n
        dict(nbits=1024, n=key.n, e=key.e, d=0),                  # zero d
        dict(nbits=1024, n=key.n, e=key.e, p=key.p, q=key.q),     # p, q without d
    ]
    codes = []
    for kw in cases:
        with pytest.raises(RsaError) as ei:
            rsa_key_record(**kw)
        codes.append(ei.value.code)
    assert codes == [-7, -2, -2, -2, -2, -2]


def test_products_per_op_closed_form(lib):
    from paper_1407_1465_gb300 import RSA_EXP_PRIVATE_CRT, RSA_EXP_PRIVATE_PLAIN, RSA_EXP_PUBLIC, rsa_products_per_op

    def mm(L):
        return 2 * L * L + L
    # public e = 65537: to-Montgomery, 16 squarings, 1 multiply, from-Montgomery
    assert rsa_products_per_op(2048, RSA_EXP_PUBLIC, 65537) == 19 * mm(64)
    # CRT 2048, w = 5: per half 2 (split) + 30 (table) + 204 windows * 6; + 3 finishing + h*q
    per_half = 2 + 30 + (205 - 1) * 6
    assert rsa_products_per_op(2048, RSA_EXP_PRIVATE_CRT, window=5) == (2 * per_half + 3) * mm(32) + 32 * 32
    nwin = -(-2048 // 4)
    assert rsa_products_per_op(2048, RSA_EXP_PRIVATE_PLAIN, window=4) == (2 + 14 + (nwin - 1) * 5) * mm(64)


def test_ctx_without_gpu_reports_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1407_1465_gb300 import RsaError, rsa_ctx_create
    with pytest.raises(RsaError) as ei:
        rsa_ctx_create(0)
    assert ei.value.code in (-1, -5)


def test_tuning_dict_has_every_field():
    from paper_1407_1465_gb300 import _lib
    import inspect
    import paper_1407_1465_gb300 as pkg
    src = inspect.getsource(pkg._tuning_dict)
    for name, _ in _lib.rsa_tuning._fields_:
        assert ('"%s": t.%s' % (name, name)) in src, name
    for fn in (pkg.rsa_get_tuning, pkg.rsa_autotune, pkg.rsa_autotune_batch):
        assert "_tuning_dict(t)" in inspect.getsource(fn)


def test_null_context_is_an_argument_error(lib):
    """Every entry point that takes a context refuses a null one with
    RSA_ERR_ARG before touching a device (host-side validation)."""
    import ctypes
    u64 = ctypes.c_uint64(0)
    calls = {
        "rsa_batch_gcd": lambda: lib.rsa_batch_gcd(None, 2048, 4, None, None, None, None),
        "rsa_batch_gcd_plan": lambda: lib.rsa_batch_gcd_plan(None, 2048, 4, None, None),
        "rsa_batch_gcd_ex": lambda: lib.rsa_batch_gcd_ex(None, 2048, 4, None, None, None, 2, None),
        "rsa_batch_gcd_method": lambda: lib.rsa_batch_gcd_method(None, 2048, 4, None),
        "rsa_mr_batch": lambda: lib.rsa_mr_batch(None, 1024, 4, None, 1, None, None, None),
        "rsa_autotune_batch": lambda: lib.rsa_autotune_batch(None, 4, None, None, None, None, None, None, None),
        "rsa_modexp_batch": lambda: lib.rsa_modexp_batch(None, 4, None, None, None, None, None, None, None),
        "rsa_sign_key": lambda: lib.rsa_sign_key(None, 0, 4, None, None, None, None),
        "rsa_verify_key": lambda: lib.rsa_verify_key(None, 0, 4, None, None, None, None),
        "rsa_server_clock": lambda: lib.rsa_server_clock(None, ctypes.byref(u64)),
        "rsa_server_drain": lambda: lib.rsa_server_drain(None, 10),
        "rsa_server_stop": lambda: lib.rsa_server_stop(None),
    }
    for name, call in calls.items():
        assert call() == -1, name


def test_batch_gcd_tree_bytes_host_checks(lib):
    """rsa_batch_gcd_tree_bytes needs no device: sizes grow with the count, the
    tree's size limit (count rounded up to a power of two times the modulus
    words at most 2^26) and unsupported sizes are refused."""
    import ctypes
    b = ctypes.c_uint64(0)
    assert lib.rsa_batch_gcd_tree_bytes(2048, 1 << 17, ctypes.byref(b)) == 0
    small = b.value
    assert lib.rsa_batch_gcd_tree_bytes(2048, 1 << 20, ctypes.byref(b)) == 0
    assert b.value > 7 * small
    assert lib.rsa_batch_gcd_tree_bytes(512, 1 << 22, ctypes.byref(b)) == 0
    assert lib.rsa_batch_gcd_tree_bytes(2048, (1 << 20) + 1, ctypes.byref(b)) == -1
    assert lib.rsa_batch_gcd_tree_bytes(4096, 4, ctypes.byref(b)) == -7
    assert lib.rsa_batch_gcd_tree_bytes(2048, 4, None) == -1
