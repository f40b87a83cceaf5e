"""CPU reference ("oracle") for batched RSA modular exponentiation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (``paper_1407_1465_gb300``) never imports it and shares no code
with it.

The arithmetic lives in ``rsa_oracle.c`` (plain C: schoolbook multiply, Knuth
Algorithm D, the paper's Fig. 4-7 exponentiation methods and a CRT reference).
This module compiles it with gcc and binds it with ctypes.  Python integers are
converted to little-endian 32-bit limb arrays at the boundary; no arithmetic of
the method happens in Python.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rsa_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "librsa_oracle.so")
_lock = threading.Lock()
_lib = None

KIND_PLAIN = 0
KIND_CRT = 1

_u32p = ctypes.POINTER(ctypes.c_uint32)


class _BatchArgs(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("msgs", _u32p),
        ("msg_stride", ctypes.c_size_t),
        ("out", _u32p),
        ("out_stride", ctypes.c_size_t),
        ("n", _u32p),
        ("n_limbs", ctypes.c_size_t),
        ("exp", _u32p),
        ("exp_limbs", ctypes.c_size_t),
        ("p", _u32p),
        ("q", _u32p),
        ("nh", ctypes.c_size_t),
    ]


def build(src: str = _SRC, out: str = _LIB_PATH, extra_flags: tuple = ()) -> str:
    """Compile the oracle into a shared library (plain gcc, -O2, pthreads)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
           "-I", _HERE, *extra_flags, src, "-o", out]
    subprocess.run(cmd, check=True)
    return out


def _bind(lib):
    sz = ctypes.c_size_t
    lib.oracle_modexp_l2r.argtypes = [_u32p, sz, _u32p, sz, _u32p, sz, _u32p]
    lib.oracle_modexp_r2l.argtypes = [_u32p, sz, _u32p, sz, _u32p, sz, _u32p]
    lib.oracle_modexp_naive.argtypes = [_u32p, sz, ctypes.c_uint64, _u32p, sz, _u32p, _u32p]
    lib.oracle_modexp_kary.argtypes = [_u32p, sz, _u32p, sz, ctypes.c_uint, _u32p, sz, _u32p]
    lib.oracle_modexp_sliding.argtypes = [_u32p, sz, _u32p, sz, ctypes.c_uint, _u32p, sz, _u32p]
    lib.oracle_crt_decrypt.argtypes = [_u32p, _u32p, _u32p, _u32p, sz, _u32p]
    lib.oracle_mul.argtypes = [_u32p, sz, _u32p, sz, _u32p]
    lib.oracle_divmod.argtypes = [_u32p, sz, _u32p, sz, _u32p, _u32p]
    lib.oracle_default_threads.restype = ctypes.c_int
    lib.oracle_modexp_batch.argtypes = [ctypes.POINTER(_BatchArgs), sz, ctypes.c_int]
    lib.oracle_modexp_batch.restype = ctypes.c_int
    lib.oracle_miller_rabin.argtypes = [_u32p, sz, _u32p, sz]
    lib.oracle_miller_rabin.restype = ctypes.c_int
    lib.oracle_batch_gcd_row.argtypes = [_u32p, sz, sz, sz, _u32p]
    lib.oracle_batch_gcd_row.restype = ctypes.c_int
    return lib


def load(path: str | None = None):
    """Load (building on first use) the oracle library; ``path`` selects another build."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
                build()
            _lib = _bind(ctypes.CDLL(_LIB_PATH))
    return _lib


# ---------------------------------------------------------------- conversions

def to_limbs(x: int, n: int) -> np.ndarray:
    """Little-endian 32-bit limbs of a non-negative int, padded to n limbs."""
    if x < 0 or x.bit_length() > 32 * n:
        raise ValueError("value does not fit in %d limbs" % n)
    return np.frombuffer(x.to_bytes(4 * n, "little"), dtype="<u4").astype(np.uint32).copy()


def from_limbs(a) -> int:
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return int.from_bytes(a.astype("<u4").tobytes(), "little")


def limbs_for(x: int) -> int:
    return max(1, (x.bit_length() + 31) // 32)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_u32p)


# ---------------------------------------------------------------- scalar API

def modexp(g: int, e: int, m: int, method: str = "l2r", k: int = 4, lib=None) -> int:
    """g^e mod m with one of the paper's methods: l2r, r2l, naive, kary, sliding."""
    lib = lib or load()
    nm = limbs_for(m)
    ng = max(limbs_for(g), 1)
    ne = limbs_for(e)
    ga, ea, ma = to_limbs(g, ng), to_limbs(e, ne), to_limbs(m, nm)
    out = np.zeros(nm, dtype=np.uint32)
    if method == "l2r":
        lib.oracle_modexp_l2r(_ptr(ga), ng, _ptr(ea), ne, _ptr(ma), nm, _ptr(out))
    elif method == "r2l":
        lib.oracle_modexp_r2l(_ptr(ga), ng, _ptr(ea), ne, _ptr(ma), nm, _ptr(out))
    elif method == "naive":
        lib.oracle_modexp_naive(_ptr(ga), ng, e, _ptr(ma), nm, _ptr(out), None)
    elif method == "kary":
        lib.oracle_modexp_kary(_ptr(ga), ng, _ptr(ea), ne, k, _ptr(ma), nm, _ptr(out))
    elif method == "sliding":
        lib.oracle_modexp_sliding(_ptr(ga), ng, _ptr(ea), ne, k, _ptr(ma), nm, _ptr(out))
    else:
        raise ValueError(method)
    return from_limbs(out)


def naive_trace(g: int, e: int, m: int, lib=None) -> list[int]:
    """[g^1 mod m, ..., g^e mod m] from the Fig. 4 repeated-multiplication loop."""
    lib = lib or load()
    nm = limbs_for(m)
    ng = limbs_for(g)
    ga, ma = to_limbs(g, ng), to_limbs(m, nm)
    out = np.zeros(nm, dtype=np.uint32)
    trace = np.zeros(max(e, 1) * nm, dtype=np.uint32)
    lib.oracle_modexp_naive(_ptr(ga), ng, e, _ptr(ma), nm, _ptr(out), _ptr(trace))
    return [from_limbs(trace[i * nm:(i + 1) * nm]) for i in range(e)]


def crt_decrypt(c: int, d: int, p: int, q: int, lib=None) -> int:
    """c^d mod pq through the CRT reference (p, q odd primes of nh limbs each)."""
    lib = lib or load()
    nh = max(limbs_for(p), limbs_for(q))
    ca, da = to_limbs(c, 2 * nh), to_limbs(d, 2 * nh)
    pa, qa = to_limbs(p, nh), to_limbs(q, nh)
    out = np.zeros(2 * nh, dtype=np.uint32)
    lib.oracle_crt_decrypt(_ptr(ca), _ptr(da), _ptr(pa), _ptr(qa), nh, _ptr(out))
    return from_limbs(out)


def mul(a: int, b: int, lib=None) -> int:
    lib = lib or load()
    na, nb = limbs_for(a), limbs_for(b)
    aa, ba = to_limbs(a, na), to_limbs(b, nb)
    out = np.zeros(na + nb, dtype=np.uint32)
    lib.oracle_mul(_ptr(aa), na, _ptr(ba), nb, _ptr(out))
    return from_limbs(out)


def divmod_(u: int, v: int, lib=None) -> tuple[int, int]:
    lib = lib or load()
    nu, nv = limbs_for(u), limbs_for(v)
    nu = max(nu, nv)
    ua, va = to_limbs(u, nu), to_limbs(v, nv)
    q = np.zeros(nu - nv + 1, dtype=np.uint32)
    r = np.zeros(nv, dtype=np.uint32)
    lib.oracle_divmod(_ptr(ua), nu, _ptr(va), nv, _ptr(q), _ptr(r))
    return from_limbs(q), from_limbs(r)


# ---------------------------------------------------------------- batch API

def modexp_batch(msgs: np.ndarray, exp: int, n: int, threads: int = 0, lib=None) -> np.ndarray:
    """Plain definition for one key: out[i] = msgs[i]^exp mod n (rows of limbs)."""
    lib = lib or load()
    msgs = np.ascontiguousarray(msgs, dtype=np.uint32)
    count, nl = msgs.shape
    ne = limbs_for(exp)
    na, ea = to_limbs(n, nl), to_limbs(exp, ne)
    out = np.zeros((count, nl), dtype=np.uint32)
    args = _BatchArgs(KIND_PLAIN, _ptr(msgs), nl, _ptr(out), nl, _ptr(na), nl, _ptr(ea), ne,
                      None, None, 0)
    lib.oracle_modexp_batch(ctypes.byref(args), count, threads)
    return out


def crt_batch(msgs: np.ndarray, d: int, p: int, q: int, threads: int = 0, lib=None) -> np.ndarray:
    """CRT reference for one key: out[i] = msgs[i]^d mod pq (rows of 2*nh limbs)."""
    lib = lib or load()
    msgs = np.ascontiguousarray(msgs, dtype=np.uint32)
    count, nl = msgs.shape
    nh = nl // 2
    da, pa, qa = to_limbs(d, nl), to_limbs(p, nh), to_limbs(q, nh)
    out = np.zeros((count, nl), dtype=np.uint32)
    args = _BatchArgs(KIND_CRT, _ptr(msgs), nl, _ptr(out), nl, None, 0, _ptr(da), nl,
                      _ptr(pa), _ptr(qa), nh)
    lib.oracle_modexp_batch(ctypes.byref(args), count, threads)
    return out


def default_threads(lib=None) -> int:
    return (lib or load()).oracle_default_threads()


# ---------------------------------------------------------------- primality (key generation)

def miller_rabin(n: int, bases, lib=None) -> int:
    """Miller-Rabin with the given bases: 1 probable prime, 0 composite, -1 invalid n."""
    lib = lib or load()
    nm = limbs_for(n)
    na = to_limbs(n, nm)
    ba = np.concatenate([to_limbs(b, nm) for b in bases]) if len(bases) else np.zeros(nm, dtype=np.uint32)
    return int(lib.oracle_miller_rabin(_ptr(na), nm, _ptr(np.ascontiguousarray(ba)), len(bases)))


def miller_rabin_batch(cands: np.ndarray, bases: np.ndarray, threads: int = 0, lib=None) -> np.ndarray:
    """cands: (count, L) uint32 rows; bases: (count, rounds, L).  Verdicts as int32."""
    from concurrent.futures import ThreadPoolExecutor
    lib = lib or load()
    cands = np.ascontiguousarray(cands, dtype=np.uint32)
    bases = np.ascontiguousarray(bases, dtype=np.uint32)
    count, L = cands.shape
    rounds = bases.shape[1]
    out = np.zeros(count, dtype=np.int32)

    def one(i):
        out[i] = lib.oracle_miller_rabin(_ptr(cands[i]), L, _ptr(bases[i]), rounds)

    with ThreadPoolExecutor(max_workers=threads or default_threads(lib)) as ex:
        list(ex.map(one, range(count)))
    return out


# ---------------------------------------------------------------- batch GCD (weak-key detection)

def batch_gcd(moduli: np.ndarray, rows=None, threads: int = 0, lib=None) -> tuple[np.ndarray, np.ndarray]:
    """moduli: (count, L) uint32 rows.  For each selected row i (all by default)
    g_i = gcd(n_i, product of the other valid moduli) and its flag (-1 invalid
    n_i, 0 g = 1, 1 proper factor, 2 g = n_i).  Returns (gcds, flags) in the
    order of ``rows``."""
    from concurrent.futures import ThreadPoolExecutor
    lib = lib or load()
    mods = np.ascontiguousarray(moduli, dtype=np.uint32)
    count, L = mods.shape
    rows = list(range(count)) if rows is None else [int(r) for r in rows]
    gcds = np.zeros((len(rows), L), dtype=np.uint32)
    flags = np.zeros(len(rows), dtype=np.int32)

    def one(k):
        flags[k] = lib.oracle_batch_gcd_row(_ptr(mods), count, L, rows[k], _ptr(gcds[k]))

    with ThreadPoolExecutor(max_workers=threads or default_threads(lib)) as ex:
        list(ex.map(one, range(len(rows))))
    return gcds, flags
