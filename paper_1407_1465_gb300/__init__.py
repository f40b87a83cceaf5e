"""Batched RSA modular exponentiation on GB300 (sm_103a).

Python binding of the C ABI in include/rsa_gb300.h.  The functions below carry
the C names and only marshal arguments (Python ints -> limb arrays, tensors ->
device pointers, streams -> cudaStream_t); every step of the computation runs
in the library's CUDA kernels.  PyTorch is used for device memory and streams.

    ctx = RsaContext()
    kid = ctx.keyload(2048, n, e, d, p, q)          # Python ints
    out = ctx.modexp_key(kid, RSA_EXP_PRIVATE_CRT, msgs)  # msgs: CUDA uint32/int32 [count, L]
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (RSA_ERR_ARG, RSA_ERR_CUDA, RSA_ERR_KEY, RSA_ERR_NOMEM, RSA_ERR_RANGE,  # noqa: F401
                   RSA_ERR_TIMEOUT, RSA_ERR_UNSUPPORTED, RSA_ERR_VERIFY, RSA_EXP_PRIVATE_CRT, RSA_EXP_PRIVATE_PLAIN,
                   RSA_EXP_PUBLIC, RSA_GCD_AUTO, RSA_GCD_SCAN, RSA_GCD_TREE, RSA_OK, RSA_TUNE_RAGGED, RsaError, check, last_error, rsa_stats, rsa_tuning)

__all__ = [
    "RsaContext", "RsaError", "int_to_limbs", "limbs_to_int",
    "rsa_ctx_create", "rsa_ctx_destroy", "rsa_keyload", "rsa_key_record", "rsa_tc_operand_image",
    "rsa_tc_round_operand_image",
    "rsa_keyunload", "rsa_key_info",
    "rsa_modexp_key", "rsa_modexp_batch", "rsa_modexp_key_host", "rsa_modexp_batch_host",
    "rsa_sign_key", "rsa_verify_key", "rsa_mr_batch", "rsa_batch_gcd", "rsa_batch_gcd_host", "rsa_batch_gcd_plan",
    "rsa_batch_gcd_ex", "rsa_batch_gcd_method", "rsa_batch_gcd_tree_bytes",
    "rsa_sync", "rsa_last_error", "rsa_set_tuning", "rsa_get_tuning", "rsa_get_stats",
    "rsa_products_per_op", "rsa_imad_probe", "rsa_crt_decrypt_noalloc", "rsa_autotune", "rsa_autotune_batch",
    "rsa_server_start", "rsa_server_submit", "rsa_server_submit_many", "rsa_server_clock", "rsa_server_poll", "rsa_server_drain", "rsa_server_get_stats",
    "rsa_server_stop",
]


def int_to_limbs(x: int, nlimbs: int) -> np.ndarray:
    if x < 0 or x.bit_length() > 32 * nlimbs:
        raise ValueError("value does not fit in %d limbs" % nlimbs)
    return np.frombuffer(x.to_bytes(4 * nlimbs, "little"), dtype="<u4").astype(np.uint32)


def limbs_to_int(a) -> int:
    return int.from_bytes(np.ascontiguousarray(a, dtype=np.uint32).astype("<u4").tobytes(), "little")


def _ptr(x):
    """Device or host address of a tensor / ndarray / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError("cannot take the address of %r" % type(x))


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


# ------------------------------------------------------------------ C-named functions

def rsa_ctx_create(device: int = 0, mem_budget_bytes: int = 0) -> int:
    h = ctypes.c_void_p()
    check(_lib.lib().rsa_ctx_create(ctypes.byref(h), device, mem_budget_bytes))
    return h.value


def rsa_ctx_destroy(ctx: int) -> None:
    check(_lib.lib().rsa_ctx_destroy(ctx))


def rsa_keyload(ctx: int, nbits: int, n: int, e: int, d: int | None = None,
                p: int | None = None, q: int | None = None) -> int:
    L = max(1, nbits // 32)
    hl = 1 if L == 1 else L // 2
    na = int_to_limbs(n, L)
    el = max(1, (e.bit_length() + 31) // 32)
    ea = int_to_limbs(e, el)
    da = int_to_limbs(d, L) if d is not None else None
    pa = int_to_limbs(p, hl) if p is not None else None
    qa = int_to_limbs(q, hl) if q is not None else None
    kid = ctypes.c_int32(-1)
    check(_lib.lib().rsa_keyload(ctx, nbits, _ptr(na), _ptr(ea), el, _ptr(da), _ptr(pa), _ptr(qa),
                                 ctypes.byref(kid)))
    return kid.value


def rsa_key_record(nbits: int, n: int, e: int, d: int | None = None, p: int | None = None,
                   q: int | None = None) -> np.ndarray:
    """Host-only: the device key record rsa_keyload would upload (uint32 words)."""
    L = max(1, nbits // 32)
    hl = 1 if L == 1 else L // 2
    na = int_to_limbs(n, L)
    el = max(1, (e.bit_length() + 31) // 32)
    ea = int_to_limbs(e, el)
    da = int_to_limbs(d, L) if d is not None else None
    pa = int_to_limbs(p, hl) if p is not None else None
    qa = int_to_limbs(q, hl) if q is not None else None
    words = ctypes.c_size_t(0)
    check(_lib.lib().rsa_key_record(nbits, _ptr(na), _ptr(ea), el, _ptr(da), _ptr(pa), _ptr(qa), None, 0,
                                    ctypes.byref(words)))
    rec = np.zeros(words.value, dtype=np.uint32)
    check(_lib.lib().rsa_key_record(nbits, _ptr(na), _ptr(ea), el, _ptr(da), _ptr(pa), _ptr(qa), _ptr(rec),
                                    rec.size, ctypes.byref(words)))
    return rec


RSA_TC_IMAGE_BYTES = 73728


def rsa_tc_operand_image(m: int) -> np.ndarray:
    """Host-only: the tensor-core operand images (uint8, RSA_TC_IMAGE_BYTES) of a
    1024-bit odd prime m, as built at key load for the variant-3 CRT path."""
    ma = int_to_limbs(m, 32)
    out = np.zeros(RSA_TC_IMAGE_BYTES, dtype=np.uint8)
    check(_lib.lib().rsa_tc_operand_image(_ptr(ma), _ptr(out), out.size))
    return out


def rsa_tc_round_image_bytes(prime_bits: int) -> int:
    d = prime_bits // 16
    return 6 * d * (d + 16)


def rsa_tc_round_operand_image(prime_bits: int, m: int) -> np.ndarray:
    """Host-only: the tensor-core operand images (uint8) of an odd prime m of
    1536 or 2048 bits, as built at key load for the RSA-3072/4096 variant-3
    path (two reduction rounds of half the prime size)."""
    ma = int_to_limbs(m, prime_bits // 32)
    out = np.zeros(rsa_tc_round_image_bytes(prime_bits), dtype=np.uint8)
    check(_lib.lib().rsa_tc_round_operand_image(prime_bits, _ptr(ma), _ptr(out), out.size))
    return out


def rsa_keyunload(ctx: int, key_id: int) -> None:
    check(_lib.lib().rsa_keyunload(ctx, key_id))


def rsa_key_info(ctx: int, key_id: int) -> tuple[int, bool, bool]:
    nb, hd, hc = ctypes.c_uint32(), ctypes.c_int32(), ctypes.c_int32()
    check(_lib.lib().rsa_key_info(ctx, key_id, ctypes.byref(nb), ctypes.byref(hd), ctypes.byref(hc)))
    return nb.value, bool(hd.value), bool(hc.value)


def rsa_modexp_key(ctx: int, key_id: int, exp_sel: int, count: int, msgs, out, op_status=None,
                   stream=None) -> None:
    check(_lib.lib().rsa_modexp_key(ctx, key_id, exp_sel, count, _ptr(msgs), _ptr(out), _ptr(op_status),
                                    _stream_ptr(stream)))


def rsa_sign_key(ctx: int, key_id: int, count: int, reps, sigs, op_status=None, stream=None) -> None:
    check(_lib.lib().rsa_sign_key(ctx, key_id, count, _ptr(reps), _ptr(sigs), _ptr(op_status),
                                  _stream_ptr(stream)))


def rsa_verify_key(ctx: int, key_id: int, count: int, sigs, reps, op_status, stream=None) -> None:
    check(_lib.lib().rsa_verify_key(ctx, key_id, count, _ptr(sigs), _ptr(reps), _ptr(op_status),
                                    _stream_ptr(stream)))


def rsa_mr_batch(ctx: int, nbits: int, count: int, cands, rounds: int, bases, verdicts, stream=None) -> None:
    check(_lib.lib().rsa_mr_batch(ctx, nbits, count, _ptr(cands), rounds, _ptr(bases), _ptr(verdicts),
                                  _stream_ptr(stream)))


def rsa_batch_gcd(ctx: int, nbits: int, count: int, moduli, gcds, flags, stream=None) -> None:
    check(_lib.lib().rsa_batch_gcd(ctx, nbits, count, _ptr(moduli), _ptr(gcds), _ptr(flags), _stream_ptr(stream)))


def rsa_batch_gcd_host(ctx: int, nbits: int, count: int, moduli: np.ndarray, gcds, flags, stream=None) -> None:
    check(_lib.lib().rsa_batch_gcd_host(ctx, nbits, count, _ptr(moduli), _ptr(gcds), _ptr(flags),
                                        _stream_ptr(stream)))


def rsa_batch_gcd_ex(ctx: int, nbits: int, count: int, moduli, gcds, flags, method: int, stream=None) -> None:
    check(_lib.lib().rsa_batch_gcd_ex(ctx, nbits, count, _ptr(moduli), _ptr(gcds), _ptr(flags), method,
                                      _stream_ptr(stream)))


def rsa_batch_gcd_method(ctx: int, nbits: int, count: int) -> int:
    """The form (RSA_GCD_SCAN or RSA_GCD_TREE) RSA_GCD_AUTO takes for count moduli."""
    m = ctypes.c_int(0)
    check(_lib.lib().rsa_batch_gcd_method(ctx, nbits, count, ctypes.byref(m)))
    return m.value


def rsa_batch_gcd_tree_bytes(nbits: int, count: int) -> int:
    """Device bytes the tree form of the batch GCD needs for count moduli."""
    b = ctypes.c_uint64(0)
    check(_lib.lib().rsa_batch_gcd_tree_bytes(nbits, count, ctypes.byref(b)))
    return b.value


def rsa_batch_gcd_plan(ctx: int, nbits: int, count: int) -> tuple[int, int]:
    """(block size, parts) of the work split rsa_batch_gcd uses for count moduli."""
    blk = ctypes.c_uint32(0)
    parts = ctypes.c_uint64(0)
    check(_lib.lib().rsa_batch_gcd_plan(ctx, nbits, count, ctypes.byref(blk), ctypes.byref(parts)))
    return blk.value, parts.value


def rsa_modexp_batch(ctx: int, count: int, key_ids, exp_sel, limb_offsets, msgs, out, op_status=None,
                     stream=None) -> None:
    check(_lib.lib().rsa_modexp_batch(ctx, count, _ptr(key_ids), _ptr(exp_sel), _ptr(limb_offsets),
                                      _ptr(msgs), _ptr(out), _ptr(op_status), _stream_ptr(stream)))


def rsa_modexp_key_host(ctx: int, key_id: int, exp_sel: int, count: int, msgs: np.ndarray, out: np.ndarray,
                        op_status: np.ndarray | None = None, stream=None) -> None:
    check(_lib.lib().rsa_modexp_key_host(ctx, key_id, exp_sel, count, _ptr(msgs), _ptr(out), _ptr(op_status),
                                         _stream_ptr(stream)))


def rsa_modexp_batch_host(ctx: int, count: int, key_ids, exp_sel, limb_offsets, total_limbs: int, msgs, out,
                          op_status=None, stream=None) -> None:
    check(_lib.lib().rsa_modexp_batch_host(ctx, count, _ptr(key_ids), _ptr(exp_sel), _ptr(limb_offsets),
                                           total_limbs, _ptr(msgs), _ptr(out), _ptr(op_status),
                                           _stream_ptr(stream)))


def rsa_sync(ctx: int, stream=None) -> int:
    """Waits for the stream; returns the device-side status (raises on CUDA errors)."""
    rc = _lib.lib().rsa_sync(ctx, _stream_ptr(stream))
    if rc == RSA_ERR_CUDA:
        raise RsaError(rc, last_error())
    return rc


def rsa_crt_decrypt_noalloc(key_record, nbits: int, count: int, msgs, out, op_status=None, stream=None) -> None:
    check(_lib.lib().rsa_crt_decrypt_noalloc(_ptr(key_record), nbits, count, _ptr(msgs), _ptr(out), _ptr(op_status),
                                             _stream_ptr(stream)))


def rsa_last_error() -> str:
    return last_error()


def rsa_set_tuning(ctx: int, nbits: int, exp_sel: int, window: int = 0, warps_per_cta: int = 0,
                   ctas_per_sm: int = 0, variant: int = 0, threads_per_op: int = 0, window_big: int = 0,
                   window_tc: int = 0, tc_min_ops: int = 0, reset: bool = False) -> None:
    if reset:
        check(_lib.lib().rsa_set_tuning(ctx, nbits, exp_sel, None))
        return
    t = rsa_tuning(window, warps_per_cta, ctas_per_sm, variant, threads_per_op, window_big, window_tc, tc_min_ops)
    check(_lib.lib().rsa_set_tuning(ctx, nbits, exp_sel, ctypes.byref(t)))


def _tuning_dict(t) -> dict:
    return {"window": t.window, "warps_per_cta": t.warps_per_cta, "ctas_per_sm": t.ctas_per_sm,
            "variant": t.variant, "threads_per_op": t.threads_per_op, "window_big": t.window_big,
            "window_tc": t.window_tc, "tc_min_ops": t.tc_min_ops}


def rsa_get_tuning(ctx: int, nbits: int, exp_sel: int) -> dict:
    t = rsa_tuning()
    check(_lib.lib().rsa_get_tuning(ctx, nbits, exp_sel, ctypes.byref(t)))
    return _tuning_dict(t)


def rsa_autotune(ctx: int, key_id: int, exp_sel: int, count: int, cache_path: str | None = None) -> dict:
    """Time the launch shapes for this key's size and kind; installs and returns the fastest."""
    t = rsa_tuning()
    ms = ctypes.c_double()
    check(_lib.lib().rsa_autotune(ctx, key_id, exp_sel, count, cache_path.encode() if cache_path else None,
                                  ctypes.byref(t), ctypes.byref(ms)))
    return dict(_tuning_dict(t), ms=ms.value)


def rsa_autotune_batch(ctx: int, count: int, key_ids, exp_sel, limb_offsets, msgs, out) -> dict:
    """Tune the ragged batch (lanes per operation, the tensor-core group, CRT
    windows, resident-CTA cap); installs the fastest as the RSA_TUNE_RAGGED
    tuning and returns it."""
    t = rsa_tuning()
    ms = ctypes.c_double()
    check(_lib.lib().rsa_autotune_batch(ctx, count, _ptr(key_ids), _ptr(exp_sel), _ptr(limb_offsets), _ptr(msgs),
                                        _ptr(out), ctypes.byref(t), ctypes.byref(ms)))
    return dict(_tuning_dict(t), ms=ms.value)


def rsa_get_stats(ctx: int) -> dict:
    s = rsa_stats()
    check(_lib.lib().rsa_get_stats(ctx, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in rsa_stats._fields_}


def rsa_products_per_op(nbits: int, exp_sel: int, e: int = 65537, window: int = 5) -> float:
    return _lib.lib().rsa_products_per_op(nbits, exp_sel, e.bit_length(), bin(e).count("1"), window)


def rsa_imad_probe(device: int = 0) -> tuple[float, float]:
    a, b = ctypes.c_double(), ctypes.c_double()
    check(_lib.lib().rsa_imad_probe(device, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


# ------------------------------------------------------------------ serving

def rsa_server_start(ctx: int, max_inflight_batches: int = 0, batch_window_us: int = 0, max_batch_ops: int = 0,
                     mem_budget_bytes: int = 0, mix_sizes: bool = False) -> None:
    flags = _lib.RSA_SERVER_MIX_SIZES if mix_sizes else 0
    cfg = _lib.rsa_server_cfg(max_inflight_batches, batch_window_us, max_batch_ops, flags, mem_budget_bytes)
    check(_lib.lib().rsa_server_start(ctx, ctypes.byref(cfg)))


def rsa_server_submit(ctx: int, key_id: int, exp_sel: int, msgs: np.ndarray, out: np.ndarray,
                      status: np.ndarray | None = None, arrive_ns: int = 0) -> int:
    """Queue one request (host buffers, which must stay alive until it completes)."""
    count = msgs.shape[0] if msgs.ndim > 1 else msgs.size
    req = _lib.rsa_request(key_id, exp_sel, count, 0, _ptr(msgs), _ptr(out), _ptr(status), arrive_ns)
    t = ctypes.c_uint64()
    check(_lib.lib().rsa_server_submit(ctx, ctypes.byref(req), ctypes.byref(t)))
    return t.value


REQUEST_DTYPE = np.dtype([("key_id", "<i4"), ("exp_sel", "<i4"), ("count", "<u4"), ("reserved", "<u4"),
                          ("msgs", "<u8"), ("out", "<u8"), ("status", "<u8"), ("arrive_ns", "<u8")])


def rsa_server_submit_many(ctx: int, reqs: np.ndarray) -> int:
    """Queue a structured array of REQUEST_DTYPE records; returns how many were accepted."""
    reqs = np.ascontiguousarray(reqs, dtype=REQUEST_DTYPE)
    acc = ctypes.c_uint32()
    check(_lib.lib().rsa_server_submit_many(ctx, reqs.ctypes.data, reqs.size, None, ctypes.byref(acc)))
    return acc.value


def rsa_server_clock(ctx: int) -> int:
    t = ctypes.c_uint64()
    check(_lib.lib().rsa_server_clock(ctx, ctypes.byref(t)))
    return t.value


def rsa_server_poll(ctx: int, ticket: int) -> int:
    d = ctypes.c_int32()
    check(_lib.lib().rsa_server_poll(ctx, ticket, ctypes.byref(d)))
    return d.value


def rsa_server_drain(ctx: int, timeout_ms: int = 0) -> None:
    check(_lib.lib().rsa_server_drain(ctx, timeout_ms))


def rsa_server_get_stats(ctx: int, reset: bool = False) -> dict:
    s = _lib.rsa_server_stats()
    check(_lib.lib().rsa_server_get_stats(ctx, ctypes.byref(s), 1 if reset else 0))
    return {k: getattr(s, k) for k, _ in _lib.rsa_server_stats._fields_}


def rsa_server_stop(ctx: int) -> None:
    check(_lib.lib().rsa_server_stop(ctx))


# ------------------------------------------------------------------ convenience wrapper

class RsaContext:
    """Owns one library context; tensors in, tensors out."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        self.device = device
        self.handle = rsa_ctx_create(device, mem_budget_bytes)
        self._bits = {}

    def close(self):
        if self.handle:
            rsa_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def keyload(self, nbits, n, e, d=None, p=None, q=None) -> int:
        kid = rsa_keyload(self.handle, nbits, n, e, d, p, q)
        self._bits[kid] = nbits
        return kid

    def keyunload(self, key_id: int) -> None:
        rsa_keyunload(self.handle, key_id)
        self._bits.pop(key_id, None)

    def modexp_key(self, key_id: int, exp_sel: int, msgs, out=None, status=None, stream=None):
        """msgs: CUDA tensor [count, L] of uint32 (or int32 bit patterns)."""
        import torch
        if out is None:
            out = torch.empty_like(msgs)
        count = msgs.shape[0] if msgs.dim() > 1 else msgs.numel()
        rsa_modexp_key(self.handle, key_id, exp_sel, count, msgs, out, status, stream)
        return out

    def sign(self, key_id: int, reps, sigs=None, status=None, stream=None):
        """reps: CUDA tensor [count, L]; returns the signatures reps^d mod n."""
        import torch
        if sigs is None:
            sigs = torch.empty_like(reps)
        count = reps.shape[0] if reps.dim() > 1 else reps.numel()
        rsa_sign_key(self.handle, key_id, count, reps, sigs, status, stream)
        return sigs

    def verify(self, key_id: int, sigs, reps, status=None, stream=None):
        """Returns an int32 CUDA tensor of verdicts: 0 valid, RSA_ERR_VERIFY, RSA_ERR_RANGE."""
        import torch
        count = sigs.shape[0] if sigs.dim() > 1 else sigs.numel()
        if status is None:
            status = torch.empty(count, dtype=torch.int32, device=sigs.device)
        rsa_verify_key(self.handle, key_id, count, sigs, reps, status, stream)
        return status

    def miller_rabin(self, nbits: int, cands, bases, verdicts=None, stream=None):
        """cands: CUDA tensor [count, nbits/32]; bases: [count, rounds, nbits/32].
        Returns int32 verdicts: 1 probable prime, 0 composite, -1 invalid."""
        import torch
        count = cands.shape[0]
        rounds = bases.shape[1] if bases.dim() == 3 else 0
        if verdicts is None:
            verdicts = torch.empty(count, dtype=torch.int32, device=cands.device)
        rsa_mr_batch(self.handle, nbits, count, cands, rounds, bases, verdicts, stream)
        return verdicts

    def batch_gcd(self, nbits: int, moduli, gcds=None, flags=None, stream=None, method: int = RSA_GCD_AUTO):
        """moduli: CUDA tensor [count, nbits/32] (int32 view of the limbs).
        Returns (gcds, flags): g_i = gcd(n_i, product of the other valid
        moduli) and int32 flags 0 coprime, 1 proper factor, 2 g = n, -1 invalid.
        method: RSA_GCD_AUTO, RSA_GCD_SCAN or RSA_GCD_TREE."""
        import torch
        count = moduli.shape[0]
        if gcds is None:
            gcds = torch.empty_like(moduli)
        if flags is None:
            flags = torch.empty(count, dtype=torch.int32, device=moduli.device)
        rsa_batch_gcd_ex(self.handle, nbits, count, moduli, gcds, flags, method, stream)
        return gcds, flags

    def modexp_key_host(self, key_id: int, exp_sel: int, msgs: np.ndarray, out: np.ndarray | None = None,
                        status: np.ndarray | None = None, stream=None) -> np.ndarray:
        msgs = np.ascontiguousarray(msgs, dtype=np.uint32)
        if out is None:
            out = np.empty_like(msgs)
        count = msgs.shape[0]
        rsa_modexp_key_host(self.handle, key_id, exp_sel, count, msgs, out, status, stream)
        return out

    def modexp_batch(self, key_ids, exp_sel, limb_offsets, msgs, out=None, status=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(msgs)
        rsa_modexp_batch(self.handle, key_ids.numel(), key_ids, exp_sel, limb_offsets, msgs, out, status, stream)
        return out

    def autotune(self, key_id: int, exp_sel: int, count: int, cache_path: str | None = None) -> dict:
        """Tune rsa_modexp_key for this key's size and kind (installs the fastest shape)."""
        return rsa_autotune(self.handle, key_id, exp_sel, count, cache_path)

    def batch_gcd_host(self, nbits: int, moduli: np.ndarray, gcds: np.ndarray | None = None,
                       flags: np.ndarray | None = None, stream=None):
        """Host-buffer batch GCD: numpy rows in, (gcds, flags) numpy arrays out."""
        moduli = np.ascontiguousarray(moduli, dtype=np.uint32)
        if gcds is None:
            gcds = np.empty_like(moduli)
        if flags is None:
            flags = np.empty(moduli.shape[0], dtype=np.int32)
        rsa_batch_gcd_host(self.handle, nbits, moduli.shape[0], moduli, gcds, flags, stream)
        return gcds, flags

    def autotune_batch(self, key_ids, exp_sel, limb_offsets, msgs, out=None) -> dict:
        """Tune rsa_modexp_batch on this batch (installs the fastest shapes)."""
        import torch
        if out is None:
            out = torch.empty_like(msgs)
        return rsa_autotune_batch(self.handle, key_ids.numel(), key_ids, exp_sel, limb_offsets, msgs, out)

    def sync(self, stream=None) -> int:
        return rsa_sync(self.handle, stream)

    def set_tuning(self, nbits, exp_sel, **kw):
        rsa_set_tuning(self.handle, nbits, exp_sel, **kw)

    def get_tuning(self, nbits, exp_sel):
        return rsa_get_tuning(self.handle, nbits, exp_sel)

    def stats(self) -> dict:
        return rsa_get_stats(self.handle)
