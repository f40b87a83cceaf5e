"""Seeded synthetic inputs for batched RSA: keys, messages, ragged mixes, arrivals.

This module is the only code shared by the CUDA path's tests/benchmark and the
CPU oracle's tests.  It holds none of the method's arithmetic: it draws random
bits and builds keys with Python's built-in arbitrary-precision integers
(``pow`` for the Miller-Rabin test and for the modular inverse, the paper's key
generation of Fig. 1), and it never calls the oracle or the GPU library.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used in its counter form: the
i-th output of a stream with key k is mix64(k + (i+1)*GAMMA).  That makes every
draw addressable, so numpy evaluates whole blocks at once, and it gives the
same numbers on x86 and Arm.

Workloads (sizes as in the benchmark configurations):
  toy      n = 17947 = 131*137, e = 131, d = 137 (paper Sec. 2 example),
           4096 single-limb packets uniform in [0, 2525]
  rsa2048  one 2048-bit key (two 1024-bit primes, Miller-Rabin 40 rounds),
           e = 65537, 65536 messages uniform in [0, n)
  rsa4096  one 4096-bit key, 16384 messages
  ragged   256 keys with sizes {1024, 2048, 3072, 4096} (p = .1/.5/.2/.2),
           Zipf(1.1) per-key counts summing to 200000, 70% CRT / 30% public
  serving  Poisson arrivals, 1..64 messages per request, keys of the ragged set
  bgcd     weak-key scan: 16384 RSA-2048-shaped moduli n = a b (a, b random odd
           1024-bit numbers with the top two bits set), 16 planted pairs that
           reuse a factor
"""
from __future__ import annotations

import hashlib
import json
import math
import multiprocessing as mp
import os
from dataclasses import dataclass, field

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1
DEFAULT_SEED = 20141465
E_PUBLIC = 65537

EXP_PUBLIC = 0        # x = e
EXP_PRIVATE_CRT = 1   # x = d through p, q
EXP_PRIVATE_PLAIN = 2  # x = d, directly mod n


# ------------------------------------------------------------------ SplitMix64

def _mix64(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def stream_key(seed: int, *tags) -> int:
    """A 64-bit stream key derived from the seed and a tuple of tags."""
    h = hashlib.sha256(repr((int(seed), tags)).encode()).digest()
    return int.from_bytes(h[:8], "little")


def draws(key: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the SplitMix64 stream ``key`` (uint64)."""
    return draws_at(key, np.arange(start, start + count, dtype=np.uint64))


def draws_at(key: int, positions: np.ndarray) -> np.ndarray:
    """Outputs at the given 0-based positions of the SplitMix64 stream ``key``."""
    with np.errstate(over="ignore"):
        i = positions.astype(np.uint64) + np.uint64(1)
        z = np.uint64(key) + i * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


class Stream:
    """Sequential reader over one counter-based stream."""

    def __init__(self, key: int):
        self.key = key
        self.pos = 0

    def u64(self) -> int:
        self.pos += 1
        return _mix64((self.key + self.pos * GAMMA) & MASK64)

    def bits(self, nbits: int) -> int:
        words = (nbits + 63) // 64
        v = 0
        for k in range(words):
            v |= self.u64() << (64 * k)
        return v & ((1 << nbits) - 1)

    def below(self, bound: int) -> int:
        """Uniform integer in [0, bound) by rejection."""
        nb = max(1, bound.bit_length())
        while True:
            v = self.bits(nb)
            if v < bound:
                return v

    def uniform01(self) -> float:
        return (self.u64() >> 11) * (1.0 / (1 << 53))


# ------------------------------------------------------------------ primes / keys

_SMALL_PRIMES = None


def small_primes(limit: int = 65536) -> np.ndarray:
    global _SMALL_PRIMES
    if _SMALL_PRIMES is None or _SMALL_PRIMES[-1] < limit - 100:
        sieve = np.ones(limit, dtype=bool)
        sieve[:2] = False
        for i in range(2, int(limit ** 0.5) + 1):
            if sieve[i]:
                sieve[i * i::i] = False
        _SMALL_PRIMES = np.nonzero(sieve)[0].astype(np.int64)
    return _SMALL_PRIMES


def miller_rabin(n: int, rounds: int, st: Stream) -> bool:
    """Probabilistic primality with ``rounds`` random bases in [2, n-2]."""
    if n < 4:
        return n in (2, 3)
    if n % 2 == 0:
        return False
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for _ in range(rounds):
        a = 2 + st.below(n - 3)
        x = pow(a, d, n)
        if x == 1 or x == n - 1:
            continue
        for _ in range(s - 1):
            x = pow(x, 2, n)
            if x == n - 1:
                break
        else:
            return False
    return True


def gen_prime(bits: int, st: Stream, e: int = E_PUBLIC, mr_rounds: int = 40) -> int:
    """Random ``bits``-bit prime with its top two bits set and gcd(e, p-1) = 1.

    A random odd start with the top two bits set is drawn, then the odd numbers
    above it are sieved by all primes below 2^16 and tested in order with
    Miller-Rabin (one round first, then the remaining rounds).
    """
    if bits < 32:
        raise ValueError("prime size below 32 bits is not supported")
    primes = small_primes()
    primes = primes[primes > 2]
    window = 4096
    while True:
        start = st.bits(bits) | (3 << (bits - 2)) | 1
        rem = np.array([start % int(p) for p in primes], dtype=np.int64)
        # candidate k is start + 2k; composite if (start + 2k) % p == 0 for some p
        alive = np.ones(window, dtype=bool)
        for p, r in zip(primes, rem):
            # smallest k >= 0 with r + 2k = 0 mod p  ->  k = (-r) * inv2 mod p
            k0 = ((p - r) * ((p + 1) // 2)) % p
            alive[k0::p] = False
        for k in np.nonzero(alive)[0]:
            cand = start + 2 * int(k)
            if cand.bit_length() != bits:
                break
            if math.gcd(e, cand - 1) != 1:
                continue
            if miller_rabin(cand, 1, st) and miller_rabin(cand, mr_rounds - 1, st):
                return cand


@dataclass
class Key:
    bits: int
    n: int
    e: int
    d: int
    p: int
    q: int

    @property
    def limbs(self) -> int:
        return self.bits // 32

    def to_json(self) -> dict:
        return {k: (hex(v) if isinstance(v, int) and k != "bits" else v)
                for k, v in self.__dict__.items()}

    @staticmethod
    def from_json(j: dict) -> "Key":
        return Key(bits=j["bits"], **{k: int(j[k], 16) for k in ("n", "e", "d", "p", "q")})


def gen_key(bits: int, seed: int, index: int = 0, e: int = E_PUBLIC, mr_rounds: int = 40) -> Key:
    """RSA key per paper Fig. 1: p != q primes of bits/2 bits, n = pq,
    phi = (p-1)(q-1), gcd(e, phi) = 1, d = e^-1 mod phi.  Ordered so p > q."""
    if bits % 64 != 0 or bits < 64:
        raise ValueError("key size must be a positive multiple of 64 bits")
    st = Stream(stream_key(seed, "key", bits, index, e))
    while True:
        p = gen_prime(bits // 2, st, e, mr_rounds)
        q = gen_prime(bits // 2, st, e, mr_rounds)
        if p == q:
            continue
        if p < q:
            p, q = q, p
        n = p * q
        assert n.bit_length() == bits
        phi = (p - 1) * (q - 1)
        d = pow(e, -1, phi)
        return Key(bits=bits, n=n, e=e, d=d, p=p, q=q)


def _gen_key_job(args):
    bits, seed, index, e, rounds = args
    return gen_key(bits, seed, index, e, rounds).to_json()


_CACHE_DIR = os.environ.get("RSA_WORKLOAD_CACHE",
                            os.path.join(os.path.dirname(os.path.abspath(__file__)), ".cache"))


def _source_tag() -> str:
    with open(os.path.abspath(__file__), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def gen_keys(specs: list[tuple[int, int]], seed: int, e: int = E_PUBLIC, mr_rounds: int = 40,
             processes: int = 0, cache: bool = True) -> list[Key]:
    """Keys for (bits, index) specs, generated in a spawn-context process pool
    and cached on disk under a tag of this file's contents."""
    tag = hashlib.sha256(repr((seed, e, mr_rounds, specs, _source_tag())).encode()).hexdigest()[:24]
    path = os.path.join(_CACHE_DIR, "keys_%s.json" % tag)
    if cache and os.path.exists(path):
        with open(path) as f:
            return [Key.from_json(j) for j in json.load(f)]
    jobs = [(b, seed, i, e, mr_rounds) for (b, i) in specs]
    nproc = processes or min(len(jobs), os.cpu_count() or 1)
    if nproc > 1 and len(jobs) > 1:
        ctx = mp.get_context("spawn")
        with ctx.Pool(nproc) as pool:
            # largest keys first so the pool's tail is short
            order = sorted(range(len(jobs)), key=lambda k: -jobs[k][0])
            res = pool.map(_gen_key_job, [jobs[k] for k in order], chunksize=1)
            out = [None] * len(jobs)
            for k, r in zip(order, res):
                out[k] = r
    else:
        out = [_gen_key_job(j) for j in jobs]
    if cache:
        os.makedirs(_CACHE_DIR, exist_ok=True)
        tmp = path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(out, f)
        os.replace(tmp, path)
    return [Key.from_json(j) for j in out]


# ------------------------------------------------------------------ messages

def int_to_limbs(x: int, nlimbs: int) -> np.ndarray:
    return np.frombuffer(x.to_bytes(4 * nlimbs, "little"), dtype="<u4").astype(np.uint32)


def limbs_to_int(a) -> int:
    return int.from_bytes(np.ascontiguousarray(a, dtype=np.uint32).astype("<u4").tobytes(), "little")


def rows_to_ints(rows: np.ndarray) -> list[int]:
    rows = np.ascontiguousarray(rows, dtype=np.uint32).astype("<u4")
    nb = rows.shape[1] * 4
    buf = rows.tobytes()
    return [int.from_bytes(buf[i * nb:(i + 1) * nb], "little") for i in range(rows.shape[0])]


def ints_to_rows(vals: list[int], nlimbs: int) -> np.ndarray:
    buf = b"".join(v.to_bytes(4 * nlimbs, "little") for v in vals)
    return np.frombuffer(buf, dtype="<u4").astype(np.uint32).reshape(len(vals), nlimbs)


def messages_below(n: int, count: int, seed: int, tag) -> np.ndarray:
    """``count`` messages uniform in [0, n) as rows of limbs (rejection sampling:
    draw as many bits as n has, redraw the rows that are >= n)."""
    nl = max(1, (n.bit_length() + 31) // 32)
    nbits = n.bit_length()
    words64 = (nl + 1) // 2
    key = stream_key(seed, "msg", tag)
    out = np.zeros((count, nl), dtype=np.uint32)
    todo = np.arange(count)
    attempt = 0
    top_mask = np.uint32((1 << (nbits - 32 * (nl - 1))) - 1) if nbits % 32 else np.uint32(0xFFFFFFFF)
    while todo.size:
        # row r, attempt a reads words [(a*count + r) * words64, ... + words64)
        base = (attempt * count + todo) * words64
        idx = base[:, None] + np.arange(words64)[None, :]
        w = draws_at(key, idx.ravel()).reshape(idx.shape)
        limbs = w.view(np.uint32).reshape(todo.size, 2 * words64)[:, :nl].copy()
        limbs[:, nl - 1] &= top_mask
        vals = rows_to_ints(limbs)
        ok = np.array([v < n for v in vals], dtype=bool)
        out[todo[ok]] = limbs[ok]
        todo = todo[~ok]
        attempt += 1
    return out


# ------------------------------------------------------------------ workloads

TOY_N, TOY_E, TOY_D, TOY_P, TOY_Q = 17947, 131, 137, 137, 131
TOY_D_CORRECTED = 14171   # e^-1 mod phi(17947) = 17680; the printed d = 137 is not an inverse
PAPER_PACKETS = [1500, 1700, 1111, 411, 413, 217, 2415, 1908, 1413]


def toy_packets(count: int = 4096, seed: int = DEFAULT_SEED) -> np.ndarray:
    """``count`` uint32 values uniform in [0, 2525] (single-limb messages)."""
    st = Stream(stream_key(seed, "toy"))
    return np.array([st.below(2526) for _ in range(count)], dtype=np.uint32)


def rsa_single(bits: int, count: int, seed: int = DEFAULT_SEED, mr_rounds: int = 40):
    """One ``bits``-bit key and ``count`` messages uniform in [0, n)."""
    key = gen_keys([(bits, 0)], seed, mr_rounds=mr_rounds)[0]
    msgs = messages_below(key.n, count, seed, ("single", bits))
    return key, msgs


@dataclass
class RaggedBatch:
    keys: list
    key_ids: np.ndarray      # [ops] index into keys
    exp_sel: np.ndarray      # [ops] EXP_PUBLIC or EXP_PRIVATE_CRT
    msgs: list               # [ops] numpy rows (each op its key's limb count)
    offsets: np.ndarray = field(default=None)  # [ops] limb offset into the packed buffer
    packed: np.ndarray = field(default=None)   # all messages back to back


def ragged_key_specs(num_keys: int, seed: int, sizes=(1024, 2048, 3072, 4096),
                     probs=(0.1, 0.5, 0.2, 0.2)) -> list[tuple[int, int]]:
    st = Stream(stream_key(seed, "ragged-sizes"))
    cum = np.cumsum(probs)
    specs = []
    for i in range(num_keys):
        u = st.uniform01()
        b = sizes[int(np.searchsorted(cum, u, side="right"))] if u < cum[-1] else sizes[-1]
        specs.append((b, i))
    return specs


def zipf_counts(num_keys: int, total: int, s: float, seed: int) -> np.ndarray:
    """Per-key counts: ranks 1..K by a seeded permutation, weight r^-s,
    floor(total*w/sum w) plus largest-remainder top-up, at least 1 each."""
    st = Stream(stream_key(seed, "zipf"))
    perm = list(range(num_keys))
    for i in range(num_keys - 1, 0, -1):   # Fisher-Yates
        j = st.below(i + 1)
        perm[i], perm[j] = perm[j], perm[i]
    ranks = np.empty(num_keys, dtype=np.int64)
    ranks[np.array(perm)] = np.arange(1, num_keys + 1)
    w = ranks.astype(np.float64) ** (-s)
    share = total * w / w.sum()
    counts = np.maximum(np.floor(share).astype(np.int64), 1)
    rem = total - counts.sum()
    frac = share - np.floor(share)
    order = np.argsort(-frac, kind="stable")
    k = 0
    while rem > 0:
        counts[order[k % num_keys]] += 1
        rem -= 1
        k += 1
    while rem < 0:   # only if the minimum of 1 overshot
        i = int(np.argmax(counts))
        counts[i] -= 1
        rem += 1
    return counts


def ragged(num_keys: int = 256, total: int = 200000, seed: int = DEFAULT_SEED,
           crt_frac: float = 0.7, zipf_s: float = 1.1, mr_rounds: int = 40,
           keys: list | None = None) -> RaggedBatch:
    specs = ragged_key_specs(num_keys, seed)
    if keys is None:
        keys = gen_keys(specs, seed, mr_rounds=mr_rounds)
    counts = zipf_counts(num_keys, total, zipf_s, seed)
    st = Stream(stream_key(seed, "ragged-kind"))
    key_ids, sels, msgs = [], [], []
    for kid, (key, c) in enumerate(zip(keys, counts)):
        rows = messages_below(key.n, int(c), seed, ("ragged", kid))
        for r in range(int(c)):
            key_ids.append(kid)
            sels.append(EXP_PRIVATE_CRT if st.uniform01() < crt_frac else EXP_PUBLIC)
            msgs.append(rows[r])
    # interleave keys: a seeded shuffle of the op order (arrivals are mixed)
    order = list(range(len(key_ids)))
    for i in range(len(order) - 1, 0, -1):
        j = st.below(i + 1)
        order[i], order[j] = order[j], order[i]
    key_ids = np.array([key_ids[i] for i in order], dtype=np.int32)
    sels = np.array([sels[i] for i in order], dtype=np.uint8)
    msgs = [msgs[i] for i in order]
    sizes = np.array([m.size for m in msgs], dtype=np.uint64)
    offsets = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.uint64)
    packed = np.concatenate(msgs).astype(np.uint32) if msgs else np.zeros(0, np.uint32)
    return RaggedBatch(keys=keys, key_ids=key_ids, exp_sel=sels, msgs=msgs,
                       offsets=offsets, packed=packed)


@dataclass
class Request:
    t_arrive: float     # seconds from start
    key_id: int
    exp_sel: int
    count: int


def poisson_requests(rate: float, duration: float, num_keys: int, seed: int,
                     min_msgs: int = 1, max_msgs: int = 64, crt_frac: float = 0.7) -> list:
    """Poisson arrivals (exponential gaps, mean 1/rate) over ``duration`` seconds."""
    st = Stream(stream_key(seed, "arrivals", rate))
    t, out = 0.0, []
    while True:
        t += -math.log(1.0 - st.uniform01()) / rate
        if t >= duration:
            return out
        out.append(Request(t_arrive=t, key_id=st.below(num_keys),
                           exp_sel=EXP_PRIVATE_CRT if st.uniform01() < crt_frac else EXP_PUBLIC,
                           count=min_msgs + st.below(max_msgs - min_msgs + 1)))


# ------------------------------------------------------------------ batch GCD (weak-key scan)

def random_odd_halves(count: int, bits: int, seed: int, tag) -> list[int]:
    """``count`` random odd ``bits``-bit integers with the top two bits set."""
    words64 = (bits + 63) // 64
    w = draws(stream_key(seed, "half", bits, tag), 0, count * words64).reshape(count, words64)
    vals = rows_to_ints(w.view(np.uint32).reshape(count, 2 * words64))
    top = 3 << (bits - 2)
    mask = (1 << bits) - 1
    return [(v & mask) | top | 1 for v in vals]


def weak_key_moduli(count: int = 16384, bits: int = 2048, seed: int = DEFAULT_SEED, shared: int = 16):
    """RSA-shaped moduli n_i = a_i b_i (a_i, b_i random odd bits/2-bit numbers,
    top two bits set, so n_i has bits or bits - 1 bits) with ``shared`` planted
    pairs (i, j): n_j = a_i b_j reuses n_i's factor a_i.  The halves are not
    forced to be prime (the scan's arithmetic is the same), so unplanted pairs
    may also share small factors.  Returns (rows (count, bits/32) uint32, pairs)."""
    a = random_odd_halves(count, bits // 2, seed, ("a", count))
    b = random_odd_halves(count, bits // 2, seed, ("b", count))
    pairs = []
    if count >= 2 and shared:
        key = stream_key(seed, "pairs", count, bits)
        pos = (draws(key, 0, 4 * shared) % np.uint64(count)).astype(np.int64).tolist()
        used = set()
        for k in range(0, len(pos), 2):
            i, j = pos[k], pos[k + 1]
            if i == j or i in used or j in used:
                continue
            used.update((i, j))
            pairs.append((i, j))
            if len(pairs) == shared:
                break
    for i, j in pairs:
        a[j] = a[i]
    return ints_to_rows([x * y for x, y in zip(a, b)], bits // 32), pairs
