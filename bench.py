"""Benchmark: RSA-2048 CRT decryptions per second on GB300 (plus roofline data).

One step = one rsa_modexp_key call decrypting the whole batch (65536 RSA-2048
ciphertexts under one seeded key, CRT + constant-time fixed window), inputs
resident in HBM.  Prints ONE JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload rsa2048|rsa4096] [--window 5] [--no-e2e] [--no-cpu]

Multi-GPU (torchrun, one process per GPU): every rank decrypts its own full
batch (weak scaling, no data exchange); the timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

WORKLOADS = {
    "rsa2048": dict(bits=2048, count=65536),
    "rsa3072": dict(bits=3072, count=16384),
    "rsa4096": dict(bits=4096, count=16384),
}


def workload_desc(bits, count, kind="crt"):
    """Names the single-key workload: key size, message count, limb layout and the
    operation (CRT decryption with d, or encryption with e = 65537)."""
    what = "CRT decryption" if kind == "crt" else "public-exponent encryption (e=65537)"
    items = "ciphertexts" if kind == "crt" else "messages"
    return ("RSA-%d %s: 1 seeded key (two %d-bit primes, Miller-Rabin 40 rounds, e=65537), %d %s uniform "
            "in [0,n) as %d x u32 limbs" % (bits, what, bits // 2, count, items, bits // 32))

# DRAM traffic of the benchmark's kernel from one ncu capture (the summaries
# under profiles/ named in "source"), valid only while the kernel sources hash
# to the recorded stamp and the window matches; otherwise reported as null.
PROFILED_TRAFFIC = {
    # (workload, variant): one ncu capture of that kernel, valid while its sources hash to the stamp
    ("rsa2048", 3): {"window": 3, "stamp": "364df77860a7059c", "dram_bytes_per_op": 976.6,
                     "files": ["crt_tc.cu", "crt_tc.h", "tc.cuh", "mont.cuh", "kernels.cuh", "keyrec.h"],
                     "source": "profiles/crt_tc_half_kernel_rsa2048_w3_ncu_full.md",
                     # what binds the kernel, from the same capture (percent of peak while active)
                     "pipes": {"issue_active_pct": 53.8, "warps_active_pct": 25.0, "alu_pipe_pct": 44.6,
                               "fma_pipe_pct": 38.9, "tensor_pipe_pct": 20.3,
                               "top_stalls": ["wait", "math_pipe_throttle", "long_scoreboard"],
                               "reading": "latency and issue: no pipe saturated; 16 warps per SM (TMEM holds four "
                                          "128-column tiles), fixed-latency carry-chain waits"}},
    ("rsa4096", 3): {"window": 3, "stamp": "ace8eb20c3bbdeff", "dram_bytes_per_op": 2127.9,
                     "files": ["crt_tc4.cu", "crt_tc.h", "tc.cuh", "mont.cuh", "kernels.cuh", "keyrec.h"],
                     "source": "profiles/crt_tc4_half_kernel_rsa4096_w3_ncu_full.md",
                     "pipes": {"issue_active_pct": 39.2, "warps_active_pct": 12.5, "alu_pipe_pct": 32.5,
                               "fma_pipe_pct": 31.2, "tensor_pipe_pct": 14.0,
                               "top_stalls": ["wait", "long_scoreboard", "math_pipe_throttle"],
                               "reading": "latency: 8 warps per SM (two tiles of 256 TMEM columns, 255 "
                                          "registers), carry-chain waits poorly hidden"}},
    ("rsa2048", "public-tc"): {"window": None, "stamp": "ace8eb20c3bbdeff", "dram_bytes_per_op": 263.6,
                               "files": ["crt_tc4.cu", "crt_tc.h", "tc.cuh", "mont.cuh", "kernels.cuh", "keyrec.h"],
                               "source": "profiles/pub_tc4_kernel_rsa2048_e65537_ncu_full.md",
                               "pipes": {"issue_active_pct": 33.2, "warps_active_pct": 12.5, "alu_pipe_pct": 23.5,
                                         "fma_pipe_pct": 28.1, "tensor_pipe_pct": 12.2,
                                         "top_stalls": ["wait", "barrier", "long_scoreboard"],
                                         "reading": "latency: 8 warps per SM, 19 Montgomery steps per tile, "
                                                    "tile barriers and per-CTA operand loads weigh more"}},
    ("rsa2048", 1): {"window": 4, "stamp": "2c547aada0325644", "dram_bytes_per_op": 257607.0,
                     "files": ["kernels.cuh", "mont.cuh", "inst_unit.cuh", "inst_h32.cu", "keyrec.h"],
                     "source": "profiles/crt_kernel_rsa2048_w4_cios_ncu_full.md"},
}


def kernel_stamp(files) -> str:
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1407_1465_gb300", "csrc")
    for fn in files:
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


IMAD_PER_SM_CLK = 64        # 32-bit integer multiply(-add) results per SM per clock
IMAD_PER_PRODUCT = 2        # a 32x32->64 word product = low half + high half


def derived_peak_tprod(sm_count: int, sm_mhz: float) -> float:
    """Word products per second (x1e12) the IMAD pipe would allow at sm_mhz if the
    high-half multiply issued at the full rate (it issues at about half on GB300)."""
    return sm_count * IMAD_PER_SM_CLK * sm_mhz * 1e6 / IMAD_PER_PRODUCT / 1e12


def sm_count_of(device: int) -> int:
    import torch
    return int(torch.cuda.get_device_properties(device).multi_processor_count)


_PEAKS = {}


def measured_imad_peak(device: int) -> dict:
    """The IMAD roofline denominators measured on this GPU, in this run, by the
    library's probe kernels (rsa_imad_probe, best of three): 32-bit multiply-add
    lane operations per second, and 32x32->64 word products per second of
    mad.lo.cc / madc.hi.cc carry chains shaped like the Montgomery product (the
    instruction form every CUDA-core kernel here issues).  Word-product
    fractions are taken against the carry-chain figure."""
    if device in _PEAKS:
        return _PEAKS[device]
    from paper_1407_1465_gb300 import rsa_imad_probe
    lanes, chain = 0.0, 0.0
    for _ in range(3):
        a, b = rsa_imad_probe(device)
        lanes, chain = max(lanes, a), max(chain, b)
    sms = sm_count_of(device)
    _PEAKS[device] = {"chain_tprod": chain / 1e12, "imad_lane_tops": lanes / 1e12, "sm_count": sms,
                      "derived_tprod": derived_peak_tprod(sms, 2070.0)}
    return _PEAKS[device]


def alu_roofline(achieved: float, device: int, what: str) -> dict:
    """A word-product roofline against the measured carry-chain peak."""
    pk = measured_imad_peak(device)
    return {"bound": "alu", "achieved": achieved, "peak": pk["chain_tprod"], "unit": "Tprod/s",
            "frac": achieved / pk["chain_tprod"], "peak_source": "measured",
            "peak_note": "rsa_imad_probe in this run on this GPU (%d SMs): carry-chain word products/s of the "
                         "kernels' product-scan rows (mad.lo.cc + madc.hi.cc chains, rows overlapping as in the "
                         "kernels), the faster of two occupancies; independent mad.lo/mad.hi lane-ops "
                         "%.2f T/s; the unit-count figure %.2f T products/s assumes a full-rate high-half multiply"
                         % (pk["sm_count"], pk["imad_lane_tops"], pk["derived_tprod"]),
            "what": what}


def tc_work_per_op(bits: int, window: int):
    """CUDA-core word products and tensor-core FLOPs of one CRT decryption on the
    tensor-core path (variant 3): per half, 2 input products + 2^w - 2 table
    products + (windows - 1) * (w + 1) window steps (+1 for q leaving Montgomery
    form); squarings issue H(H+1)/2 word products, other products H^2; every step
    runs two fp16 MMAs of 9 K-steps (M = 128 rows: 2 * 128 * 16 FLOPs per row
    each); Garner adds two CIOS products and one H x H product.
    Returns (issued word products, issued MMA FLOPs, method MMA FLOPs): the
    method's share of the MMAs is the nonzero part of the two Toeplitz products
    per step, without the bias block -- mu = T_lo * m' mod R needs the byte
    products of columns 0..D-1 (D(D+1)/2 of them, D = 4H digits) and mu * m the
    byte products of positions D-4 .. 2D-5 (what MMA 2 produces)."""
    H = bits // 64
    D = 4 * H
    nwin = -(-32 * H // window)
    steps_half = (1 << window) + (nwin - 1) * (window + 1)
    squares_half = 1 + (nwin - 1) * window
    steps = 2 * steps_half + 1
    mults = steps - 2 * squares_half
    issued = 2 * squares_half * (H * (H + 1) // 2) + mults * H * H + 2 * (2 * H * H + H) + H * H
    tensor_flops = steps * 2 * 9 * 2 * 128 * 16
    mma1 = D * (D + 1) // 2
    mma2 = sum(min(j, D - 1) - max(0, j - (D - 1)) + 1 for j in range(D - 4, 2 * D - 4))
    method_flops = steps * 2 * (mma1 + mma2)
    return issued, tensor_flops, method_flops


def tc4_work_per_op(window: int, bits: int = 4096):
    """CUDA-core word products and tensor-core FLOPs of one RSA-3072/4096 CRT
    decryption on the tensor-core path (primes of H = bits/64 limbs, two
    reduction rounds of r = 2^(16H) per Montgomery product, D = 2H digits): per half 2 input products, 2^w - 2
    table products, (windows - 1)(w + 1) window steps (+1 for q leaving
    Montgomery form); a squaring issues H(H+1)/2 word products (cross products
    once), another step H x H, and every step two rounds of MMA 1 (N = D) and
    MMA 2 (N = 2D), D/16 + 1 K-steps each; Garner adds two CIOS products and
    one H x H product.
    Returns (issued word products, issued MMA FLOPs, method MMA FLOPs): the
    method's share of a round is the nonzero part of its two Toeplitz products,
    D(D+1)/2 byte products for mu = (T mod r) m' mod r and those of positions
    D-4 .. 3D-5 of mu * m (m of 2D digits)."""
    H = bits // 64
    D = 2 * H
    nwin = -(-32 * H // window)
    steps = 2 * ((1 << window) + (nwin - 1) * (window + 1)) + 1
    squares = 2 * (1 + (nwin - 1) * window)
    issued = squares * (H * (H + 1) // 2) + (steps - squares) * H * H + 2 * (2 * H * H + H) + H * H
    ks = D // 16 + 1                     # K-steps of 16 digits, the bias block included
    issued_flops = steps * 2 * (ks * 2 * 16 * D + ks * 2 * 16 * 2 * D)   # per round: MMA 1 (N = D), MMA 2 (N = 2D)
    mma1 = D * (D + 1) // 2
    mma2 = sum(min(j, D - 1) - max(0, j - (2 * D - 1)) + 1 for j in range(D - 4, 3 * D - 4))
    method_flops = steps * 2 * 2 * (mma1 + mma2)
    return issued, issued_flops, method_flops


def pub_tc_work_per_op(e: int, H: int = 64):
    """CUDA-core word products and tensor-core FLOPs of one RSA-2048 public-
    exponent operation on the tensor-core path (n of H = 64 limbs, two
    reduction rounds of 2^1024 per Montgomery product, as for an RSA-4096
    prime): x R with R^2, e_bits - 1 squarings (H(H+1)/2 word products each),
    popcount(e) - 1 multiplications by x R and the product by 1 that leaves
    Montgomery form (H^2 each), and per Montgomery product the MMAs of
    tc4_work_per_op.  Returns (issued word products, issued MMA FLOPs, method
    MMA FLOPs)."""
    D = 2 * H
    squares = e.bit_length() - 1
    others = 2 + bin(e).count("1") - 1
    steps = squares + others
    issued = squares * (H * (H + 1) // 2) + others * H * H
    ks = D // 16 + 1
    issued_flops = steps * 2 * (ks * 2 * 16 * D + ks * 2 * 16 * 2 * D)
    mma1 = D * (D + 1) // 2
    mma2 = sum(min(j, D - 1) - max(0, j - (2 * D - 1)) + 1 for j in range(D - 4, 3 * D - 4))
    return issued, issued_flops, steps * 2 * 2 * (mma1 + mma2)


def pub_tc_taken(bits: int, e: int, count: int, variant: int) -> bool:
    """Whether rsa_modexp_key runs a public exponent on the tensor cores:
    2048-bit keys, variant 3, or automatically (variant 0) for exponents up to
    64 bits in batches of at least 4096 operations."""
    return bits == 2048 and (variant == 3 or (variant == 0 and e.bit_length() <= 64 and count >= 4096))


def measured_bf16_tflops():
    """Burst dense bf16 TFLOP/s from MEASURED_PEAKS.json (fp16 runs at the same
    rate), else the fallback figure for GB300."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        loaded = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                name = line.split(":", 1)[1].strip()
                vendor = next((l.split(":", 1)[1].strip() for l in out.splitlines()
                               if l.lower().startswith("vendor id:")), "")
                return (vendor + " " + name).strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def cpu_baseline(key, rows, target_s: float = 12.0, public: bool = False, e: int = 0) -> dict:
    """The oracle (as written) on every host core, on a bounded sample: its CRT
    routine for decryptions, its left-to-right binary method with e for encryptions."""
    import oracle
    threads = oracle.default_threads()

    def run(r):
        if public:
            oracle.modexp_batch(r, e or key.e, key.n, threads=threads)
        else:
            oracle.crt_batch(r, key.d, key.p, key.q, threads=threads)

    probe = min(rows.shape[0], max(threads * 4, 64))
    t0 = time.perf_counter()
    run(rows[:probe])
    rate = probe / (time.perf_counter() - t0)
    n = int(min(rows.shape[0], max(probe, rate * target_s)))
    t0 = time.perf_counter()
    run(rows[:n])
    dt = time.perf_counter() - t0
    what = ("left-to-right binary modexp with e" if public else "CRT routine") + \
        " (schoolbook multiply + Algorithm D + binary square-and-multiply)"
    return {"value": n / dt, "unit": "encryptions/s" if public else "decrypts/s", "cores": threads,
            "cpu_model": cpu_model(), "kind": "oracle",
            "sample": "first %d of the %d messages, oracle %s, %d POSIX threads, %.1f s"
                      % (n, rows.shape[0], what, threads, dt)}


def run_toy(args):
    """The paper's own example (Sec. 2): n = 17947 = 131*137, e = 131, d = 137; 4096
    single-limb packets uniform in [0, 2525], encrypted then decrypted (plain d, as
    printed), one launch each per step.  Launch-latency bound: reported as ops/s
    and microseconds per launch, no roofline claim."""
    import torch
    from paper_1407_1465_gb300 import (RSA_EXP_PRIVATE_PLAIN, RSA_EXP_PUBLIC, RsaContext, build,
                                       rsa_modexp_key)
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ctx = RsaContext(0)
    t = workloads
    kid = ctx.keyload(32, t.TOY_N, t.TOY_E, t.TOY_D, t.TOY_P, t.TOY_Q)
    pk = torch.from_numpy(t.toy_packets(4096).view(np.int32)).to(dev)
    enc, dec = torch.empty_like(pk), torch.empty_like(pk)
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream

    def step():
        rsa_modexp_key(ctx.handle, kid, RSA_EXP_PUBLIC, 4096, pk, enc, None, sptr)
        rsa_modexp_key(ctx.handle, kid, RSA_EXP_PRIVATE_PLAIN, 4096, enc, dec, None, sptr)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        step()
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.steps
    import oracle
    want = [oracle.modexp(int(m), t.TOY_D, t.TOY_N) for m in enc.cpu().numpy().view(np.uint32)[:64]]
    if list(dec.cpu().numpy().view(np.uint32)[:64]) != want:
        raise RuntimeError("toy results differ from the oracle")
    line = {"metric": "toy key (n=17947, e=131, d=137): modexps/sec", "value": 8192 / (ms / 1e3),
            "unit": "ops/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "us_per_launch": ms * 1e3 / 2, "higher_is_better": True, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "4096 packets uniform in [0,2525], encrypt (e=131) + decrypt (d=137) per step"}}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def mr_issued_products(cands: np.ndarray, rounds: int, L: int = 32, W: int = 4) -> float:
    """Word products of one rsa_mr_batch launch (one thread per candidate, 32
    per warp): per candidate log2(L/2) squarings for R^2 mod n,
    then per round 1 (into Montgomery form) + 2^W - 2 table entries +
    (32L/W - 1)(W + 1) window steps + the warp's largest s - 1 squarings."""
    mm = 2 * L * L + L
    # s = trailing zero bits of n - 1 (n odd: n - 1 is n with bit 0 cleared), as
    # the kernel finds it: the first nonzero limb, then its trailing zeros
    m = cands.astype(np.uint64)
    m[:, 0] &= np.uint64(0xFFFFFFFE)
    nz = m != 0
    first = np.where(nz.any(axis=1), nz.argmax(axis=1), L - 1)
    word = m[np.arange(len(m)), first]
    tz = np.zeros(len(m), dtype=np.int64)
    for b in range(32):
        tz += ((word & np.uint64((1 << (b + 1)) - 1)) == 0) & (word != 0)
    s = 32 * first.astype(np.int64) + tz
    count = len(cands)
    warps = -(-count // 32)
    s_pad = np.concatenate([s, np.full(warps * 32 - count, s[-1] if count else 0)]).reshape(warps, 32)
    sq_tail = np.maximum(s_pad.max(axis=1) - 1, 0).sum() * 32
    per_round = 1 + (2 ** W - 2) + (32 * L // W - 1) * (W + 1)
    sq_to_r2 = {16: 3, 32: 4, 64: 5}[L]
    return float(mm) * (sq_to_r2 * warps * 32 + rounds * (per_round * warps * 32 + sq_tail))


def run_mr(args):
    """Key generation's primality step: one Miller-Rabin round per seeded odd
    candidate of --mr-bits bits (1024 default, the primes of RSA-2048; 2048 for
    RSA-4096; top bit set, bases in [2, n/2)), 65536 candidates per step, all
    device-resident; a sample of verdicts is checked against the oracle.
    Reported as rounds/s."""
    import torch
    from paper_1407_1465_gb300 import RsaContext, build
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    count = args.count or 65536
    bits = args.mr_bits
    L = bits // 32
    rng = np.random.default_rng(workloads.DEFAULT_SEED + bits)
    cands = rng.integers(0, 1 << 32, size=(count, L), dtype=np.uint64).astype(np.uint32)
    cands[:, 0] |= 1
    cands[:, L - 1] |= 0x80000000
    bases = rng.integers(0, 1 << 32, size=(count, 1, L), dtype=np.uint64).astype(np.uint32)
    bases[:, 0, L - 1] &= 0x3FFFFFFF
    bases[:, 0, 0] |= 2
    ctx = RsaContext(0, mem_budget_bytes=4 << 30)
    c = torch.from_numpy(cands.view(np.int32)).to(dev)
    b = torch.from_numpy(bases.view(np.int32)).to(dev)
    v = torch.empty(count, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 1)):
        ctx.miller_rabin(bits, c, b, v, stream.cuda_stream)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(args.steps):
        ctx.miller_rabin(bits, c, b, v, stream.cuda_stream)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / args.steps
    import oracle
    got = v.cpu().numpy()
    idx = np.arange(0, count, max(1, count // 24))
    want = [oracle.miller_rabin(workloads.rows_to_ints(cands[i:i + 1])[0],
                                workloads.rows_to_ints(bases[i, :, :])) for i in idx]
    if list(got[idx]) != want:
        raise RuntimeError("Miller-Rabin verdicts differ from the oracle")
    issued = mr_issued_products(cands, rounds=1, L=L)
    achieved = issued / (ms / 1e3) / 1e12
    roofline = alu_roofline(achieved, 0, "CIOS Montgomery products (2L^2 + L word products each) the kernel runs: "
                                         "R^2 by log2(L/2) squarings, to Montgomery form, 14 table entries, 8L - 1 "
                                         "windows x 5 steps, and each warp's largest s - 1 squarings")
    roofline.update({"traffic": None, "issued_products_per_step": issued})
    line = {"metric": "Miller-Rabin rounds/sec (%d-bit candidates)" % bits, "value": count / (ms / 1e3),
            "unit": "rounds/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "probable_primes_in_batch": int((got == 1).sum()), "roofline": roofline,
            "config": {"workload": "%d seeded odd %d-bit candidates, one base each, one launch per step" % (count, bits)}}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def bgcd_issued_products(count: int, L: int, blk: int, parts: int) -> float:
    """Word products the batch-GCD kernels issue (block products, per-modulus
    word reductions L per word, Montgomery multiplications 2L^2 + L each; the
    parts' partial products are multiplied pairwise, parts - 1 products per
    modulus in all)."""
    nblk = -(-count // blk)
    mm = 2 * L * L + L
    own = min(32, count)
    pre = nblk * L * L * blk * (blk - 1) / 2
    per_lane = (count - own) * L * L + max(0, nblk - -(-own // blk)) * mm + (own - 1) * mm + (parts - 1) * mm
    return pre + count * per_lane


def bgcd_tree_work(count: int, L: int, t0: int = -1, school_max: int = 512, tile: int = 4096) -> dict:
    """Work of one tree-form batch GCD (the product sequence of
    batch_gcd_tree_run): product tree; per remainder level from the top the
    squares, the inverses (Newton from one word at the top level, one product
    from the parent's below), the two products of the remainder step -- below
    the top level with the level's shared transforms (each node's square
    transformed once for two products, the parent's inverse and value once
    for both children); the leaves.  Products of up to school_max words are schoolbook
    (word products); longer ones are three-prime transforms, counted in
    Montgomery products mod the primes: log2(n)/2 per word and transform, one
    per word for a pointwise product (two for a kept square), six per column of
    the recombination (19 columns per 16 words)."""
    if t0 < 0:
        t0 = 4 if L >= 64 else 5 if L >= 32 else 6        # the library's default leaf level
    K = 2
    while K < count:
        K *= 2
    T = K.bit_length() - 1
    t0 = min(t0, T)
    w = {"school_products": 0, "montgomery_products": 0, "transforms": 0, "products": 0}

    def log2(n):
        return n.bit_length() - 1

    def transform(cnt, n, pointwise=0):
        es = -(-cnt * n // tile) * tile
        w["transforms"] += 3
        w["montgomery_products"] += 3 * ((es // 2) * log2(n) + pointwise * es)

    def recombine(cnt, hi):
        w["montgomery_products"] += 6 * cnt * (-(-hi // 16)) * 19

    def mul(na, nb, cnt, hi, square=False):
        w["products"] += cnt
        if na + nb <= school_max:
            w["school_products"] += cnt * na * nb
            return
        n = 1
        while n < na + nb:
            n *= 2
        if not square:
            transform(cnt, n)
        transform(cnt, n, pointwise=1)
        transform(cnt, n)
        recombine(cnt, hi)

    for t in range(T):
        st = L << t
        mul(st, st, K >> (t + 1), 2 * st)
    for t in range(T - 1, t0 - 1, -1):
        st, cnt = L << t, K >> t
        k = 2 * st
        if t + 1 < T and 2 * k >= tile:
            n = 2 * k
            w["products"] += 3 * cnt
            mul(st, st, cnt, k, square=True)            # Y = X^2 carried into words
            transform(cnt, n)                           # Y^, kept for two products
            transform(cnt // 2, n)                      # parent's mu
            transform(cnt, n, pointwise=1)              # Y_sibling mu_parent, inverse
            recombine(cnt, k)
            transform(cnt, n)                           # mu
            transform(cnt // 2, n)                      # parent's Z
            transform(cnt, n, pointwise=1)              # mu Z_parent, inverse
            recombine(cnt, k)
            transform(cnt, n)                           # q
            transform(cnt, n, pointwise=1)              # q Y, inverse
            recombine(cnt, 2 * k + 1)
            continue
        mul(st, st, cnt, k, square=True)
        if t == T - 1:
            wd = 1
            while wd < k:
                mul(2 * wd, wd, cnt, 2 * wd)
                mul(wd, wd, cnt, wd)
                wd *= 2
        else:
            mul(k, k, cnt, k)
        mul(k, k, cnt, k)
        mul(k, k, cnt, 2 * k + 1)
    M = 2 * (L << t0) + 1
    w["leaf_products"] = count * (M * 2 * L + 2 * L * L)
    w.update(K=K, T=T, t0=t0)
    return w


def bgcd_measure(count: int, method: int, steps: int, warmup: int, e2e: bool = False, cpu: bool = False,
                 check: bool = True) -> dict:
    """One batch-GCD form timed on count RSA-2048-shaped moduli (planted shared
    factors), moduli device-resident, CUDA events around `steps` calls; sampled
    rows checked against the oracle.  e2e: the host-buffer entry point (moduli
    in, flags out, copies timed).  cpu: the oracle on the host cores on a
    bounded sample of rows."""
    import torch
    import oracle
    from paper_1407_1465_gb300 import (RSA_GCD_TREE, RsaContext, build, rsa_batch_gcd_ex, rsa_batch_gcd_method,
                                       rsa_batch_gcd_plan)
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    bits = 2048
    L = bits // 32
    rows, pairs = workloads.weak_key_moduli(count, bits)
    ctx = RsaContext(0, mem_budget_bytes=12 << 30)
    m = torch.from_numpy(rows.view(np.int32)).to(dev)
    g = torch.empty_like(m)
    fl = torch.empty(count, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    for _ in range(max(warmup, 3)):
        rsa_batch_gcd_ex(ctx.handle, bits, count, m, g, fl, method, sptr)
    torch.cuda.synchronize()
    clk = ClockSampler(0)
    clk.start()
    time.sleep(0.3)                   # the sampler's start-up off the host thread that launches
    launches0 = ctx.stats()["kernel_launches"]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(steps):
        rsa_batch_gcd_ex(ctx.handle, bits, count, m, g, fl, method, sptr)
    ev[1].record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    launches = (ctx.stats()["kernel_launches"] - launches0) // steps
    ms = ev[0].elapsed_time(ev[1]) / steps
    flags = fl.cpu().numpy()
    if check:
        idx = sorted({0, count - 1, pairs[0][0], pairs[0][1]} | set(range(1, count, max(1, count // 6))))
        og, of = oracle.batch_gcd(rows, rows=idx)
        if not (np.array_equal(g.cpu().numpy().view(np.uint32)[idx], og) and np.array_equal(flags[idx], of)):
            raise RuntimeError("batch gcd differs from the oracle")
        for i, j in pairs:
            if flags[i] < 1 or flags[j] < 1:
                raise RuntimeError("a planted shared factor was not found")
    res = {"count": count, "ms_per_scan": ms, "pairs_per_s": count * (count - 1) / (ms / 1e3),
           "moduli_per_s": count / (ms / 1e3), "gpu_launches": int(launches), "clocks": clocks,
           "planted_pairs": len(pairs),
           "flags": {"coprime": int((flags == 0).sum()), "factor_found": int((flags == 1).sum()),
                     "whole_modulus": int((flags == 2).sum())}}
    if method == RSA_GCD_TREE:
        w = bgcd_tree_work(count, L)
        pk = measured_imad_peak(0)
        achieved = w["montgomery_products"] / (ms / 1e3) / 1e12
        peak = pk["imad_lane_tops"] / 4
        res["form"] = "tree"
        res["roofline"] = {
            "bound": "alu", "achieved": achieved, "peak": peak, "unit": "T Montgomery products/s",
            "frac": achieved / peak, "peak_source": "measured",
            "peak_note": "rsa_imad_probe's independent 32-bit multiply lane rate %.2f T/s over 4 (a Montgomery "
                         "product modulo a 32-bit prime: the 64-bit product, q = lo * p^-1, hi(q p))"
                         % pk["imad_lane_tops"],
            "what": "Montgomery products modulo the three transform primes per second over the whole scan "
                    "(butterflies, pointwise products, recombination); schoolbook and leaf word products "
                    "not counted",
            "work": w, "traffic": None}
    else:
        blk, parts = rsa_batch_gcd_plan(ctx.handle, bits, count)
        issued = bgcd_issued_products(count, L, blk, parts)
        res["form"] = "scan"
        res["block"], res["parts"] = blk, parts
        res["roofline"] = alu_roofline(issued / (ms / 1e3) / 1e12, 0,
                                       "issued word products of the three kernels (word reductions cost L per "
                                       "word, half of a Montgomery multiplication)")
        res["roofline"].update({"traffic": None, "issued_products_per_step": issued})
    res["auto_form"] = "tree" if rsa_batch_gcd_method(ctx.handle, bits, count) == RSA_GCD_TREE else "scan"
    if e2e:
        from paper_1407_1465_gb300 import rsa_batch_gcd_host
        host = torch.from_numpy(rows.view(np.int32)).pin_memory()
        fh = torch.empty(count, dtype=torch.int32).pin_memory()
        rsa_batch_gcd_host(ctx.handle, bits, count, host, None, fh, sptr)
        torch.cuda.synchronize()
        ev2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev2[0].record(stream)
        for _ in range(steps):
            rsa_batch_gcd_host(ctx.handle, bits, count, host, None, fh, sptr)
        ev2[1].record(stream)
        torch.cuda.synchronize()
        ms2 = ev2[0].elapsed_time(ev2[1]) / steps
        res["e2e"] = {"value": count * (count - 1) / (ms2 / 1e3), "unit": "pairs/s", "form": res["auto_form"],
                      "h2d_bytes_per_step": int(rows.nbytes), "d2h_bytes_per_step": int(count * 4)}
    if cpu:
        threads = oracle.default_threads()
        sample = list(range(0, count, max(1, count // (2 * threads))))[: 2 * threads]
        t0 = time.perf_counter()
        oracle.batch_gcd(rows, rows=sample, threads=threads)
        dt = time.perf_counter() - t0
        res["cpu_baseline"] = {"value": len(sample) * (count - 1) / dt, "unit": "pairs/s", "cores": threads,
                               "cpu_model": cpu_model(), "kind": "oracle",
                               "sample": "%d of the %d moduli (each against all %d others), oracle product mod "
                                         "n_i and Euclid, %d POSIX threads" % (len(sample), count, count - 1,
                                                                                threads)}
    ctx.close()
    return res


def run_bgcd(args):
    """Weak-key scan: g_i = gcd(n_i, product of the other moduli) over 131072
    RSA-2048-shaped moduli (16 planted shared factors) by the product and
    remainder trees, one rsa_batch_gcd_ex per step, moduli device-resident;
    reported as modulus pairs/s (count (count - 1) per scan).  --count and
    --gcd-form pick another size or the scan form."""
    from paper_1407_1465_gb300 import RSA_GCD_SCAN, RSA_GCD_TREE
    method = RSA_GCD_SCAN if args.gcd_form == "scan" else RSA_GCD_TREE
    count = args.count or (16384 if method == RSA_GCD_SCAN else 131072)
    r = bgcd_measure(count, method, args.steps, args.warmup, e2e=not args.no_e2e, cpu=not args.no_cpu)
    line = {"metric": "batch GCD modulus pairs/sec (RSA-2048 weak-key scan)", "value": r["pairs_per_s"],
            "unit": "pairs/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_scan"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "gpu_launches": r["gpu_launches"], "moduli_per_s": r["moduli_per_s"],
            "config": {"workload": "%d RSA-2048-shaped moduli (products of random odd 1024-bit halves), %d planted "
                                   "shared factors, one rsa_batch_gcd_ex per step (%s form)"
                                   % (count, r["planted_pairs"], r["form"]),
                       "form": r["form"], "l2": "no flush: the scan's working set (moduli and tree levels) "
                                                "exceeds L2 at this size" if r["form"] == "tree" else
                                                "moduli and block products stay L2-resident (4 MiB each)"},
            "flags": r["flags"], "roofline": r["roofline"], "clocks": r["clocks"], "e2e": r.get("e2e"),
            "cpu_baseline": r.get("cpu_baseline")}
    print(json.dumps(line), flush=True)
    return 0


def ragged_measure(steps: int, warmup: int, autotune: bool = False, loop_steps: int = 0, loop: bool = True) -> dict:
    """The ragged workload (256 keys, 200000 operations, one rsa_modexp_batch
    -- one graph launch -- per step) timed with CUDA events, against a loop of
    one rsa_modexp_key launch per (key, kind) group over the same operations.
    Sampled results are checked against the loop's and against the oracle."""
    import torch
    import oracle
    from paper_1407_1465_gb300 import (RSA_TUNE_RAGGED, RsaContext, build, rsa_modexp_batch, rsa_modexp_key)
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rb = workloads.ragged()
    ctx = RsaContext(0, mem_budget_bytes=16 << 30)
    kids = [ctx.keyload(k.bits, k.n, k.e, k.d, k.p, k.q) for k in rb.keys]
    key_ids = torch.from_numpy(np.array([kids[k] for k in rb.key_ids], dtype=np.int32)).to(dev)
    sels = torch.from_numpy(rb.exp_sel).to(dev)
    offs = torch.from_numpy(rb.offsets.view(np.int64)).to(dev)
    msgs = torch.from_numpy(rb.packed.view(np.int32)).to(dev)
    out = torch.empty_like(msgs)
    status = torch.empty(len(rb.msgs), dtype=torch.int32, device=dev)
    count = len(rb.msgs)
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    # groups for the one-key-per-launch loop, gathered contiguously (untimed)
    groups = {}
    for i, (k, sel) in enumerate(zip(rb.key_ids, rb.exp_sel)):
        groups.setdefault((int(k), int(sel)), []).append(i)
    gbufs = []
    for (k, sel), idx in sorted(groups.items()):
        rows = np.stack([rb.msgs[i] for i in idx])
        t = torch.from_numpy(rows.view(np.int32)).to(dev)
        gbufs.append((kids[k], sel, len(idx), t, torch.empty_like(t), idx))
    tuned_ms = None
    if autotune:
        # the ragged autotuner on this very batch (untimed)
        from paper_1407_1465_gb300 import rsa_autotune_batch
        tuned_ms = rsa_autotune_batch(ctx.handle, count, key_ids, sels, offs, msgs, out)["ms"]
    tuning = ctx.get_tuning(0, RSA_TUNE_RAGGED)
    work = ragged_work(rb, tuning)

    def step_ragged():
        rsa_modexp_batch(ctx.handle, count, key_ids, sels, offs, msgs, out, status, sptr)

    def step_loop():
        for kid, sel, n, t, o, _ in gbufs:
            rsa_modexp_key(ctx.handle, kid, sel, n, t, o, None, sptr)

    res = {"loop": float("nan")}
    legs = [("ragged", step_ragged, steps, warmup)]
    if loop:
        legs.append(("loop", step_loop, loop_steps or steps, min(warmup, 1 if loop_steps else warmup)))
    for name, fn, k_steps, k_warm in legs:
        for _ in range(k_warm):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k_steps)]
        for a, b in ev:
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        res[name] = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
    if ctx.sync() != 0 or not bool((status == 0).all()):
        raise RuntimeError("ragged batch reported errors")
    # the loop's results must equal the ragged batch's, and sampled ones the oracle's
    got = out.cpu().numpy().view(np.uint32)
    for kid, sel, n, t, o, idx in (gbufs[:40] if loop else []):
        oo = o.cpu().numpy().view(np.uint32)
        for j, i in enumerate(idx[:4]):
            off = int(rb.offsets[i])
            if not np.array_equal(got[off:off + oo.shape[1]], oo[j]):
                raise RuntimeError("ragged and per-key results differ")
    for i in np.random.default_rng(3).choice(count, 12, replace=False):
        key, row, off = rb.keys[rb.key_ids[i]], rb.msgs[i], int(rb.offsets[i])
        m = workloads.limbs_to_int(row)
        v = oracle.crt_decrypt(m, key.d, key.p, key.q) if rb.exp_sel[i] == 1 else oracle.modexp(m, key.e, key.n)
        if not np.array_equal(got[off:off + row.size], workloads.int_to_limbs(v, row.size)):
            raise RuntimeError("ragged result differs from the oracle")
    launches0 = ctx.stats()["kernel_launches"]
    step_ragged()
    torch.cuda.synchronize()
    per_step = ctx.stats()["kernel_launches"] - launches0
    ctx.close()
    return {"value": count / (res["ragged"] / 1e3), "unit": "ops/s", "ms_per_step": res["ragged"],
            "kernel_launches_per_step": int(per_step),
            "one_key_per_launch": {"ms_per_step": res["loop"], "value": count / (res["loop"] / 1e3),
                                   "launches": len(gbufs)},
            "speedup_vs_loop": res["loop"] / res["ragged"], "tuning": tuning,
            "autotuned_ms": tuned_ms, "count": count, **work}


def ragged_work(rb, tuning: dict) -> dict:
    """Per-step work of the ragged batch as its kernels issue it.  A CRT bucket
    of one 2048-, 3072- or 4096-bit key with at least tc_min_ops operations
    sends all of them to its tensor-core group (tiles of 128, the last possibly
    partial; 2048 bits at the tuned tensor-core window, 3072 at window 4, 4096
    at window 3); those operations issue the CUDA-core word products and MMA
    FLOPs of the tensor-core path, every other operation the CIOS count
    2L^2 + L per Montgomery product (window 5 for private exponents).  Rows
    past a partial tile's operations compute too and are not counted."""
    from paper_1407_1465_gb300 import rsa_products_per_op
    buckets = {}
    for k, sel in zip(rb.key_ids, rb.exp_sel):
        buckets[(int(k), int(sel))] = buckets.get((int(k), int(sel)), 0) + 1
    tc_on = tuning.get("variant", 0) != 1 and tuning.get("tc_min_ops", 128) > 0
    issued = method_flops = issued_flops = 0.0
    tc_ops = 0
    for (k, sel), c in buckets.items():
        key = rb.keys[k]
        nt = 0
        if tc_on and sel == 1 and key.bits in (2048, 3072, 4096) and c >= tuning.get("tc_min_ops", 128):
            nt = c
        if nt:
            if key.bits == 2048:
                w = tc_work_per_op(2048, tuning.get("window_tc") or 3)
            else:
                w = tc4_work_per_op(4 if key.bits == 3072 else 3, key.bits)
            issued += nt * w[0]
            issued_flops += nt * w[1]
            method_flops += nt * w[2]
            tc_ops += nt
        issued += (c - nt) * rsa_products_per_op(key.bits, sel, key.e, 5)
    return {"products_per_step": issued, "tc_ops": tc_ops, "tc_method_flops_per_step": method_flops,
            "tc_issued_flops_per_step": issued_flops}


def single_key_rate(bits: int, count: int, kind: str = "crt", window: int = 0, steps: int = 3, warmup: int = 2,
                    threads_per_op: int = 0) -> dict:
    """One uniform batch under one seeded key (inputs resident on the device,
    L2 flushed between timed steps), timed with CUDA events; sampled results
    are checked against the oracle.  kind: "crt" (decryption) or "public"
    (encryption with e = 65537)."""
    import torch
    import oracle
    from paper_1407_1465_gb300 import RSA_EXP_PRIVATE_CRT, RSA_EXP_PUBLIC, RsaContext, build, rsa_modexp_key
    build.build()
    dev = torch.device("cuda", 0)
    key, rows = workloads.rsa_single(bits, WORKLOADS["rsa%d" % bits]["count"] if "rsa%d" % bits in WORKLOADS else count)
    rows = rows[:count]
    sel = RSA_EXP_PRIVATE_CRT if kind == "crt" else RSA_EXP_PUBLIC
    ctx = RsaContext(0, mem_budget_bytes=8 << 30)
    try:
        kid = ctx.keyload(bits, key.n, key.e, key.d, key.p, key.q)
        if window or threads_per_op:
            ctx.set_tuning(bits, sel, window=window, threads_per_op=threads_per_op)
        tune = ctx.get_tuning(bits, sel)
        msgs = torch.from_numpy(rows.view(np.int32)).to(dev)
        out = torch.empty_like(msgs)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        stream = torch.cuda.current_stream(dev)
        for _ in range(warmup):
            rsa_modexp_key(ctx.handle, kid, sel, count, msgs, out, None, stream.cuda_stream)
        ms = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            rsa_modexp_key(ctx.handle, kid, sel, count, msgs, out, None, stream.cuda_stream)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        got = out.cpu().numpy().view(np.uint32)
        idx = np.arange(0, count, max(1, count // 6))
        want = (oracle.crt_batch(rows[idx], key.d, key.p, key.q) if kind == "crt"
                else oracle.modexp_batch(rows[idx], key.e, key.n))
        if not np.array_equal(got[idx], want):
            raise RuntimeError("RSA-%d %s results differ from the oracle" % (bits, kind))
        t = statistics.median(ms)
        return {"value": count / (t / 1e3), "ms_per_batch": t, "count": count, "window": tune["window"],
                "threads_per_op": tune["threads_per_op"], "variant": tune["variant"]}
    finally:
        ctx.close()


def toy_rate(steps: int = 20, warmup: int = 3) -> dict:
    """The paper's own example (Sec. 2): n = 17947, e = 131, d = 137 as printed;
    4096 single-limb packets uniform in [0, 2525], encrypted then decrypted per
    step (one launch each); checked against the oracle."""
    import torch
    import oracle
    from paper_1407_1465_gb300 import RSA_EXP_PRIVATE_PLAIN, RSA_EXP_PUBLIC, RsaContext, build, rsa_modexp_key
    build.build()
    dev = torch.device("cuda", 0)
    t = workloads
    ctx = RsaContext(0)
    try:
        kid = ctx.keyload(32, t.TOY_N, t.TOY_E, t.TOY_D, t.TOY_P, t.TOY_Q)
        pk = torch.from_numpy(t.toy_packets(4096).view(np.int32)).to(dev)
        enc, dec = torch.empty_like(pk), torch.empty_like(pk)
        sptr = torch.cuda.current_stream(dev).cuda_stream

        def step():
            rsa_modexp_key(ctx.handle, kid, RSA_EXP_PUBLIC, 4096, pk, enc, None, sptr)
            rsa_modexp_key(ctx.handle, kid, RSA_EXP_PRIVATE_PLAIN, 4096, enc, dec, None, sptr)

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            step()
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        e_np, d_np = enc.cpu().numpy().view(np.uint32), dec.cpu().numpy().view(np.uint32)
        p_np = t.toy_packets(4096)
        if (list(e_np[:64]) != [oracle.modexp(int(m), t.TOY_E, t.TOY_N) for m in p_np[:64]] or
                list(d_np[:64]) != [oracle.modexp(int(c), t.TOY_D, t.TOY_N) for c in e_np[:64]]):
            raise RuntimeError("toy results differ from the oracle")
        return {"value": 8192 / (ms / 1e3), "unit": "ops/s", "ms_per_step": ms, "us_per_launch": ms * 1e3 / 2}
    finally:
        ctx.close()


def tensor_share(r: dict) -> dict:
    """The tensor-core groups' MMA work of a ragged step, as a rate over the
    whole step against the measured bf16 peak (fp16 runs at the same rate)."""
    tpk, tsrc = measured_bf16_tflops()
    sec = r["ms_per_step"] / 1e3
    return {"ops_in_tiles": r["tc_ops"], "method_flops_per_step": r["tc_method_flops_per_step"],
            "issued_flops_per_step": r["tc_issued_flops_per_step"],
            "method_tflops_over_step": r["tc_method_flops_per_step"] / sec / 1e12,
            "peak": tpk, "peak_source": tsrc,
            "frac_over_step": r["tc_method_flops_per_step"] / sec / 1e12 / tpk}


def run_ragged(args):
    """Ragged batch: 256 keys, 200000 operations, one rsa_modexp_batch (one graph
    launch) per step, against a loop of one rsa_modexp_key launch per
    (key, kind) group over the same operations."""
    r = ragged_measure(args.steps, args.warmup, args.autotune, loop=not args.no_loop)
    line = {
        "metric": "ragged-batch ops/sec (256 keys, 200000 ops, one graph launch)",
        "value": r["value"], "unit": "ops/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic", "gpu_launches": r["kernel_launches_per_step"] * args.steps,
        "config": {"workload": "ragged: 256 seeded keys (1024/2048/3072/4096 bits at 0.1/0.5/0.2/0.2), "
                               "Zipf(1.1) counts summing to 200000, 70% CRT decrypt / 30% public",
                   "groups": r["one_key_per_launch"]["launches"]},
        "one_key_per_launch": r["one_key_per_launch"], "speedup_vs_loop": r["speedup_vs_loop"],
        "tuning": r["tuning"], "autotuned": bool(args.autotune),
        "roofline": dict(alu_roofline(r["products_per_step"] / (r["ms_per_step"] / 1e3) / 1e12, 0,
                                      "CUDA-core word products issued per second: the CIOS count 2L^2 + L per "
                                      "Montgomery product (window 5 for private exponents) for operations on the "
                                      "CUDA-core groups, the tensor-core path's own count (squarings H(H+1)/2, "
                                      "other products H^2 per half, plus Garner) for the %d operations in "
                                      "tensor-core tiles" % r["tc_ops"]),
                         products_per_step=r["products_per_step"]),
        "tensor_cores": tensor_share(r),
    }
    print(json.dumps(line), flush=True)
    return 0


def serving_sweep(rates, duration, slots, window_us, key_bits=0, mix_sizes=False):
    """The request loop under Poisson arrivals over the 256 ragged keys (1-64
    messages per request, 70% CRT / 30% public, 2 GiB budget for in-flight
    requests), one pass per rate of `duration` seconds of arrivals (a number,
    or one per rate); returns a result dict per rate."""
    import torch
    from paper_1407_1465_gb300 import (REQUEST_DTYPE, RsaContext, build, rsa_server_clock, rsa_server_drain,
                                       rsa_server_get_stats, rsa_server_start, rsa_server_stop, rsa_server_submit,
                                       rsa_server_submit_many)
    build.build()
    torch.cuda.set_device(0)
    rb_keys = workloads.gen_keys(workloads.ragged_key_specs(256, workloads.DEFAULT_SEED), workloads.DEFAULT_SEED)
    ctx = RsaContext(0, mem_budget_bytes=24 << 30)
    kids = [ctx.keyload(k.bits, k.n, k.e, k.d, k.p, k.q) for k in rb_keys]
    # 64 messages per key shared by the requests; results land in one scratch row set per key
    pools = [workloads.messages_below(k.n, 64, 9, ("pool", i)) for i, k in enumerate(rb_keys)]
    scratch = [np.zeros_like(p) for p in pools]
    results = []
    rsa_server_start(ctx.handle, max_inflight_batches=slots, batch_window_us=window_us, mem_budget_bytes=2 << 30,
                     mix_sizes=mix_sizes)
    for i in range(64):   # warm-up: graphs and workspaces of every slot
        k = i % len(kids)
        rsa_server_submit(ctx.handle, kids[k], 1, pools[k][:8], scratch[k][:8])
    rsa_server_drain(ctx.handle, 600000)
    # key_bits: requests only under the keys of that size (latency of one size class)
    subset = [i for i, k in enumerate(rb_keys) if not key_bits or k.bits == key_bits]
    durations = list(duration) if isinstance(duration, (list, tuple)) else [duration] * len(rates)
    for rate, duration in zip(rates, durations):
        reqs = workloads.poisson_requests(rate, duration, len(kids), workloads.DEFAULT_SEED)
        arr = np.zeros(len(reqs), dtype=REQUEST_DTYPE)
        lead = rsa_server_clock(ctx.handle) + 200_000_000      # arrivals start 200 ms from now
        for j, rq in enumerate(reqs):
            k = subset[rq.key_id % len(subset)]
            arr[j] = (kids[k], rq.exp_sel, rq.count, 0, pools[k].ctypes.data, scratch[k].ctypes.data, 0,
                      lead + int(rq.t_arrive * 1e9))
        rsa_server_get_stats(ctx.handle, reset=True)
        rsa_server_submit_many(ctx.handle, arr)
        rsa_server_drain(ctx.handle, 900000)
        st = rsa_server_get_stats(ctx.handle)
        offered_ops = sum(rq.count for rq in reqs) / duration
        results.append({"offered_req_per_s": rate, "offered_ops_per_s": offered_ops,
                        "requests": st["completed"], "ops": st["ops_completed"],
                        "sustained_ops_per_s": st["ops_completed"] / st["span_s"] if st["span_s"] else None,
                        "p50_ms": st["p50_us"] / 1e3, "p99_ms": st["p99_us"] / 1e3, "max_ms": st["max_us"] / 1e3,
                        "batches": st["batches"], "peak_inflight_bytes": st["peak_bytes"]})
    rsa_server_stop(ctx.handle)
    ctx.close()
    return results


def run_serving(args):
    """Serving loop: Poisson request arrivals over the 256 ragged keys at each
    rate, 1-64 messages per request, 70% CRT / 30% public, a 2 GiB budget for
    in-flight requests; p50/p99 request latency (arrival -> result in the host
    buffer) against sustained operations per second."""
    rates = [float(r) for r in args.rates.split(",")]
    results = serving_sweep(rates, args.duration, args.slots, args.window_us, args.key_bits, args.mix_sizes)
    best = max(results, key=lambda r: r["sustained_ops_per_s"] or 0)
    line = {"metric": "serving: sustained ops/sec and p50/p99 request latency (Poisson arrivals)",
            "value": best["sustained_ops_per_s"], "unit": "ops/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": "256 ragged keys, 1-64 msgs/request, 70%% CRT / 30%% public, 2 GiB budget, "
                                   "%.1f s of arrivals per rate" % args.duration, "rates": rates,
                       "batch_window_us": args.window_us, "slots": args.slots,
                       "key_bits": args.key_bits or "all",
                       "batching": ("every modulus size in one batch" if args.mix_sizes else
                                    "one modulus size per batch (the oldest waiting request picks it)")},
            "sweep": results}
    print(json.dumps(line), flush=True)
    return 0


def aggregate_ranks(ms_per_step: float, units_per_rank: int, world_size: int, dist=None, device=None):
    """Max-over-ranks step time and the whole-job rate (weak scaling: every rank
    processes its own batch, no data exchange).  Returns (ms, units per second)."""
    if world_size > 1:
        import torch
        t = torch.tensor([ms_per_step], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_per_step = float(t.item())
    return ms_per_step, world_size * units_per_rank / (ms_per_step / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args, spec):
    """--impl reference: the CPU oracle itself, timed per step on a bounded sample."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    key, rows = workloads.rsa_single(spec["bits"], WORKLOADS[args.workload]["count"])
    threads = oracle.default_threads()
    public = args.kind == "public"

    def run(sub):
        if public:
            return oracle.modexp_batch(sub, key.e, key.n, threads=threads)
        return oracle.crt_batch(sub, key.d, key.p, key.q, threads=threads)

    probe = min(rows.shape[0], max(threads * 4, 64))
    t0 = time.perf_counter()
    run(rows[:probe])
    rate = probe / (time.perf_counter() - t0)
    # size each step so the whole run stays within a couple of minutes
    per_step = int(max(threads, min(rows.shape[0], rate * 120.0 / max(1, args.steps + args.warmup))))
    for _ in range(args.warmup):
        run(rows[:per_step])
    times = []
    for k in range(args.steps):
        lo = (k * per_step) % max(1, rows.shape[0] - per_step)
        t0 = time.perf_counter()
        run(rows[lo:lo + per_step])
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = per_step / (ms / 1e3)
    unit = "encryptions/s" if public else "decrypts/s"
    metric = ("RSA-%d encryptions/sec (e=65537)" if public else "RSA-%d CRT decrypts/sec") % spec["bits"]
    items = "messages" if public else "ciphertexts"
    routine = "left-to-right binary modexp with e" if public else "CRT routine"
    line = {
        "impl": "reference", "metric": metric, "value": value,
        "unit": unit, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "gpu_launches": 0,
        "config": {"workload": workload_desc(spec["bits"], spec["count"], args.kind),
                   "step": "%d %s per step (bounded sample)" % (per_step, items)},
        "cpu_baseline": {"value": value, "unit": unit, "cores": threads, "cpu_model": cpu_model(), "kind": "oracle",
                         "sample": "%d %s per step, oracle %s, %d POSIX threads"
                                   % (per_step, items, routine, threads)},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="rsa2048", choices=sorted(WORKLOADS) + ["ragged", "serving", "toy", "mr", "bgcd"])
    ap.add_argument("--slots", type=int, default=16, help="serving: batches in flight at once")
    ap.add_argument("--key-bits", type=int, default=0, help="serving: only requests under keys of this size")
    ap.add_argument("--mix-sizes", action="store_true", help="serving: batches take every modulus size")
    ap.add_argument("--mr-bits", type=int, default=1024, choices=[512, 1024, 2048], help="mr: candidate size")
    ap.add_argument("--gcd-form", default="tree", choices=["tree", "scan"], help="bgcd: the form timed")
    ap.add_argument("--e-bits", type=int, default=0,
                    help="--kind public: a seeded random public exponent of this many bits instead of 65537")
    ap.add_argument("--kind", default="crt", choices=["crt", "public"],
                    help="rsa2048/rsa4096: CRT decryption (default) or public-exponent encryption")
    ap.add_argument("--rates", default="1000,2000,5000,10000,20000,50000,100000,200000")
    ap.add_argument("--duration", type=float, default=1.0, help="seconds of arrivals per rate (serving)")
    ap.add_argument("--window-us", type=int, default=200, help="batching window of the serving loop")
    ap.add_argument("--window", type=int, default=0)
    ap.add_argument("--warps", type=int, default=0)
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--variant", type=int, default=0, help="squaring variant: 1 CIOS, 2 separated, 0 auto")
    ap.add_argument("--tpo", type=int, default=0, help="lanes per operation: 1, 2, 4 (0 auto)")
    ap.add_argument("--count", type=int, default=0, help="override the message count (small profiling cases)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-latency", action="store_true", help="skip the serving-latency sweep of the default run")
    ap.add_argument("--no-ragged", action="store_true", help="skip the ragged-batch measurement of the default run")
    ap.add_argument("--no-loop", action="store_true", help="ragged: skip the one-key-per-launch comparison")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the encryption, toy-key and RSA-4096 lines of the default run")
    ap.add_argument("--autotune", action="store_true", help="ragged: run the ragged autotuner on the batch first")
    args = ap.parse_args()
    if args.workload == "ragged":
        return run_ragged(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "toy":
        return run_toy(args)
    if args.workload == "mr":
        return run_mr(args)
    if args.workload == "bgcd":
        return run_bgcd(args)
    spec = dict(WORKLOADS[args.workload])
    if args.count:
        spec["count"] = args.count
    if args.impl == "reference":
        return run_reference(args, spec)
    if args.warmup < 3:
        args.warmup = 3

    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1407_1465_gb300 import (RSA_EXP_PRIVATE_CRT, RSA_EXP_PUBLIC, RsaContext, build, rsa_modexp_key,
                                       rsa_products_per_op)
    build.build()
    kind = RSA_EXP_PRIVATE_CRT if args.kind == "crt" else RSA_EXP_PUBLIC
    metric = ("RSA-%d CRT decrypts/sec" if args.kind == "crt" else "RSA-%d encryptions/sec (e=65537)") % spec["bits"]
    unit = "decrypts/s" if args.kind == "crt" else "encryptions/s"
    if args.kind == "public" and args.e_bits:
        metric = "RSA-%d public-exponent operations/sec (e of %d bits)" % (spec["bits"], args.e_bits)
        unit = "ops/s"

    key, rows = workloads.rsa_single(spec["bits"], WORKLOADS[args.workload]["count"])
    rows = rows[:spec["count"]] if spec["count"] <= rows.shape[0] else \
        workloads.messages_below(key.n, spec["count"], workloads.DEFAULT_SEED, ("single", spec["bits"]))
    count, L = rows.shape
    ctx = RsaContext(local, mem_budget_bytes=16 << 30)
    e_pub = key.e
    if args.kind == "public" and args.e_bits:
        # a long public (non-secret) exponent: the case the sliding-window method serves
        rng = np.random.default_rng(workloads.DEFAULT_SEED + args.e_bits)
        e_pub = (1 << (args.e_bits - 1)) | (int.from_bytes(rng.bytes((args.e_bits + 7) // 8), "little")
                                            % (1 << (args.e_bits - 1))) | 1
        kid = ctx.keyload(spec["bits"], key.n, e_pub)
    else:
        kid = ctx.keyload(spec["bits"], key.n, key.e, key.d, key.p, key.q)
    if args.window or args.warps or args.ctas_per_sm or args.variant or args.tpo:
        ctx.set_tuning(spec["bits"], kind, window=args.window, warps_per_cta=args.warps,
                       ctas_per_sm=args.ctas_per_sm, variant=args.variant, threads_per_op=args.tpo)
    tune = ctx.get_tuning(spec["bits"], kind)
    msgs = torch.from_numpy(rows.view(np.int32)).to(dev)
    out = torch.empty_like(msgs)
    status = torch.empty(count, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 126 MB of L2
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream

    def step():
        rsa_modexp_key(ctx.handle, kid, kind, count, msgs, out, status, sptr)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if not bool((status == 0).all()):
        raise RuntimeError("warm-up produced non-OK statuses")

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    launches0 = ctx.stats()["kernel_launches"]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()                     # L2 flushed between timed steps (not timed)
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    launches = ctx.stats()["kernel_launches"] - launches0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms, value = aggregate_ranks(sum(step_ms) / len(step_ms), count, ws, dist, dev)

    # e2e: the host-buffer entry point, pinned host memory, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        h_in = torch.from_numpy(rows.view(np.int32)).pin_memory()
        h_out = torch.empty_like(h_in).pin_memory()
        from paper_1407_1465_gb300 import rsa_modexp_key_host
        for _ in range(2):
            rsa_modexp_key_host(ctx.handle, kid, kind, count, h_in.data_ptr(), h_out.data_ptr(),
                                None, sptr)
        ek = max(3, args.steps // 4)
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(ek):
            rsa_modexp_key_host(ctx.handle, kid, kind, count, h_in.data_ptr(), h_out.data_ptr(),
                                None, sptr)
        e_s = (time.perf_counter() - t0) / ek
        if ws > 1:
            t = torch.tensor([e_s], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e_s = float(t.item())
        e2e = {"value": ws * count / e_s, "unit": unit, "h2d_bytes_per_step": count * L * 4,
               "d2h_bytes_per_step": count * L * 4, "steps": ek,
               "api": "rsa_modexp_key_host (pinned host buffers)"}
        if not np.array_equal(h_out.numpy().view(np.uint32), out.cpu().numpy().view(np.uint32)):
            raise RuntimeError("e2e output differs from the device-resident run")

    # Roofline of the dominant kernel.  The step is one rsa_modexp_key call; on the
    # tensor-core path its exponentiation kernel is 99.5% of the step (the launch
    # list in profiles/), so the step time stands in for that kernel's duration
    # (a slight understatement of its rate).
    prods = rsa_products_per_op(spec["bits"], kind, e=e_pub, window=tune["window"])
    cios_achieved = prods * count / (ms / 1e3) / 1e12
    pub_tc = args.kind == "public" and pub_tc_taken(spec["bits"], e_pub, count, tune["variant"])
    tc_path = (tune["variant"] == 3 and args.kind == "crt") or pub_tc
    prof = (PROFILED_TRAFFIC.get((args.workload, tune["variant"])) if args.kind == "crt" else
            PROFILED_TRAFFIC.get((args.workload, "public-tc")) if pub_tc and e_pub == 65537 else None)
    prof_valid = bool(prof and prof["window"] in (None, tune["window"])
                      and (tune["threads_per_op"] == 1 or tc_path)   # lanes: CUDA-core kernels only
                      and prof["stamp"] == kernel_stamp(prof["files"]))
    traffic = prof["dram_bytes_per_op"] * count if prof_valid else None
    if tc_path:
        if pub_tc:
            issued, tflops_op, method_flops_op = pub_tc_work_per_op(e_pub)
        else:
            issued, tflops_op, method_flops_op = (tc4_work_per_op(tune["window"], spec["bits"])
                                                  if spec["bits"] in (3072, 4096)
                                                  else tc_work_per_op(spec["bits"], tune["window"]))
        roofline = alu_roofline(issued * count / (ms / 1e3) / 1e12, local,
                                "32x32->64 word products the CUDA cores issue per second (per-message products "
                                "A*B and squarings%s); the Montgomery reductions run on the tensor cores and are "
                                "reported under `tensor`" % ("" if pub_tc else ", the Garner step"))
        roofline["issued_products_per_op"] = issued
        tpk, tsrc = measured_bf16_tflops()
        t_method = method_flops_op * count / (ms / 1e3) / 1e12
        t_issued = tflops_op * count / (ms / 1e3) / 1e12
        roofline["tensor"] = {"achieved": t_method, "peak": tpk, "unit": "TFLOP/s", "frac": t_method / tpk,
                              "flops_per_op": method_flops_op, "peak_source": tsrc + " dense bf16 (fp16 same rate)",
                              "what": "the nonzero byte products of the two Toeplitz products per Montgomery step "
                                      "(mu = T_lo m' mod R, positions of mu m), bias block excluded",
                              "issued_achieved": t_issued, "issued_frac": t_issued / tpk,
                              "issued_flops_per_op": tflops_op}
        roofline["algorithmic"] = {"products_per_op": prods, "achieved": cios_achieved,
                                   "note": "the CIOS count 2H^2 + H per Montgomery product; with the reductions on "
                                           "the tensor cores this rate is not bounded by the IMAD pipe"}
    else:
        roofline = alu_roofline(cios_achieved, local,
                                "32x32->64 word products per second under the CIOS count 2L^2 + L per Montgomery "
                                "product (what these kernels issue)")
        roofline["products_per_op"] = prods
    roofline.update({"traffic": traffic, "traffic_unit": "DRAM bytes per launch",
                     "traffic_source": prof["source"] if traffic else None,
                     "algorithmic_io_bytes": count * L * 4 * 2})
    if prof_valid and "pipes" in prof:
        roofline["limiter"] = dict(prof["pipes"], source=prof["source"])
    if clk.get("sm_mhz"):
        roofline["sm_mhz"] = clk["sm_mhz"]

    line = {
        "metric": metric, "value": value, "unit": unit,
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "gpu_launches": int(launches),
        "config": {"workload": workload_desc(spec["bits"], count, args.kind), "window": tune["window"], "warps_per_cta": tune["warps_per_cta"],
                   "ctas_per_sm": tune["ctas_per_sm"], "variant": tune["variant"],
                   "threads_per_op": tune["threads_per_op"], "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": "dp%d (independent batches per GPU)" % ws},
        "wall_s": wall, "clocks": clk, "roofline": roofline, "e2e": e2e,
    }
    if args.kind == "public" and args.e_bits:
        line["config"]["workload"] = line["config"]["workload"].replace(
            "(e=65537)", "(seeded odd e of %d bits)" % args.e_bits)
    if rank == 0 and ws == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(key, rows, public=(kind == RSA_EXP_PUBLIC), e=e_pub)
    ctx.close()
    if rank == 0 and ws == 1 and not args.no_configs and args.workload == "rsa2048" and args.kind == "crt":
        # the other configurations of the benchmark, short and checked against the oracle:
        # RSA-2048 encryption, the paper's toy key, RSA-4096 CRT over windows 4-6
        enc = single_key_rate(2048, 65536, "public", steps=5, warmup=2)
        line["encrypt"] = dict(enc, unit="encryptions/s", what="RSA-2048 encryption (e = 65537, binary method, "
                               "Fig. 5, the Montgomery reductions mod n on the tensor cores in two rounds of 2^1024): "
                               "the benchmark key's 65536 messages, one rsa_modexp_key per step")
        line["toy"] = dict(toy_rate(), what="the paper's toy key n = 17947, e = 131, d = 137 (Sec. 2): 4096 "
                           "packets in [0, 2525] encrypted then decrypted per step; launch-latency bound")
        # RSA-4096 CRT: the default path (Montgomery reductions on the tensor cores, w = 3) and the
        # CUDA-core four-lane kernel over windows 4-6
        tc4096 = single_key_rate(4096, 16384, "crt", steps=3, warmup=1)
        sweep4096 = {w: single_key_rate(4096, 16384, "crt", window=w, steps=3, warmup=1, threads_per_op=4)
                     for w in (4, 5, 6)}
        best_w = max(sweep4096, key=lambda w: sweep4096[w]["value"])
        iss4, fl4, mfl4 = tc4_work_per_op(tc4096["window"])
        tpk, tsrc = measured_bf16_tflops()
        roof4 = alu_roofline(iss4 * tc4096["value"] / 1e12, local,
                             "32x32->64 word products the CUDA cores issue per second (per-message products and "
                             "squarings, Garner); the Montgomery reductions run on the tensor cores in two rounds")
        roof4["tensor"] = {"achieved": mfl4 * tc4096["value"] / 1e12, "peak": tpk, "unit": "TFLOP/s",
                           "frac": mfl4 * tc4096["value"] / 1e12 / tpk, "peak_source": tsrc,
                           "issued_frac": fl4 * tc4096["value"] / 1e12 / tpk}
        line["rsa4096"] = {
            "what": "RSA-4096 CRT decryption: 1 seeded key (two 2048-bit primes), 16384 ciphertexts; the default "
                    "path (tensor-core Montgomery reductions, variant 3) and the four-lane CUDA-core kernel with "
                    "the window width swept 4-6",
            "value": tc4096["value"], "unit": "decrypts/s", "ms_per_batch": tc4096["ms_per_batch"],
            "window": tc4096["window"], "variant": tc4096["variant"], "roofline": roof4,
            "cuda_core_window_sweep": {str(w): {"value": r["value"], "ms_per_batch": r["ms_per_batch"]}
                                       for w, r in sweep4096.items()},
            "cuda_core_best_window": best_w,
            "cuda_core_roofline": alu_roofline(
                rsa_products_per_op(4096, RSA_EXP_PRIVATE_CRT, e=65537, window=best_w) *
                sweep4096[best_w]["value"] / 1e12, local,
                "word products per second under the CIOS count 2H^2 + H per Montgomery product (what the "
                "four-lane kernel issues)")}
    if rank == 0 and ws == 1 and not args.no_ragged and args.workload == "rsa2048" and args.kind == "crt":
        # the ragged batch (256 keys, 200000 operations, one graph launch) against
        # a loop of one launch per (key, kind) group
        r = ragged_measure(3, 1, loop_steps=1)
        line["ragged"] = {
            "what": "ragged batch: 256 seeded keys (1024/2048/3072/4096 bits at 0.1/0.5/0.2/0.2), Zipf(1.1) counts "
                    "summing to 200000 operations, 70% CRT / 30% public, one rsa_modexp_batch (one CUDA graph) per "
                    "step; sampled results checked against the oracle",
            "value": r["value"], "unit": "ops/s", "ms_per_step": r["ms_per_step"],
            "one_key_per_launch": r["one_key_per_launch"], "speedup_vs_loop": r["speedup_vs_loop"],
            "kernel_launches_per_step": r["kernel_launches_per_step"], "tuning": r["tuning"],
            "issued_cuda_core_tprod_per_s": r["products_per_step"] / (r["ms_per_step"] / 1e3) / 1e12,
            "tensor_cores": tensor_share(r)}
    if rank == 0 and ws == 1 and not args.no_configs and args.workload == "rsa2048" and args.kind == "crt":
        # the weak-key scan (batch GCD): the tree form at 131072 moduli and, at 16384
        # moduli, both forms (where the scan was the library's only one)
        from paper_1407_1465_gb300 import RSA_GCD_SCAN, RSA_GCD_TREE
        tree = bgcd_measure(131072, RSA_GCD_TREE, 3, 3)
        small = {f: bgcd_measure(16384, m, 3, 3, check=(f == "tree")) for f, m in (("tree", RSA_GCD_TREE),
                                                                                 ("scan", RSA_GCD_SCAN))}
        line["bgcd"] = {
            "what": "batch GCD weak-key scan g_i = gcd(n_i, prod_{j != i} n_j) over RSA-2048-shaped moduli with "
                    "16 planted shared factors, one rsa_batch_gcd_ex per step; sampled rows checked against the "
                    "oracle; the product/remainder-tree form at 131072 moduli, both forms at 16384",
            "value": tree["pairs_per_s"], "unit": "pairs/s", "ms_per_scan": tree["ms_per_scan"],
            "moduli": 131072, "moduli_per_s": tree["moduli_per_s"], "gpu_launches": tree["gpu_launches"],
            "roofline": tree["roofline"],
            "at_16384": {f: {"ms_per_scan": r["ms_per_scan"], "pairs_per_s": r["pairs_per_s"]}
                         for f, r in small.items()}}
    if rank == 0 and ws == 1 and not args.no_latency and args.workload == "rsa2048" and args.kind == "crt":
        # the metric's latency half: ragged-batch request latency through the
        # serving loop (256 keys of 1024-4096 bits), offered load swept from
        # 1 k to 200 k requests/s (past saturation)
        rates = [1000.0, 2000.0, 5000.0, 10000.0, 20000.0, 50000.0, 100000.0, 200000.0]
        # a second of arrivals up to 20 k req/s (the knee), half a second past it (the
        # backlog of a saturated rate takes seconds to drain)
        durations = [1.0 if r <= 20000 else 0.5 for r in rates]
        sweep = serving_sweep(rates, durations, args.slots, args.window_us)
        rows = [{"offered_req_per_s": r["offered_req_per_s"], "offered_ops_per_s": r["offered_ops_per_s"],
                 "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"], "sustained_ops_per_s": r["sustained_ops_per_s"],
                 "peak_inflight_bytes": r["peak_inflight_bytes"]} for r in sweep]
        kept = [x for x in rows if x["sustained_ops_per_s"] and x["sustained_ops_per_s"] >= 0.9 * x["offered_ops_per_s"]]
        line["latency"] = {
            "what": "ragged-batch request latency (arrival -> result in the host buffer) through rsa_server_*, "
                    "256 keys of 1024-4096 bits, 1-64 messages per request, 70%% CRT / 30%% public, "
                    "1 s of Poisson arrivals per rate up to 20 k req/s, 0.5 s above, %d slots, 2 GiB admission "
                    "budget" % args.slots,
            "sweep": rows,
            "knee_req_per_s": max(x["offered_req_per_s"] for x in kept) if kept else None,
            "saturated_ops_per_s": max((x["sustained_ops_per_s"] or 0) for x in rows)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
