"""The benchmark's roofline numerators, counted step by step.

bench.py reports achieved word products per second from closed forms; here the
same counts are re-derived by walking the kernels' loops (blocks, super-blocks,
lanes, tree levels, window steps), so a slip in a closed form shows up.
"""
import numpy as np
import pytest

import bench


def _bgcd_walk(count, L, blk, parts):
    """Word products of one batch-GCD scan, loop by loop (count a multiple of 32)."""
    mm = 2 * L * L + L
    nblk = -(-count // blk)
    total = 0
    # block products: a product tree per block; level l multiplies blk / 2^l pairs of
    # 2^(l-1) L-word numbers, each split over 2^(l-1) chunks of L words (s words x L words)
    for _c in range(nblk):
        lev, s = 1, L
        while (1 << lev) <= blk:
            lanes = blk // 2
            total += lanes * s * L
            lev += 1
            s *= 2
    nsb = -(-count // 32)
    for i in range(count):
        w = i // 32
        for sb in range(nsb):
            if sb == w:
                members = min(count, 32 * sb + 32) - 32 * sb
                total += (members - 1) * mm                       # CIOS per own modulus, j != i
            else:
                for c in range(sb * (32 // blk), min(nblk, (sb + 1) * (32 // blk))):
                    members = min(count, (c + 1) * blk) - c * blk
                    total += members * L * L                      # word reductions: L per word
                    total += mm                                   # into the running product
        total += (parts - 1) * mm                                 # the combine tree, per lane
    return total


@pytest.mark.parametrize("count,L,blk,parts", [(32, 16, 8, 1), (96, 16, 16, 3), (256, 32, 32, 5),
                                               (640, 64, 16, 10)])
def test_bgcd_issued_products_matches_loop_count(count, L, blk, parts):
    assert bench.bgcd_issued_products(count, L, blk, parts) == _bgcd_walk(count, L, blk, parts)


def _mr_walk(cands, rounds, L, W=4):
    """Word products of one Miller-Rabin launch, per lane, from the kernel's loops."""
    mm = 2 * L * L + L
    count = cands.shape[0]
    warps = -(-count // 32)
    nwin = -(-(32 * L) // W)
    total = 0
    for wi in range(warps):
        rows = [min(wi * 32 + ln, count - 1) for ln in range(32)]   # dead lanes repeat the last row
        ss = []
        for r in rows:
            n = int.from_bytes(cands[r].astype("<u4").tobytes(), "little")
            m = n - 1
            ss.append((m & -m).bit_length() - 1)
        s_max = max(ss)
        for _ in range(32):
            total += {16: 3, 32: 4, 64: 5}[L] * mm              # R^2 by squarings
            for _r in range(rounds):
                total += mm                                      # into Montgomery form
                total += (2 ** W - 2) * mm                       # table entries 2 .. 2^W - 1
                total += (nwin - 1) * (W + 1) * mm               # W squarings + 1 product per window
                total += max(s_max - 1, 0) * mm                  # the n - 1 search
    return total


@pytest.mark.parametrize("L", [16, 32])
def test_mr_issued_products_matches_loop_count(L):
    rng = np.random.default_rng(L)
    cands = rng.integers(0, 1 << 32, size=(77, L), dtype=np.uint64).astype(np.uint32)
    cands[:, 0] |= 1
    cands[5, 0] = 0x00000001                                     # n - 1 with many trailing zeros
    cands[5, 1] = 0x80000000
    assert bench.mr_issued_products(cands, 1, L=L) == _mr_walk(cands, 1, L)


def _tc_walk(bits, W):
    """CUDA-core word products and tensor FLOPs of one RSA-2048 CRT decryption on
    the tensor-core path, replaying the kernel's step loop: per half, steps 0-1
    bring c_lo, c_hi into Montgomery form, steps 2 .. 2^W - 1 build the table
    (step 2 squares), then each window is W squarings and one product by the
    selected entry; the q half adds one product leaving Montgomery form; then
    Garner (two CIOS products and one H x H product)."""
    H = bits // 64
    D = 4 * H                                                # byte digits of a prime
    # the method's byte products per step, by enumerating digit pairs: mu's
    # columns 0..D-1 of T_lo * m' (digit k of T_lo, digit n-k of m'), and the
    # positions D-4 .. 2D-5 of mu * m that MMA 2 returns (digit i of mu, j-i of m)
    pairs1 = sum(1 for n in range(D) for k in range(D) if 0 <= n - k < D)
    pairs2 = sum(1 for j in range(D - 4, 2 * D - 4) for i in range(D) if 0 <= j - i < D)
    nwin = -(-(32 * H) // W)
    ntab = 1 << W
    nexp = (nwin - 1) * (W + 1)
    prods = flops = method = 0
    for pi in (0, 1):
        s = 0
        for st in range(ntab + nexp + (1 if pi == 0 else 0)):
            sq = False
            if 2 <= st < ntab:
                sq = st == 2
            elif ntab <= st < ntab + nexp:
                if s < W:
                    sq, s = True, s + 1
                else:
                    s = 0
            prods += H * (H + 1) // 2 if sq else H * H
            flops += 2 * (2 * 128 * (9 * 16))                # two MMAs, N = 128, K = 144, per row
            method += 2 * (pairs1 + pairs2)
    prods += 2 * (2 * H * H + H) + H * H
    return prods, flops, method


@pytest.mark.parametrize("W", [3, 4])
def test_tc_work_per_op_matches_the_step_loop(W):
    assert bench.tc_work_per_op(2048, W) == _tc_walk(2048, W)


def test_measured_roofline_fraction_uses_the_probe_figure(monkeypatch):
    """alu_roofline divides by the measured carry-chain rate, not the unit-count figure."""
    monkeypatch.setitem(bench._PEAKS, 7, {"chain_tprod": 6.5, "imad_lane_tops": 19.5, "sm_count": 152,
                                          "derived_tprod": bench.derived_peak_tprod(152, 2070.0)})
    r = bench.alu_roofline(3.25, 7, "test")
    assert r["peak"] == 6.5 and r["frac"] == 0.5 and r["peak_source"] == "measured"
    assert abs(bench.derived_peak_tprod(152, 2070.0) - 10.06848) < 1e-9


def _tc4_walk(W, bits):
    """The RSA-3072/4096 tensor-core path's work per decryption, replaying its
    step loop (as _tc_walk: squarings issue each cross product once) with two
    reduction rounds per step; the method's MMA work by enumerating the digit
    pairs of mu = (T mod r) m' and of positions D-4 .. 3D-5 of mu * m (m: 2D digits)."""
    H = bits // 64
    D = 2 * H
    pairs1 = sum(1 for n in range(D) for k in range(D) if 0 <= n - k < D)
    pairs2 = sum(1 for j in range(D - 4, 3 * D - 4) for i in range(D) if 0 <= j - i < 2 * D)
    nwin = -(-(32 * H) // W)
    ntab, nexp = 1 << W, (nwin - 1) * (W + 1)
    prods = flops = method = 0
    for pi in (0, 1):
        s = 0
        for st in range(ntab + nexp + (1 if pi == 0 else 0)):
            sq = False
            if 2 <= st < ntab:
                sq = st == 2
            elif ntab <= st < ntab + nexp:
                if s < W:
                    sq, s = True, s + 1
                else:
                    s = 0
            prods += H * (H + 1) // 2 if sq else H * H
            # per round: MMA 1 (N = D) and MMA 2 (N = 2D), D/16 + 1 K-steps of 16 for each of 128 rows
            flops += 2 * (2 * D * (16 * (D // 16 + 1)) + 2 * 2 * D * (16 * (D // 16 + 1)))
            method += 2 * 2 * (pairs1 + pairs2)
    prods += 2 * (2 * H * H + H) + H * H
    return prods, flops, method


@pytest.mark.parametrize("bits", [3072, 4096])
@pytest.mark.parametrize("W", [3, 4])
def test_tc4_work_per_op_matches_the_step_loop(W, bits):
    assert bench.tc4_work_per_op(W, bits) == _tc4_walk(W, bits)


def test_ragged_work_routes_crt_buckets_to_the_tensor_core_count(monkeypatch):
    """2048/3072/4096-bit CRT buckets at or above the threshold count the
    tensor-core path's work for all their operations; public operations,
    1024-bit keys, buckets below the threshold and everything with the groups
    off (variant 1) count the CIOS products."""
    import types
    import paper_1407_1465_gb300 as pkg
    monkeypatch.setattr(pkg, "rsa_products_per_op", lambda bits, sel, e=65537, window=5: 1000.0 * bits + sel)
    keys = [types.SimpleNamespace(bits=b, e=65537) for b in (1024, 2048, 2048, 3072, 4096)]
    # (key, kind, count): 1024 CRT 300; 2048 CRT 300 (2 tiles + 44); 2048 CRT 100 (below); 3072 CRT 129; 4096 CRT
    # 256 and public 200
    plan = [(0, 1, 300), (1, 1, 300), (2, 1, 100), (3, 1, 129), (4, 1, 256), (4, 0, 200)]
    key_ids = np.concatenate([np.full(c, k) for k, _, c in plan])
    sels = np.concatenate([np.full(c, s) for _, s, c in plan])
    rb = types.SimpleNamespace(keys=keys, key_ids=key_ids, exp_sel=sels)
    cios = sum(c * (1000.0 * keys[k].bits + s) for k, s, c in plan)
    for off in ({"variant": 1, "tc_min_ops": 128, "window_tc": 3}, {"variant": 0, "tc_min_ops": 0, "window_tc": 3}):
        w = bench.ragged_work(rb, off)
        assert w["tc_ops"] == 0 and w["products_per_step"] == cios and w["tc_method_flops_per_step"] == 0
    w = bench.ragged_work(rb, {"variant": 0, "tc_min_ops": 128, "window_tc": 4})
    t2, t3, t4 = bench.tc_work_per_op(2048, 4), bench.tc4_work_per_op(4, 3072), bench.tc4_work_per_op(3, 4096)
    assert w["tc_ops"] == 300 + 129 + 256
    want = cios - 300 * (2048e3 + 1) - 129 * (3072e3 + 1) - 256 * (4096e3 + 1) + 300 * t2[0] + 129 * t3[0] + 256 * t4[0]
    assert w["products_per_step"] == want
    assert w["tc_method_flops_per_step"] == 300 * t2[2] + 129 * t3[2] + 256 * t4[2]
    assert w["tc_issued_flops_per_step"] == 300 * t2[1] + 129 * t3[1] + 256 * t4[1]
    # no bucket reaches a 512-operation threshold
    assert bench.ragged_work(rb, {"variant": 0, "tc_min_ops": 512, "window_tc": 3})["tc_ops"] == 0


def _pub_tc_walk(e, H=64):
    """The RSA-2048 public exponent on the tensor cores, replaying the
    kernel's steps: x R (a general product), for each bit of e below the top
    one a squaring and, for a 1 bit, a product by x R, then the product by 1;
    per step two reduction rounds of MMA 1 (N = D) and MMA 2 (N = 2D) over
    D/16 + 1 K-steps, the method's part by enumerating digit pairs."""
    D = 2 * H
    pairs1 = sum(1 for n in range(D) for k in range(D) if 0 <= n - k < D)
    pairs2 = sum(1 for j in range(D - 4, 3 * D - 4) for i in range(D) if 0 <= j - i < 2 * D)
    steps = [False]                                  # x R
    for bit in range(e.bit_length() - 2, -1, -1):
        steps.append(True)
        if (e >> bit) & 1:
            steps.append(False)
    steps.append(False)                              # leave Montgomery form
    prods = sum(H * (H + 1) // 2 if sq else H * H for sq in steps)
    flops = len(steps) * 2 * (2 * D * (16 * (D // 16 + 1)) + 2 * 2 * D * (16 * (D // 16 + 1)))
    method = len(steps) * 2 * 2 * (pairs1 + pairs2)
    return prods, flops, method


@pytest.mark.parametrize("e", [3, 65537, (1 << 100) + 12345, (1 << 2047) + 3])
def test_pub_tc_work_per_op_matches_the_step_loop(e):
    assert bench.pub_tc_work_per_op(e) == _pub_tc_walk(e)


def test_pub_tc_taken_mirrors_the_library_rule():
    assert bench.pub_tc_taken(2048, 65537, 4096, 0) and not bench.pub_tc_taken(2048, 65537, 4095, 0)
    assert bench.pub_tc_taken(2048, (1 << 200) + 1, 10, 3) and not bench.pub_tc_taken(2048, (1 << 200) + 1, 65536, 0)
    assert not bench.pub_tc_taken(4096, 65537, 65536, 0) and not bench.pub_tc_taken(2048, 65537, 65536, 1)


def test_bgcd_tree_work_small_cases_by_hand():
    """Two 2048-bit moduli: one 64 x 64-word schoolbook product (the root), the
    leaf reduction of the root's 257 words modulo each n_i^2 (128 words), n_i^2
    and the exact division (64^2 each).  Eight 512-bit moduli: the product tree's
    4 + 2 + 1 schoolbook products of 16, 32, 64 words; no transform anywhere."""
    w = bench.bgcd_tree_work(2, 64)
    assert (w["K"], w["T"], w["t0"]) == (2, 1, 1)
    assert w["school_products"] == 64 * 64 and w["montgomery_products"] == 0 and w["products"] == 1
    assert w["leaf_products"] == 2 * (257 * 128 + 2 * 64 * 64)
    w = bench.bgcd_tree_work(8, 16)
    assert (w["T"], w["t0"]) == (3, 3)
    assert w["school_products"] == 4 * 16 * 16 + 2 * 32 * 32 + 64 * 64 and w["montgomery_products"] == 0
    assert w["leaf_products"] == 8 * ((2 * 128 + 1) * 32 + 2 * 16 * 16)


def test_bgcd_tree_work_transform_count():
    """131072 2048-bit moduli: the remainder tree's levels from t0 = 4 each run
    two transform products (q and the quotient step) of 4 s_t words; every
    transform product is counted once per prime and transform."""
    w = bench.bgcd_tree_work(131072, 64)
    assert (w["K"], w["T"], w["t0"]) == (131072, 17, 4)
    assert w["transforms"] % 3 == 0 and w["montgomery_products"] > 1e11
