"""Planted mistakes: every plausible slip in the oracle must break a pin.

Each case copies oracle/rsa_oracle.c, applies one textual edit (a dropped
carry, a wrong index, a missing correction step, a swapped operation), builds
the mutant with gcc into a temporary directory and runs a battery of checks
against Python's integers and the paper's printed values.  The real oracle
passes the battery (first case); every mutant must fail it.
"""
import os
import random
import shutil
import subprocess
import tempfile

import pytest

import oracle
import workloads
from conftest import read_golden

SRC = os.path.join(os.path.dirname(oracle.__file__), "rsa_oracle.c")

MUTANTS = [
    ("mul drops final carry", "out[i + nb] = (uint32_t)carry;", "out[i + nb] = 0;"),
    ("mul wrong column", "uint64_t t = (uint64_t)a[i] * b[j] + out[i + j] + carry;",
     "uint64_t t = (uint64_t)a[i] * b[j] + out[j] + carry;"),
    ("divmod divisor left unshifted", "uint32_t hi = v[i] << s;", "uint32_t hi = v[i];"),
    ("divmod remainder not unnormalised", "uint32_t lo = un[i] >> s;", "uint32_t lo = un[i];"),
    ("divmod D3 wrong divisor limb", "qhat * vn[n - 2] >", "qhat * vn[n - 1] >"),
    ("divmod no D3 correction",
     "while (qhat >= B || qhat * vn[n - 2] > ((rhat << 32) | un[j + n - 2])) {",
     "while (qhat >= B) {"),
    ("divmod no add-back", "        if (borrow) {\n            qhat -= 1;", "        if (0) {\n            qhat -= 1;"),
    ("divmod top borrow ignored", "uint64_t diff = (uint64_t)un[j + n] - mul_carry - borrow;",
     "uint64_t diff = (uint64_t)un[j + n] - mul_carry;"),
    ("divmod short division remainder",
     "rem = cur % v[0];", "rem = cur / v[0];"),
    ("l2r multiply before square",
     "        nat_mulmod(A, A, m, nm, T, w);\n        memcpy(A, T, nm * 4);\n        if (exp_bit(e, (size_t)i)) {",
     "        if (exp_bit(e, (size_t)i)) {\n            nat_mulmod(A, gm, m, nm, T, w);\n            memcpy(A, T, nm * 4);\n        }\n        nat_mulmod(A, A, m, nm, T, w);\n        memcpy(A, T, nm * 4);\n        if (0) {"),
    ("l2r misses the top bit", "for (long i = exp_top_bit(e, ne); i >= 0; i--) {",
     "for (long i = exp_top_bit(e, ne) - 1; i >= 0; i--) {"),
    ("exp_bit wrong shift", "return (int)((e[i / 32] >> (i % 32)) & 1u);",
     "return (int)((e[i / 32] >> (31 - i % 32)) & 1u);"),
    ("r2l halves wrong", "uint32_t hi = (k + 1 < ne) ? (E[k + 1] << 31) : 0;",
     "uint32_t hi = 0;"),
    ("kary digit bit order", "if (bit < 32 * ne && exp_bit(e, bit)) digit |= 1u << b;",
     "if (bit < 32 * ne && exp_bit(e, bit)) digit |= 1u << (k - 1 - b);"),
    ("kary one squaring short", "for (unsigned s = 0; s < k; s++) {", "for (unsigned s = 1; s < k; s++) {"),
    ("sliding window start off by one", "long l = i - (long)k + 1;", "long l = i - (long)k;"),
    ("crt swaps dp and dq", "oracle_modexp_l2r(c, nn, dp, nh, p, nh, mp);",
     "oracle_modexp_l2r(c, nn, dq, nh, p, nh, mp);"),
    ("crt garner sign", "uint64_t t = (uint64_t)diff[i] - sub - borrow;",
     "uint64_t t = (uint64_t)diff[i] + sub - borrow;"),
    ("crt drops m_q", "uint64_t t = (uint64_t)hq[i] + (i < nh ? mq[i] : 0) + carry;",
     "uint64_t t = (uint64_t)hq[i] + carry;"),
    ("naive one multiplication short", "for (uint64_t k = 2; k <= e; k++) {",
     "for (uint64_t k = 3; k <= e; k++) {"),
    ("mr skips the a^d = n-1 check", "int pass = nat_cmp(x, nm, one, nm) == 0 || nat_cmp(x, nm, nm1, nm) == 0;",
     "int pass = nat_cmp(x, nm, one, nm) == 0;"),
    ("mr one squaring short", "for (size_t r = 1; r < s && !pass; r++) {",
     "for (size_t r = 2; r < s && !pass; r++) {"),
    ("mr accepts a square root of 1", "            if (nat_cmp(x, nm, nm1, nm) == 0) pass = 1;",
     "            if (nat_cmp(x, nm, nm1, nm) == 0 || nat_cmp(x, nm, one, nm) == 0) pass = 1;"),
    ("mr exponent not halved enough", "while (!exp_bit(nm1, s)) s++;", "while (!exp_bit(nm1, s + 1)) s++;"),
    ("bgcd multiplies n_i into its own product", "if (j == i || !valid_modulus(nj, L)) continue;",
     "if (!valid_modulus(nj, L)) continue;"),
    ("bgcd keeps invalid moduli", "if (j == i || !valid_modulus(nj, L)) continue;", "if (j == i) continue;"),
    ("bgcd rejects the modulus 3", "return (n[0] & 1u) && nat_cmp(n, L, &three, 1) >= 0;",
     "return (n[0] & 1u) && nat_cmp(n, L, &three, 1) > 0;"),
    ("bgcd returns the last remainder", "    memcpy(g, a, L * 4);\n    const uint32_t one", "    memcpy(g, r, L * 4);\n    const uint32_t one"),
    ("bgcd euclid updates in the wrong order", "        memcpy(a, r, L * 4);\n        memcpy(r, t, L * 4);\n",
     "        memcpy(r, t, L * 4);\n        memcpy(a, r, L * 4);\n"),
    ("bgcd product forgets earlier factors", "        nat_mulmod(r, x, ni, L, t, w);\n        memcpy(r, t, L * 4);\n",
     "        memcpy(r, x, L * 4);\n"),
    ("bgcd flags swapped", "nat_cmp(g, L, ni, L) == 0 ? 2 : 1;", "nat_cmp(g, L, ni, L) == 0 ? 1 : 2;"),
]


def battery(lib) -> list:
    """Returns the list of failed checks (empty = passes)."""
    fails = []
    g = read_golden("fig4_naive_trace.txt")
    try:
        if oracle.naive_trace(g["g"], g["e"], g["m"], lib=lib) != g["trace"]:
            fails.append("fig4 trace")
    except Exception as exc:  # a mutant may crash a conversion
        fails.append("fig4 trace raised %r" % exc)
    for method in ("l2r", "r2l"):
        if oracle.modexp(g["g"], g["e"], g["m"], method, lib=lib) != 445:
            fails.append("fig4 " + method)
    for k in (2, 3, 4):
        if oracle.modexp(g["g"], g["e"], g["m"], "kary", k=k, lib=lib) != 445:
            fails.append("fig4 kary%d" % k)
        if oracle.modexp(g["g"], g["e"], g["m"], "sliding", k=k, lib=lib) != 445:
            fails.append("fig4 sliding%d" % k)
    rng = random.Random(99)
    special = [0, 1, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFE, 0xFFFFFFFF]
    for _ in range(700):
        nu, nv = rng.randrange(1, 7), rng.randrange(1, 5)
        if rng.random() < 0.5:
            u = sum(rng.choice(special) << (32 * i) for i in range(nu))
            v = sum(rng.choice(special) << (32 * i) for i in range(nv))
        else:
            u, v = rng.getrandbits(32 * nu), rng.getrandbits(32 * nv)
        if v == 0:
            continue
        if oracle.mul(u, v, lib=lib) != u * v:
            fails.append("mul")
            break
        if oracle.divmod_(u, v, lib=lib) != divmod(u, v):
            fails.append("divmod")
            break
    for _ in range(1200):  # three-limb divisors whose low limb decides the quotient digit
        vtop = 0x80000000 | rng.getrandbits(rng.choice([1, 8, 31]))
        v = (vtop << 64) | (rng.choice([0, 0xFFFFFFFF, rng.getrandbits(32)]) << 32) | rng.getrandbits(32)
        q, r = rng.getrandbits(32), rng.randrange(v)
        if oracle.divmod_(q * v + r, v, lib=lib) != (q, r):
            fails.append("divmod 3-limb")
            break
    for _ in range(60):
        nl = rng.choice([1, 2, 5])
        m = rng.getrandbits(32 * nl) | 1 | (1 << (32 * nl - 1))
        gg = rng.randrange(m)
        e = rng.getrandbits(rng.choice([5, 33, 70]))
        ref = pow(gg, e, m)
        for method in ("l2r", "r2l"):
            if oracle.modexp(gg, e, m, method, lib=lib) != ref:
                fails.append(method)
        for k in (1, 3, 5):
            if oracle.modexp(gg, e, m, "kary", k=k, lib=lib) != ref:
                fails.append("kary")
            if e and oracle.modexp(gg, e, m, "sliding", k=k, lib=lib) != ref:
                fails.append("sliding")
    # Miller-Rabin: trial division below 3000 (bases 2, 3, 5, 7 are exact there),
    # the strong pseudoprime 2047 (passes base 2 only), Carmichael numbers
    try:
        for n in range(5, 3000, 2):
            bases = [b for b in (2, 3, 5, 7) if b <= n - 2]
            isp = all(n % f for f in range(3, int(n ** 0.5) + 1, 2))
            if oracle.miller_rabin(n, bases, lib=lib) != int(isp):
                fails.append("mr trial division")
                break
        if oracle.miller_rabin(2047, [2], lib=lib) != 1 or oracle.miller_rabin(2047, [3], lib=lib) != 0:
            fails.append("mr 2047")
        if any(oracle.miller_rabin(n, [2], lib=lib) != 0 for n in (561, 1105, 1729, 8911)):
            fails.append("mr carmichael")
        if oracle.miller_rabin((1 << 127) - 1, [3, 5, 7], lib=lib) != 1:
            fails.append("mr mersenne")
    except Exception as exc:
        fails.append("mr raised %r" % exc)
    # batch GCD: constructed sharing and brute force on tiny moduli.  Euclid's
    # loop ends only with a correct remainder, so these run only when division
    # passed (a broken division is already caught above)
    try:
        if any(f.startswith("divmod") for f in fails):
            raise StopIteration
        import bgcd_cases
        values, _, want, flags = bgcd_cases.constructed_case()
        g, f = oracle.batch_gcd(workloads.ints_to_rows(values, 8), threads=2, lib=lib)
        if workloads.rows_to_ints(g) != want or f.tolist() != flags:
            fails.append("bgcd constructed")
        for mods in bgcd_cases.brute_cases(trials=15):
            want, flags = bgcd_cases.brute_case(mods)
            g, f = oracle.batch_gcd(workloads.ints_to_rows(mods, 1), threads=1, lib=lib)
            if workloads.rows_to_ints(g) != want or f.tolist() != flags:
                fails.append("bgcd brute force")
                break
    except StopIteration:
        pass
    except Exception as exc:
        fails.append("bgcd raised %r" % exc)
    key = workloads.gen_key(256, seed=5, index=1, mr_rounds=10)
    for mm in workloads.rows_to_ints(workloads.messages_below(key.n, 8, 5, "mut")):
        c = pow(mm, key.e, key.n)
        if oracle.crt_decrypt(c, key.d, key.p, key.q, lib=lib) != mm:
            fails.append("crt")
            break
    return sorted(set(fails))


def _build_variant(tmp, text, name):
    src = os.path.join(tmp, name + ".c")
    with open(src, "w") as f:
        f.write(text)
    shutil.copy(os.path.join(os.path.dirname(SRC), "rsa_oracle.h"), tmp)
    out = os.path.join(tmp, "lib" + name + ".so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread", "-I", tmp, src, "-o", out],
                   check=True, capture_output=True)
    return oracle.load(out)


@pytest.fixture(scope="module")
def tmpdir_mod():
    d = tempfile.mkdtemp(prefix="oracle_mut_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


def test_real_oracle_passes_battery(tmpdir_mod):
    with open(SRC) as f:
        text = f.read()
    lib = _build_variant(tmpdir_mod, text, "orig")
    assert battery(lib) == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmpdir_mod, name, old, new):
    with open(SRC) as f:
        text = f.read()
    assert text.count(old) == 1, "mutation anchor not unique/present: %s" % name
    lib = _build_variant(tmpdir_mod, text.replace(old, new), "m%d" % (abs(hash(name)) % 10**8))
    assert battery(lib) != [], "planted mistake not detected: %s" % name
