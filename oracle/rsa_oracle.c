/*
 * rsa_oracle.c -- plain, slow, obviously-correct CPU reference for batched RSA
 * modular exponentiation.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check
 * and the benchmark's CPU-baseline leg call it; the product path never does.
 *
 * What it computes (paper, Sec. 2 and Sec. 3.2-3.3):
 *     C = M^e mod n      (encryption)
 *     M = C^d mod n      (decryption)
 * with 0 <= M < n.  Numbers are little-endian arrays of 32-bit limbs
 * (limb 0 least significant); the paper is silent on limb order.
 *
 * Building blocks, each the textbook definition with no blocking or fusion:
 *   - schoolbook multiplication (every a_i * b_j added into position i+j);
 *   - long division with remainder, Knuth TAOCP Vol. 2, Sec. 4.3.1,
 *     Algorithm D (normalise, estimate each quotient digit from the top two
 *     limbs, multiply-and-subtract, add back when the estimate was one too
 *     large, unnormalise);
 *   - modular multiplication = schoolbook product, then Algorithm D remainder
 *     (paper Fig. 3: (u*v) mod m = ((u mod m)*(v mod m)) mod m);
 *   - exponentiation methods of the paper, in its order and notation:
 *       naive repeated multiplication          (Fig. 4)
 *       right-to-left binary                   (Fig. 5, first algorithm)
 *       left-to-right binary  [the main one]   (Fig. 5, second algorithm)
 *       left-to-right k-ary                    (Fig. 6)
 *       sliding window                         (Fig. 7)
 *   - a CRT decryption reference (m_p = c^(d mod p-1) mod p, m_q likewise,
 *     Garner recombination).  The paper has no CRT; it is used only to check
 *     that CRT and the plain definition agree.
 *
 * No Montgomery or Barrett reduction appears here; the GPU path uses both
 * Montgomery multiplication and CRT, so the two share no arithmetic.
 */
#include "rsa_oracle.h"

#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ------------------------------------------------------------------ */
/* natural numbers: (limbs, length), most significant limb may be 0     */
/* ------------------------------------------------------------------ */

/* number of significant limbs (0 for the value zero) */
static size_t nat_len(const uint32_t *a, size_t n) {
    while (n > 0 && a[n - 1] == 0) n--;
    return n;
}

/* compare a (na limbs) with b (nb limbs): -1, 0, +1 */
static int nat_cmp(const uint32_t *a, size_t na, const uint32_t *b, size_t nb) {
    na = nat_len(a, na);
    nb = nat_len(b, nb);
    if (na != nb) return na < nb ? -1 : 1;
    for (size_t i = na; i-- > 0;) {
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    }
    return 0;
}

/* out[0 .. na+nb) = a * b, schoolbook: out must not alias a or b */
static void nat_mul(const uint32_t *a, size_t na, const uint32_t *b, size_t nb,
                    uint32_t *out) {
    memset(out, 0, (na + nb) * sizeof(uint32_t));
    for (size_t i = 0; i < na; i++) {
        uint64_t carry = 0;
        for (size_t j = 0; j < nb; j++) {
            uint64_t t = (uint64_t)a[i] * b[j] + out[i + j] + carry;
            out[i + j] = (uint32_t)t;
            carry = t >> 32;
        }
        out[i + nb] = (uint32_t)carry;
    }
}

/* number of leading zero bits of a nonzero 32-bit word */
static int clz32(uint32_t x) {
    int k = 0;
    while ((x & 0x80000000u) == 0) {
        x <<= 1;
        k++;
    }
    return k;
}

/*
 * r[0 .. nv) = u mod v, q[0 .. nu-nv+1) = u div v (q may be NULL).
 * Knuth Algorithm D.  Requires v != 0.  u has nu limbs, v has nv limbs.
 */
static void nat_divmod(const uint32_t *u, size_t nu, const uint32_t *v, size_t nv,
                       uint32_t *q, uint32_t *r) {
    size_t n = nat_len(v, nv);
    size_t ulen = nat_len(u, nu);
    if (q) memset(q, 0, (nu >= nv ? nu - nv + 1 : 1) * sizeof(uint32_t));
    memset(r, 0, nv * sizeof(uint32_t));
    if (ulen < n || (ulen == n && nat_cmp(u, ulen, v, n) < 0)) {
        /* u < v: quotient 0, remainder u */
        memcpy(r, u, ulen * sizeof(uint32_t));
        return;
    }
    if (n == 1) {
        /* single-limb divisor: short division from the top */
        uint64_t rem = 0;
        for (size_t i = ulen; i-- > 0;) {
            uint64_t cur = (rem << 32) | u[i];
            if (q) q[i] = (uint32_t)(cur / v[0]);
            rem = cur % v[0];
        }
        r[0] = (uint32_t)rem;
        return;
    }
    size_t m = ulen - n; /* quotient has m+1 digits */

    /* D1: normalise so that the top bit of the divisor is set */
    int s = clz32(v[n - 1]);
    uint32_t *vn = (uint32_t *)malloc(n * sizeof(uint32_t));
    uint32_t *un = (uint32_t *)malloc((ulen + 1) * sizeof(uint32_t));
    for (size_t i = n; i-- > 0;) {
        uint32_t hi = v[i] << s;
        uint32_t lo = (s && i > 0) ? (v[i - 1] >> (32 - s)) : 0;
        vn[i] = hi | lo;
    }
    un[ulen] = s ? (u[ulen - 1] >> (32 - s)) : 0;
    for (size_t i = ulen; i-- > 0;) {
        uint32_t hi = u[i] << s;
        uint32_t lo = (s && i > 0) ? (u[i - 1] >> (32 - s)) : 0;
        un[i] = hi | lo;
    }

    const uint64_t B = (uint64_t)1 << 32;
    /* D2 .. D7: one quotient digit per step, from the top */
    for (size_t jj = m + 1; jj-- > 0;) {
        size_t j = jj;
        /* D3: estimate qhat from the top two limbs of the current remainder */
        uint64_t num = ((uint64_t)un[j + n] << 32) | un[j + n - 1];
        uint64_t qhat = num / vn[n - 1];
        uint64_t rhat = num % vn[n - 1];
        while (qhat >= B || qhat * vn[n - 2] > ((rhat << 32) | un[j + n - 2])) {
            qhat -= 1;
            rhat += vn[n - 1];
            if (rhat >= B) break;
        }
        /* D4: un[j .. j+n] -= qhat * vn */
        uint64_t mul_carry = 0;  /* high part of qhat*vn[i] still to subtract */
        uint32_t borrow = 0;     /* borrow of the subtraction chain */
        for (size_t i = 0; i < n; i++) {
            uint64_t p = qhat * vn[i] + mul_carry;
            mul_carry = p >> 32;
            uint32_t sub = (uint32_t)p;
            uint32_t cur = un[i + j];
            uint64_t diff = (uint64_t)cur - sub - borrow;
            un[i + j] = (uint32_t)diff;
            borrow = (diff >> 63) ? 1u : 0u; /* went below zero */
        }
        {
            uint64_t diff = (uint64_t)un[j + n] - mul_carry - borrow;
            un[j + n] = (uint32_t)diff;
            borrow = (diff >> 63) ? 1u : 0u;
        }
        /* D5/D6: the estimate was one too large -> add the divisor back */
        if (borrow) {
            qhat -= 1;
            uint64_t carry = 0;
            for (size_t i = 0; i < n; i++) {
                uint64_t t = (uint64_t)un[i + j] + vn[i] + carry;
                un[i + j] = (uint32_t)t;
                carry = t >> 32;
            }
            un[j + n] = (uint32_t)((uint64_t)un[j + n] + carry);
        }
        if (q) q[j] = (uint32_t)qhat;
    }
    /* D8: unnormalise the remainder */
    for (size_t i = 0; i < n; i++) {
        uint32_t lo = un[i] >> s;
        uint32_t hi = s ? (un[i + 1] << (32 - s)) : 0;
        r[i] = lo | hi;
    }
    free(vn);
    free(un);
}

/* out[0..nm) = (a * b) mod m; a, b each have nm limbs and are < m */
static void nat_mulmod(const uint32_t *a, const uint32_t *b, const uint32_t *m,
                       size_t nm, uint32_t *out, uint32_t *scratch2n) {
    nat_mul(a, nm, b, nm, scratch2n);
    nat_divmod(scratch2n, 2 * nm, m, nm, NULL, out);
}

/* value of bit i of e (e has ne limbs) */
static int exp_bit(const uint32_t *e, size_t i) {
    return (int)((e[i / 32] >> (i % 32)) & 1u);
}

/* index of the top set bit of e, or -1 if e == 0 */
static long exp_top_bit(const uint32_t *e, size_t ne) {
    size_t n = nat_len(e, ne);
    if (n == 0) return -1;
    return (long)(32 * (n - 1) + (31 - clz32(e[n - 1])));
}

/* A = 1 mod m (0 when m == 1) */
static void set_one_mod(uint32_t *a, const uint32_t *m, size_t nm) {
    memset(a, 0, nm * sizeof(uint32_t));
    uint32_t one = 1;
    if (nat_cmp(&one, 1, m, nm) < 0) a[0] = 1;
}

/* g mod m into gm (nm limbs); g has ng limbs */
static void reduce(const uint32_t *g, size_t ng, const uint32_t *m, size_t nm, uint32_t *gm) {
    nat_divmod(g, ng, m, nm, NULL, gm);
}

/* ------------------------------------------------------------------ */
/* Exponentiation methods (paper Sec. 3.6)                             */
/* ------------------------------------------------------------------ */

/* Fig. 5, left-to-right binary: A = 1; for i = t..0: A = A*A mod m; if e_i, A = A*g mod m */
void oracle_modexp_l2r(const uint32_t *g, size_t ng, const uint32_t *e, size_t ne,
                       const uint32_t *m, size_t nm, uint32_t *out) {
    uint32_t *gm = calloc(nm, 4), *A = calloc(nm, 4), *T = calloc(nm, 4);
    uint32_t *w = calloc(2 * nm, 4);
    reduce(g, ng, m, nm, gm);
    set_one_mod(A, m, nm);
    for (long i = exp_top_bit(e, ne); i >= 0; i--) {
        nat_mulmod(A, A, m, nm, T, w);
        memcpy(A, T, nm * 4);
        if (exp_bit(e, (size_t)i)) {
            nat_mulmod(A, gm, m, nm, T, w);
            memcpy(A, T, nm * 4);
        }
    }
    memcpy(out, A, nm * 4);
    free(gm); free(A); free(T); free(w);
}

/* Fig. 5, right-to-left binary: A = 1, S = g, E = e; while E != 0: if E odd A = A*S;
 * E = floor(E/2); if E != 0, S = S*S. */
void oracle_modexp_r2l(const uint32_t *g, size_t ng, const uint32_t *e, size_t ne,
                       const uint32_t *m, size_t nm, uint32_t *out) {
    uint32_t *A = calloc(nm, 4), *S = calloc(nm, 4), *T = calloc(nm, 4);
    uint32_t *w = calloc(2 * nm, 4);
    uint32_t *E = calloc(ne ? ne : 1, 4);
    memcpy(E, e, ne * 4);
    reduce(g, ng, m, nm, S);
    set_one_mod(A, m, nm);
    while (nat_len(E, ne) != 0) {
        if (E[0] & 1u) {
            nat_mulmod(A, S, m, nm, T, w);
            memcpy(A, T, nm * 4);
            E[0] &= ~1u; /* E = E - 1 */
        }
        /* E = E / 2 */
        for (size_t k = 0; k < ne; k++) {
            uint32_t hi = (k + 1 < ne) ? (E[k + 1] << 31) : 0;
            E[k] = (E[k] >> 1) | hi;
        }
        if (nat_len(E, ne) != 0) {
            nat_mulmod(S, S, m, nm, T, w);
            memcpy(S, T, nm * 4);
        }
    }
    memcpy(out, A, nm * 4);
    free(A); free(S); free(T); free(w); free(E);
}

/* Fig. 4, naive: c = g mod m, then e-1 further multiplications by g (e >= 1).
 * e == 0 gives 1 mod m.  trace (may be NULL) receives c after each step,
 * trace[k-1] = g^k mod m for k = 1..e, nm limbs each. */
void oracle_modexp_naive(const uint32_t *g, size_t ng, uint64_t e, const uint32_t *m,
                         size_t nm, uint32_t *out, uint32_t *trace) {
    uint32_t *gm = calloc(nm, 4), *c = calloc(nm, 4), *T = calloc(nm, 4);
    uint32_t *w = calloc(2 * nm, 4);
    reduce(g, ng, m, nm, gm);
    if (e == 0) {
        set_one_mod(c, m, nm);
    } else {
        memcpy(c, gm, nm * 4);
        if (trace) memcpy(trace, c, nm * 4);
        for (uint64_t k = 2; k <= e; k++) {
            nat_mulmod(c, gm, m, nm, T, w);
            memcpy(c, T, nm * 4);
            if (trace) memcpy(trace + (k - 1) * nm, c, nm * 4);
        }
    }
    memcpy(out, c, nm * 4);
    free(gm); free(c); free(T); free(w);
}

/* Fig. 6, left-to-right k-ary: g_0 = 1, g_i = g_{i-1}*g mod m for i < 2^k; A = 1;
 * for each base-2^k digit e_i from the top: A = A^(2^k) mod m, A = A*g_{e_i} mod m.
 * (Step 1.2 of the figure omits "mod m"; every product here is reduced.) */
void oracle_modexp_kary(const uint32_t *g, size_t ng, const uint32_t *e, size_t ne,
                        unsigned k, const uint32_t *m, size_t nm, uint32_t *out) {
    size_t nent = (size_t)1 << k;
    uint32_t *tab = calloc(nent * nm, 4);
    uint32_t *A = calloc(nm, 4), *T = calloc(nm, 4), *gm = calloc(nm, 4);
    uint32_t *w = calloc(2 * nm, 4);
    reduce(g, ng, m, nm, gm);
    set_one_mod(tab, m, nm);
    for (size_t i = 1; i < nent; i++) nat_mulmod(tab + (i - 1) * nm, gm, m, nm, tab + i * nm, w);
    set_one_mod(A, m, nm);
    long top = exp_top_bit(e, ne);
    size_t ndig = top < 0 ? 0 : ((size_t)top + k) / k; /* digits t..0 */
    for (size_t di = ndig; di-- > 0;) {
        for (unsigned s = 0; s < k; s++) {
            nat_mulmod(A, A, m, nm, T, w);
            memcpy(A, T, nm * 4);
        }
        unsigned digit = 0;
        for (unsigned b = 0; b < k; b++) {
            size_t bit = di * k + b;
            if (bit < 32 * ne && exp_bit(e, bit)) digit |= 1u << b;
        }
        nat_mulmod(A, tab + (size_t)digit * nm, m, nm, T, w);
        memcpy(A, T, nm * 4);
    }
    memcpy(out, A, nm * 4);
    free(tab); free(A); free(T); free(gm); free(w);
}

/* Fig. 7, sliding window (e >= 1): g_1 = g, g_2 = g^2, g_{2i+1} = g_{2i-1}*g_2;
 * scan bits from the top: a 0 bit squares once; otherwise take the longest run
 * e_i..e_l with i-l+1 <= k and e_l = 1, square i-l+1 times and multiply by
 * g_{(e_i..e_l)_2}. */
void oracle_modexp_sliding(const uint32_t *g, size_t ng, const uint32_t *e, size_t ne,
                           unsigned k, const uint32_t *m, size_t nm, uint32_t *out) {
    size_t nent = (size_t)1 << k; /* odd powers g_1, g_3, ..., g_{2^k - 1} live at index i */
    uint32_t *tab = calloc(nent * nm, 4), *g2 = calloc(nm, 4);
    uint32_t *A = calloc(nm, 4), *T = calloc(nm, 4);
    uint32_t *w = calloc(2 * nm, 4);
    reduce(g, ng, m, nm, tab + 1 * nm);
    nat_mulmod(tab + 1 * nm, tab + 1 * nm, m, nm, g2, w);
    for (size_t i = 1; 2 * i + 1 < nent; i++)
        nat_mulmod(tab + (2 * i - 1) * nm, g2, m, nm, tab + (2 * i + 1) * nm, w);
    set_one_mod(A, m, nm);
    long i = exp_top_bit(e, ne);
    while (i >= 0) {
        if (!exp_bit(e, (size_t)i)) {
            nat_mulmod(A, A, m, nm, T, w);
            memcpy(A, T, nm * 4);
            i -= 1;
            continue;
        }
        long l = i - (long)k + 1;
        if (l < 0) l = 0;
        while (!exp_bit(e, (size_t)l)) l++;
        unsigned val = 0;
        for (long b = i; b >= l; b--) val = (val << 1) | (unsigned)exp_bit(e, (size_t)b);
        for (long s = 0; s < i - l + 1; s++) {
            nat_mulmod(A, A, m, nm, T, w);
            memcpy(A, T, nm * 4);
        }
        nat_mulmod(A, tab + (size_t)val * nm, m, nm, T, w);
        memcpy(A, T, nm * 4);
        i = l - 1;
    }
    memcpy(out, A, nm * 4);
    free(tab); free(g2); free(A); free(T); free(w);
}

/* ------------------------------------------------------------------ */
/* CRT decryption reference (not in the paper; checks CRT == plain)    */
/* ------------------------------------------------------------------ */

/*
 * m = c^d mod (p*q) by the Chinese remainder theorem with Garner's formula:
 *   dp = d mod (p-1), dq = d mod (q-1), qinv = q^(p-2) mod p (p prime),
 *   m_p = c^dp mod p, m_q = c^dq mod q,
 *   h = qinv * (m_p - m_q) mod p,  m = m_q + h*q.
 * c and d have 2*nh limbs, p and q have nh limbs, out gets 2*nh limbs.
 * Exponentiation is the left-to-right binary method above.
 */
void oracle_crt_decrypt(const uint32_t *c, const uint32_t *d, const uint32_t *p,
                        const uint32_t *q, size_t nh, uint32_t *out) {
    size_t nn = 2 * nh;
    uint32_t *pm1 = calloc(nh, 4), *qm1 = calloc(nh, 4), *pm2 = calloc(nh, 4);
    uint32_t *dp = calloc(nh, 4), *dq = calloc(nh, 4), *qinv = calloc(nh, 4);
    uint32_t *mp = calloc(nh, 4), *mq = calloc(nh, 4), *mqp = calloc(nh, 4);
    uint32_t *diff = calloc(nh + 1, 4), *h = calloc(nh, 4), *hq = calloc(nn, 4);
    uint32_t *w = calloc(2 * nh, 4);
    /* p-1, q-1, p-2 (p, q odd primes >= 3, so no borrow beyond limb 0 matters) */
    memcpy(pm1, p, nh * 4);
    memcpy(qm1, q, nh * 4);
    memcpy(pm2, p, nh * 4);
    {
        uint64_t b1 = 1, b2 = 1, b3 = 2;
        for (size_t i = 0; i < nh; i++) {
            uint64_t t1 = (uint64_t)pm1[i] - b1; pm1[i] = (uint32_t)t1; b1 = (t1 >> 63) & 1;
            uint64_t t2 = (uint64_t)qm1[i] - b2; qm1[i] = (uint32_t)t2; b2 = (t2 >> 63) & 1;
            uint64_t t3 = (uint64_t)pm2[i] - b3; pm2[i] = (uint32_t)t3; b3 = (t3 >> 63) & 1;
        }
    }
    nat_divmod(d, nn, pm1, nh, NULL, dp);
    nat_divmod(d, nn, qm1, nh, NULL, dq);
    oracle_modexp_l2r(q, nh, pm2, nh, p, nh, qinv);
    oracle_modexp_l2r(c, nn, dp, nh, p, nh, mp);
    oracle_modexp_l2r(c, nn, dq, nh, q, nh, mq);
    /* diff = (m_p - (m_q mod p)) mod p, computed as m_p + p - (m_q mod p) then reduced */
    reduce(mq, nh, p, nh, mqp);
    {
        uint64_t carry = 0;
        for (size_t i = 0; i < nh; i++) {
            uint64_t t = (uint64_t)mp[i] + p[i] + carry;
            diff[i] = (uint32_t)t;
            carry = t >> 32;
        }
        diff[nh] = (uint32_t)carry;
        uint64_t borrow = 0;
        for (size_t i = 0; i <= nh; i++) {
            uint64_t sub = i < nh ? mqp[i] : 0;
            uint64_t t = (uint64_t)diff[i] - sub - borrow;
            diff[i] = (uint32_t)t;
            borrow = (t >> 63) & 1;
        }
        uint32_t *dred = calloc(nh, 4);
        nat_divmod(diff, nh + 1, p, nh, NULL, dred);
        nat_mulmod(qinv, dred, p, nh, h, w);
        free(dred);
    }
    /* m = m_q + h*q */
    nat_mul(h, nh, q, nh, hq);
    {
        uint64_t carry = 0;
        for (size_t i = 0; i < nn; i++) {
            uint64_t t = (uint64_t)hq[i] + (i < nh ? mq[i] : 0) + carry;
            out[i] = (uint32_t)t;
            carry = t >> 32;
        }
    }
    free(pm1); free(qm1); free(pm2); free(dp); free(dq); free(qinv);
    free(mp); free(mq); free(mqp); free(diff); free(h); free(hq); free(w);
}

/* ------------------------------------------------------------------ */
/* Exposed primitives (for the pins) and batched drivers               */
/* ------------------------------------------------------------------ */

void oracle_mul(const uint32_t *a, size_t na, const uint32_t *b, size_t nb, uint32_t *out) {
    nat_mul(a, na, b, nb, out);
}

void oracle_divmod(const uint32_t *u, size_t nu, const uint32_t *v, size_t nv,
                   uint32_t *q, uint32_t *r) {
    nat_divmod(u, nu, v, nv, q, r);
}

typedef struct {
    size_t begin, end;
    const oracle_batch_args *a;
} batch_slice;

/* ------------------------------------------------------------------ */
/* Miller-Rabin probable-prime test (key generation, Fig. 1: "choose two   */
/* large primes"; the paper names no test, this is the standard one)       */
/* ------------------------------------------------------------------ */

/* n odd, n >= 5, nm limbs; bases: nbases numbers of nm limbs, each in [2, n-2].
 * Write n - 1 = d * 2^s with d odd.  Base a passes when a^d = 1 (mod n) or
 * a^(d * 2^r) = n - 1 (mod n) for some 0 <= r < s.  Returns 1 when every base
 * passes (n is a probable prime), 0 when some base witnesses that n is
 * composite, -1 for an even n or n < 5.  Powers by the left-to-right binary
 * method (Fig. 5), squarings by the schoolbook product and Algorithm D. */
int oracle_miller_rabin(const uint32_t *n, size_t nm, const uint32_t *bases, size_t nbases) {
    const uint32_t five = 5;
    if ((n[0] & 1u) == 0 || nat_cmp(n, nm, &five, 1) < 0) return -1;
    uint32_t *nm1 = calloc(nm, 4), *d = calloc(nm, 4), *x = calloc(nm, 4), *t = calloc(nm, 4);
    uint32_t *one = calloc(nm, 4), *w = calloc(2 * nm, 4);
    memcpy(nm1, n, nm * 4);
    nm1[0] -= 1u;                               /* n odd: no borrow */
    one[0] = 1u;
    size_t s = 0;                               /* trailing zero bits of n - 1 */
    while (!exp_bit(nm1, s)) s++;
    for (size_t i = 0; i < nm; i++) {           /* d = (n - 1) >> s */
        const size_t src = i + s / 32, sh = s % 32;
        uint32_t lo = src < nm ? nm1[src] : 0u, hi = src + 1 < nm ? nm1[src + 1] : 0u;
        d[i] = sh ? (lo >> sh) | (hi << (32 - sh)) : lo;
    }
    int result = 1;
    for (size_t b = 0; b < nbases && result == 1; b++) {
        oracle_modexp_l2r(bases + b * nm, nm, d, nm, n, nm, x);
        int pass = nat_cmp(x, nm, one, nm) == 0 || nat_cmp(x, nm, nm1, nm) == 0;
        for (size_t r = 1; r < s && !pass; r++) {
            nat_mulmod(x, x, n, nm, t, w);
            memcpy(x, t, nm * 4);
            if (nat_cmp(x, nm, nm1, nm) == 0) pass = 1;
        }
        if (!pass) result = 0;
    }
    free(nm1); free(d); free(x); free(t); free(one); free(w);
    return result;
}

/* ------------------------------------------------------------------ */
/* Batch GCD (weak-key detection, the introduction's motivation)       */
/* ------------------------------------------------------------------ */

/* a modulus takes part when it is odd and at least 3 */
static int valid_modulus(const uint32_t *n, size_t L) {
    const uint32_t three = 3;
    return (n[0] & 1u) && nat_cmp(n, L, &three, 1) >= 0;
}

/* g (L limbs) = gcd(n_i, product of the other valid moduli), by the
 * definition taken modulo n_i: r = 1, r = r * (n_j mod n_i) mod n_i for every
 * valid j != i (Fig. 3's identity), then Euclid's algorithm,
 * gcd(a, b) = gcd(b, a mod b) until b = 0, with Algorithm D remainders.
 * Returns -1 for an invalid n_i (g = 0), 0 when g = 1, 2 when g = n_i and 1
 * otherwise. */
int oracle_batch_gcd_row(const uint32_t *mods, size_t count, size_t L, size_t i, uint32_t *g) {
    const uint32_t *ni = mods + i * L;
    memset(g, 0, L * 4);
    if (!valid_modulus(ni, L)) return -1;
    uint32_t *r = calloc(L, 4), *x = calloc(L, 4), *t = calloc(L, 4), *w = calloc(2 * L, 4);
    uint32_t *a = calloc(L, 4);
    r[0] = 1u;
    for (size_t j = 0; j < count; j++) {
        const uint32_t *nj = mods + j * L;
        if (j == i || !valid_modulus(nj, L)) continue;
        reduce(nj, L, ni, L, x);
        nat_mulmod(r, x, ni, L, t, w);
        memcpy(r, t, L * 4);
    }
    memcpy(a, ni, L * 4);
    while (nat_len(r, L) != 0) {
        nat_divmod(a, L, r, L, NULL, t);
        memcpy(a, r, L * 4);
        memcpy(r, t, L * 4);
    }
    memcpy(g, a, L * 4);
    const uint32_t one = 1;
    const int flag = nat_cmp(g, L, &one, 1) == 0 ? 0 : nat_cmp(g, L, ni, L) == 0 ? 2 : 1;
    free(r); free(x); free(t); free(w); free(a);
    return flag;
}

static void run_one(const oracle_batch_args *a, size_t i) {
    const uint32_t *msg = a->msgs + i * a->msg_stride;
    uint32_t *out = a->out + i * a->out_stride;
    if (a->kind == ORACLE_KIND_CRT) {
        oracle_crt_decrypt(msg, a->exp, a->p, a->q, a->nh, out);
    } else {
        oracle_modexp_l2r(msg, a->n_limbs, a->exp, a->exp_limbs, a->n, a->n_limbs, out);
    }
}

static void *batch_worker(void *arg) {
    batch_slice *s = (batch_slice *)arg;
    for (size_t i = s->begin; i < s->end; i++) run_one(s->a, i);
    return NULL;
}

int oracle_default_threads(void) {
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

/* Runs count independent operations of one key over nthreads POSIX threads
 * (contiguous slices).  Returns 0 on success. */
int oracle_modexp_batch(const oracle_batch_args *a, size_t count, int nthreads) {
    if (nthreads <= 0) nthreads = oracle_default_threads();
    if ((size_t)nthreads > count) nthreads = count ? (int)count : 1;
    pthread_t *th = calloc((size_t)nthreads, sizeof(pthread_t));
    batch_slice *sl = calloc((size_t)nthreads, sizeof(batch_slice));
    size_t per = count / (size_t)nthreads, extra = count % (size_t)nthreads, pos = 0;
    for (int t = 0; t < nthreads; t++) {
        size_t len = per + ((size_t)t < extra ? 1 : 0);
        sl[t].begin = pos;
        sl[t].end = pos + len;
        sl[t].a = a;
        pos += len;
        pthread_create(&th[t], NULL, batch_worker, &sl[t]);
    }
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    free(th);
    free(sl);
    return 0;
}
