/*
 * rsa_oracle.h -- declarations of the CPU reference (test infrastructure only;
 * see rsa_oracle.c).  All numbers are little-endian arrays of 32-bit limbs.
 * This header belongs to the oracle alone; the CUDA library has its own.
 */
#ifndef RSA_ORACLE_H
#define RSA_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Fig. 5 left-to-right binary: out (nm limbs) = g^e mod m */
void oracle_modexp_l2r(const uint32_t *g, size_t ng, const uint32_t *e, size_t ne,
                       const uint32_t *m, size_t nm, uint32_t *out);
/* Fig. 5 right-to-left binary */
void oracle_modexp_r2l(const uint32_t *g, size_t ng, const uint32_t *e, size_t ne,
                       const uint32_t *m, size_t nm, uint32_t *out);
/* Fig. 4 naive repeated multiplication; trace[k-1] = g^k mod m (may be NULL) */
void oracle_modexp_naive(const uint32_t *g, size_t ng, uint64_t e, const uint32_t *m,
                         size_t nm, uint32_t *out, uint32_t *trace);
/* Fig. 6 left-to-right k-ary */
void oracle_modexp_kary(const uint32_t *g, size_t ng, const uint32_t *e, size_t ne,
                        unsigned k, const uint32_t *m, size_t nm, uint32_t *out);
/* Fig. 7 sliding window */
void oracle_modexp_sliding(const uint32_t *g, size_t ng, const uint32_t *e, size_t ne,
                           unsigned k, const uint32_t *m, size_t nm, uint32_t *out);
/* CRT + Garner reference: c, d have 2*nh limbs; p, q have nh limbs */
void oracle_crt_decrypt(const uint32_t *c, const uint32_t *d, const uint32_t *p,
                        const uint32_t *q, size_t nh, uint32_t *out);

/* schoolbook product, out has na+nb limbs */
void oracle_mul(const uint32_t *a, size_t na, const uint32_t *b, size_t nb, uint32_t *out);
/* Algorithm D: q (nu-nv+1 limbs, may be NULL) and r (nv limbs) */
void oracle_divmod(const uint32_t *u, size_t nu, const uint32_t *v, size_t nv,
                   uint32_t *q, uint32_t *r);

enum { ORACLE_KIND_PLAIN = 0, ORACLE_KIND_CRT = 1 };

/* one key, many messages */
typedef struct {
    int kind;                 /* ORACLE_KIND_PLAIN: msg^exp mod n; ORACLE_KIND_CRT: via p, q */
    const uint32_t *msgs;     /* count rows, msg_stride limbs apart */
    size_t msg_stride;
    uint32_t *out;            /* count rows, out_stride limbs apart */
    size_t out_stride;
    const uint32_t *n;        /* PLAIN: modulus, n_limbs limbs */
    size_t n_limbs;
    const uint32_t *exp;      /* PLAIN: exp_limbs limbs; CRT: d with 2*nh limbs */
    size_t exp_limbs;
    const uint32_t *p, *q;    /* CRT: nh limbs each */
    size_t nh;
} oracle_batch_args;

/* Miller-Rabin: 1 probable prime, 0 composite, -1 invalid n (even or < 5). */
int oracle_miller_rabin(const uint32_t *n, size_t nm, const uint32_t *bases, size_t nbases);

/* Batch GCD, one row: g (L limbs) = gcd(n_i, prod of the other valid moduli);
 * mods holds count rows of L limbs; a modulus is valid when odd and >= 3.
 * Returns -1 invalid n_i (g = 0), 0 g = 1, 1 proper factor, 2 g = n_i. */
int oracle_batch_gcd_row(const uint32_t *mods, size_t count, size_t L, size_t i, uint32_t *g);

int oracle_default_threads(void);
int oracle_modexp_batch(const oracle_batch_args *a, size_t count, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
