/*
 * oracle/ring.c -- exact arithmetic in Z_q and in Z_q[X]/(X^n + 1) for the CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is part of the independent CPU oracle that the
 * GPU library is checked against; nothing in the product links it.  It shares no code,
 * header or table with the CUDA sources.
 *
 * Every routine is the plain definition: products are formed in 128-bit integers and
 * reduced with the C `%` operator.  The BFV scheme the paper uses (Sec. 2.1) works in the
 * ring R_q = Z_q[X]/(X^n + 1); a product there is the negacyclic convolution
 *     c_k = sum_{i+j=k} a_i b_j  -  sum_{i+j=k+n} a_i b_j   (mod q),
 * written out in orc_negacyclic_schoolbook.  orc_negacyclic_mul computes the same product
 * through the evaluation map a -> (a(psi^(2k+1)))_k at the odd powers of a primitive 2n-th
 * root psi (a textbook radix-2 FFT, natural order), which the oracle's tests pin against
 * the schoolbook definition.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) {
    return (uint64_t)(((u128)a * (u128)b) % (u128)q);
}

static uint64_t addmod(uint64_t a, uint64_t b, uint64_t q) {
    return (uint64_t)(((u128)a + (u128)b) % (u128)q);
}

static uint64_t submod(uint64_t a, uint64_t b, uint64_t q) {
    return (uint64_t)(((u128)a + (u128)q - (u128)(b % q)) % (u128)q);
}

uint64_t orc_powmod(uint64_t a, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q, x = a % q;
    while (e) {
        if (e & 1) r = mulmod(r, x, q);
        x = mulmod(x, x, q);
        e >>= 1;
    }
    return r;
}

/* ---- element-wise vectors (all outputs in [0, q)) ---- */

void orc_vec_add(const uint64_t* a, const uint64_t* b, uint64_t* out, int64_t n, uint64_t q) {
    for (int64_t i = 0; i < n; ++i) out[i] = addmod(a[i], b[i], q);
}

void orc_vec_sub(const uint64_t* a, const uint64_t* b, uint64_t* out, int64_t n, uint64_t q) {
    for (int64_t i = 0; i < n; ++i) out[i] = submod(a[i] % q, b[i], q);
}

void orc_vec_mul(const uint64_t* a, const uint64_t* b, uint64_t* out, int64_t n, uint64_t q) {
    for (int64_t i = 0; i < n; ++i) out[i] = mulmod(a[i], b[i], q);
}

void orc_vec_mul_scalar(const uint64_t* a, uint64_t s, uint64_t* out, int64_t n, uint64_t q) {
    for (int64_t i = 0; i < n; ++i) out[i] = mulmod(a[i], s, q);
}

/* out = (acc + a * s) mod q */
void orc_vec_mac_scalar(const uint64_t* acc, const uint64_t* a, uint64_t s, uint64_t* out,
                        int64_t n, uint64_t q) {
    for (int64_t i = 0; i < n; ++i) out[i] = addmod(acc[i], mulmod(a[i], s, q), q);
}

/* out = a mod q for arbitrary 64-bit a */
void orc_vec_reduce(const uint64_t* a, uint64_t* out, int64_t n, uint64_t q) {
    for (int64_t i = 0; i < n; ++i) out[i] = a[i] % q;
}

/* out = a mod q for signed a, result in [0, q) */
void orc_vec_from_signed(const int64_t* a, uint64_t* out, int64_t n, uint64_t q) {
    for (int64_t i = 0; i < n; ++i) {
        int64_t v = a[i];
        if (v >= 0) out[i] = (uint64_t)v % q;
        else {
            uint64_t m = (uint64_t)(-(v + 1)) + 1u;   /* |v| without overflow */
            uint64_t r = m % q;
            out[i] = r ? q - r : 0;
        }
    }
}

/* ---- ring products ---- */

/* The definition of the product in Z_q[X]/(X^n+1). O(n^2). */
void orc_negacyclic_schoolbook(const uint64_t* a, const uint64_t* b, uint64_t* c, int64_t n,
                               uint64_t q) {
    for (int64_t k = 0; k < n; ++k) c[k] = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (a[i] == 0) continue;
        for (int64_t j = 0; j < n; ++j) {
            uint64_t p = mulmod(a[i], b[j], q);
            int64_t k = i + j;
            if (k < n) c[k] = addmod(c[k], p, q);
            else c[k - n] = submod(c[k - n], p, q);
        }
    }
}

/* One coefficient of the definition above; used to spot-check large products. */
uint64_t orc_negacyclic_coeff(const uint64_t* a, const uint64_t* b, int64_t n, uint64_t q,
                              int64_t k) {
    uint64_t s = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t j = k - i;
        if (j >= 0) s = addmod(s, mulmod(a[i], b[j], q), q);
        else s = submod(s, mulmod(a[i], b[j + n], q), q);
    }
    return s;
}

/* Cyclic DFT of length n (power of two) with root w, natural order in and out:
 *   out[k] = sum_i x[i] w^(k i).  Iterative radix-2 (bit-reverse copy, then butterflies). */
static void cyclic_dft(uint64_t* x, int64_t n, uint64_t q, uint64_t w) {
    int64_t lg = 0;
    while (((int64_t)1 << lg) < n) ++lg;
    for (int64_t i = 0; i < n; ++i) {
        int64_t r = 0;
        for (int64_t b = 0; b < lg; ++b)
            if (i & ((int64_t)1 << b)) r |= (int64_t)1 << (lg - 1 - b);
        if (r > i) { uint64_t t = x[i]; x[i] = x[r]; x[r] = t; }
    }
    for (int64_t len = 2; len <= n; len <<= 1) {
        uint64_t wl = orc_powmod(w, (uint64_t)(n / len), q); /* primitive len-th root */
        for (int64_t s = 0; s < n; s += len) {
            uint64_t wk = 1;
            for (int64_t j = 0; j < len / 2; ++j) {
                uint64_t u = x[s + j];
                uint64_t v = mulmod(x[s + j + len / 2], wk, q);
                x[s + j] = addmod(u, v, q);
                x[s + j + len / 2] = submod(u, v, q);
                wk = mulmod(wk, wl, q);
            }
        }
    }
}

/* out[k] = a(psi^(2k+1)) = sum_i a_i psi^((2k+1) i), k = 0..n-1.  psi: primitive 2n-th root. */
void orc_negacyclic_eval(const uint64_t* a, uint64_t* out, int64_t n, uint64_t q, uint64_t psi) {
    uint64_t pw = 1;
    for (int64_t i = 0; i < n; ++i) {
        out[i] = mulmod(a[i] % q, pw, q);
        pw = mulmod(pw, psi, q);
    }
    cyclic_dft(out, n, q, mulmod(psi, psi, q));
}

/* Inverse of orc_negacyclic_eval: the polynomial whose values at psi^(2k+1) are v[k]. */
void orc_negacyclic_interp(const uint64_t* v, uint64_t* out, int64_t n, uint64_t q,
                           uint64_t psi) {
    uint64_t psi_inv = orc_powmod(psi, q - 2, q);
    uint64_t n_inv = orc_powmod((uint64_t)n % q, q - 2, q);
    for (int64_t i = 0; i < n; ++i) out[i] = v[i] % q;
    cyclic_dft(out, n, q, mulmod(psi_inv, psi_inv, q));
    uint64_t pw = n_inv;
    for (int64_t i = 0; i < n; ++i) {
        out[i] = mulmod(out[i], pw, q);
        pw = mulmod(pw, psi_inv, q);
    }
}

/* c = a * b in Z_q[X]/(X^n+1) through the evaluation map. */
void orc_negacyclic_mul(const uint64_t* a, const uint64_t* b, uint64_t* c, int64_t n, uint64_t q,
                        uint64_t psi) {
    uint64_t* ea = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
    uint64_t* eb = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
    orc_negacyclic_eval(a, ea, n, q, psi);
    orc_negacyclic_eval(b, eb, n, q, psi);
    for (int64_t i = 0; i < n; ++i) ea[i] = mulmod(ea[i], eb[i], q);
    orc_negacyclic_interp(ea, c, n, q, psi);
    free(ea);
    free(eb);
}

/* ---- uniform sampling map: floor((hi * 2^64 + lo) * q / 2^128) ---- */
void orc_uniform_mod(const uint64_t* hi, const uint64_t* lo, uint64_t q, int64_t n, uint64_t* out) {
    for (int64_t i = 0; i < n; ++i) {
        u128 a = (u128)hi[i] * q;            /* contributes a / 2^64 */
        u128 b = (u128)lo[i] * q;            /* contributes b / 2^128 */
        u128 mid = (a & 0xFFFFFFFFFFFFFFFFull) + (b >> 64);
        out[i] = (uint64_t)((a >> 64) + (mid >> 64));
    }
}
