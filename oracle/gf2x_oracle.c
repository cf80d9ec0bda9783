/*
 * gf2x_oracle.c -- the ORACLE for multiplication in F2[X] and F2[X]/(X^n - 1).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The GPU
 * product path never calls, links or imports anything from oracle/.
 *
 * It shares no code with the CUDA path: no headers, tables, helpers or
 * constants.  Every function is the plain definition, written for clarity,
 * not speed (the batch driver only runs independent products on several
 * host threads).
 *
 * Data layout (a reading: the paper packs polynomials into 64-bit words but
 * does not fix the order): bit k of a polynomial of n coefficients is bit
 * (k mod 64) of limb floor(k / 64), limbs stored little-endian first, so a
 * polynomial with n coefficients takes ceil(n/64) limbs.  Bits at or above
 * position n of the inputs are ignored (masked); unused bits of every output
 * are written as zero.
 *
 * Definitions followed (paper, Sec. 2.1 and the introduction):
 *   - full product:   c_k = XOR_{i+j=k} a_i b_j,  0 <= k <= 2n-2, stored in
 *                     ceil((2n-1)/64) limbs;
 *   - reduced product: r = c mod (X^n - 1); since X^n = 1 in that ring and
 *                     -1 = 1 in F2, r_k = c_k XOR c_{k+n} for 0 <= k < n
 *                     (the circulant-matrix isomorphism of Sec. 1);
 *   - circulant form:  r_k = XOR_j a_{(k-j) mod n} b_j, the first row of the
 *                     circulant matrix psi^{-1}(a) applied to b (Sec. 1).
 *
 * Parity is pinned by tests/test_oracle_pins.py: brute force over all
 * operand pairs for tiny n, Python big-integer carry-less products,
 * Lucas' theorem closed forms for (1+X)^p (1+X)^q, shift/rotation by X^k,
 * squaring as bit interleaving, parity and degree laws, distributivity.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOMEM 2

static size_t limbs_for_bits(uint64_t bits) { return (size_t)((bits + 63) / 64); }

static int get_bit(const uint64_t *v, uint64_t k) { return (int)((v[k >> 6] >> (k & 63)) & 1u); }

static void flip_bit(uint64_t *v, uint64_t k) { v[k >> 6] ^= (uint64_t)1 << (k & 63); }

/* number of limbs of the full product of two n-coefficient polynomials */
size_t oracle_full_limbs(uint32_t n) { return n == 0 ? 0 : limbs_for_bits(2ull * n - 1); }

/* number of limbs of a polynomial with n coefficients */
size_t oracle_limbs(uint32_t n) { return limbs_for_bits(n); }

/* copy the first n coefficients of src into dst (ceil(n/64) limbs), zeroing
 * every bit at position >= n */
static void copy_masked(uint64_t *dst, const uint64_t *src, uint32_t n)
{
    size_t L = limbs_for_bits(n);
    memcpy(dst, src, L * sizeof(uint64_t));
    if (n % 64)
        dst[L - 1] &= ((uint64_t)1 << (n % 64)) - 1;
}

/* Full product, bit by bit: for every pair (i, j) with a_i = b_j = 1 flip
 * coefficient i+j.  O(n^2) bit operations; meant for n up to a few
 * thousand.  c gets ceil((2n-1)/64) limbs. */
int oracle_mul_bitwise(uint64_t *c, const uint64_t *a, const uint64_t *b, uint32_t n)
{
    if (n == 0 || !c || !a || !b)
        return ORACLE_EINVAL;
    memset(c, 0, oracle_full_limbs(n) * sizeof(uint64_t));
    for (uint32_t i = 0; i < n; ++i) {
        if (!get_bit(a, i))
            continue;
        for (uint32_t j = 0; j < n; ++j)
            if (get_bit(b, j))
                flip_bit(c, (uint64_t)i + j);
    }
    return ORACLE_OK;
}

/* Full product by shift-and-XOR over 64-bit limbs: for every set bit i of b
 * XOR (a << i) into the accumulator.  c gets ceil((2n-1)/64) limbs. */
int oracle_mul(uint64_t *c, const uint64_t *a, const uint64_t *b, uint32_t n)
{
    if (n == 0 || !c || !a || !b)
        return ORACLE_EINVAL;
    size_t L = limbs_for_bits(n);
    size_t Lc = oracle_full_limbs(n);
    uint64_t *am = (uint64_t *)malloc(L * sizeof(uint64_t));
    uint64_t *bm = (uint64_t *)malloc(L * sizeof(uint64_t));
    uint64_t *acc = (uint64_t *)calloc(2 * L + 1, sizeof(uint64_t));
    if (!am || !bm || !acc) {
        free(am); free(bm); free(acc);
        return ORACLE_ENOMEM;
    }
    copy_masked(am, a, n);
    copy_masked(bm, b, n);
    for (uint32_t i = 0; i < n; ++i) {
        if (!get_bit(bm, i))
            continue;
        size_t off = i / 64;
        unsigned s = i % 64;
        for (size_t k = 0; k < L; ++k) {
            acc[off + k] ^= am[k] << s;
            if (s)
                acc[off + k + 1] ^= am[k] >> (64 - s);
        }
    }
    memcpy(c, acc, Lc * sizeof(uint64_t));
    free(am); free(bm); free(acc);
    return ORACLE_OK;
}

/* Fold a full product into F2[X]/(X^n - 1): r_k = c_k XOR c_{k+n}. */
static void fold_xn1(uint64_t *r, const uint64_t *c, uint32_t n)
{
    size_t L = limbs_for_bits(n);
    memset(r, 0, L * sizeof(uint64_t));
    for (uint64_t k = 0; k < 2ull * n - 1; ++k)
        if (get_bit(c, k))
            flip_bit(r, k < n ? k : k - n);
}

/* Reduced product r = a*b mod (X^n - 1), via the full product and a
 * bit-by-bit fold.  r gets ceil(n/64) limbs. */
int oracle_mulmod(uint64_t *r, const uint64_t *a, const uint64_t *b, uint32_t n)
{
    if (n == 0 || !r || !a || !b)
        return ORACLE_EINVAL;
    uint64_t *c = (uint64_t *)malloc(oracle_full_limbs(n) * sizeof(uint64_t));
    if (!c)
        return ORACLE_ENOMEM;
    int st = oracle_mul(c, a, b, n);
    if (st == ORACLE_OK)
        fold_xn1(r, c, n);
    free(c);
    return st;
}

/* Reduced product through the circulant formulation: r_k is the XOR over j
 * of a_{(k-j) mod n} b_j.  Shares nothing with oracle_mul; O(n^2). */
int oracle_mulmod_circulant(uint64_t *r, const uint64_t *a, const uint64_t *b, uint32_t n)
{
    if (n == 0 || !r || !a || !b)
        return ORACLE_EINVAL;
    memset(r, 0, limbs_for_bits(n) * sizeof(uint64_t));
    for (uint32_t k = 0; k < n; ++k) {
        int acc = 0;
        for (uint32_t j = 0; j < n; ++j) {
            uint32_t i = (k >= j) ? k - j : k + n - j;
            acc ^= get_bit(a, i) & get_bit(b, j);
        }
        if (acc)
            flip_bit(r, k);
    }
    return ORACLE_OK;
}

/* Many independent products of the same size, on `nthreads` host threads
 * (0 = all available).  Operand p starts at a + p*stride_in limbs, result p
 * at out + p*stride_out limbs; reduce != 0 selects oracle_mulmod.  Returns
 * the first non-zero status. */
int oracle_mul_batch(uint64_t *out, const uint64_t *a, const uint64_t *b, uint32_t n,
                     size_t count, size_t stride_in, size_t stride_out, int reduce,
                     int nthreads)
{
    if (n == 0 || !out || !a || !b)
        return ORACLE_EINVAL;
    int status = ORACLE_OK;
#ifdef _OPENMP
    if (nthreads <= 0)
        nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (long long p = 0; p < (long long)count; ++p) {
        int st = reduce ? oracle_mulmod(out + p * stride_out, a + p * stride_in, b + p * stride_in, n)
                        : oracle_mul(out + p * stride_out, a + p * stride_in, b + p * stride_in, n);
        if (st != ORACLE_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
            status = st;
        }
    }
    (void)nthreads;
    return status;
}

/* threads the batch driver would use by default */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
