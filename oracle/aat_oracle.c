/*
 * aat_oracle.c -- plain, slow CPU oracle for the product of a matrix by its
 * adjoint (Dumas, Pernet, Sedoglavic, "Some fast algorithms multiplying a
 * matrix by its adjoint").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library links, includes or calls
 * this file; only the tests, the package's smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA path.
 *
 * Every routine is the plain definition of what it computes, written out
 * loop by loop, so that it can be checked against the paper by eye:
 *
 *   orc_aat_modp_low      Low(A A^T) mod p                 (Sec. 2, Low/Up
 *                         definition; Algorithm 1 "Ensure"; Thm 3.1 shows the
 *                         recursion reaches exactly this value)
 *   orc_aat_modp_entries  the same value at chosen (i, j)
 *   orc_gemm_modp         X Y^T mod p (the general products P3, P4 of Alg. 1)
 *   orc_complex_low       Low(A A^H) or Low(A A^T) over C in fp64 (Sec. 4.1,
 *                         Sec. 6.1: what Algorithm 2 returns)
 *   orc_freivalds_modp    Sym(C) x == A (A^T x) mod p, a probabilistic check of
 *                         a full-size result
 *   orc_is_prime, orc_legendre, orc_sqrt_mod, orc_sos_modp
 *                         the host number theory of Sec. 4: Euler's criterion,
 *                         Tonelli-Shanks square roots, and Algorithm 3 (SoS)
 *   orc_alg1_sblocks      the four block additions of Algorithm 1 (S1..S4)
 *                         with the skew-unitary Y applied as a dense matrix
 *
 * Residues: an input entry may be any int32; it is first reduced to the
 * canonical range [0, p).  Outputs over F_p are canonical.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

static uint64_t canon(int64_t a, uint64_t p)
{
    int64_t r = a % (int64_t)p;
    if (r < 0) r += (int64_t)p;
    return (uint64_t)r;
}

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t p)
{
    return (uint64_t)(((u128)a * (u128)b) % p);
}

static uint64_t powmod(uint64_t a, uint64_t e, uint64_t p)
{
    uint64_t r = 1 % p;
    a %= p;
    while (e) {
        if (e & 1) r = mulmod(r, a, p);
        a = mulmod(a, a, p);
        e >>= 1;
    }
    return r;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ F_p */

/* C[i*ldc + j] = (sum_l A[i,l] * A[j,l]) mod p for 0 <= j <= i < n.
 * Entries above the diagonal are left untouched. */
int orc_aat_modp_low(const int32_t *A, int64_t n, int64_t k, int64_t lda,
                     uint32_t p, uint32_t *C, int64_t ldc, int threads)
{
    if (n < 0 || k < 0 || p < 2) return -1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t i = n - 1; i >= 0; --i) {
        for (int64_t j = 0; j <= i; ++j) {
            u128 s = 0;
            for (int64_t l = 0; l < k; ++l)
                s += (u128)canon(A[i * lda + l], p) * canon(A[j * lda + l], p);
            C[i * ldc + j] = (uint32_t)(s % p);
        }
    }
    return 0;
}

/* out[t] = (sum_l A[i_t,l] * A[j_t,l]) mod p for the pairs ij[2t], ij[2t+1]. */
int orc_aat_modp_entries(const int32_t *A, int64_t n, int64_t k, int64_t lda,
                         uint32_t p, const int64_t *ij, int64_t count,
                         uint32_t *out, int threads)
{
    if (p < 2) return -1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(static)
#endif
    for (int64_t t = 0; t < count; ++t) {
        int64_t i = ij[2 * t], j = ij[2 * t + 1];
        u128 s = 0;
        if (i >= 0 && i < n && j >= 0 && j < n)
            for (int64_t l = 0; l < k; ++l)
                s += (u128)canon(A[i * lda + l], p) * canon(A[j * lda + l], p);
        out[t] = (uint32_t)(s % p);
    }
    return 0;
}

/* C = X Y^T mod p, X is m x k, Y is n x k, C is m x n (all entries). */
int orc_gemm_modp(const int32_t *X, int64_t ldx, const int32_t *Y, int64_t ldy,
                  int64_t m, int64_t n, int64_t k, uint32_t p,
                  uint32_t *C, int64_t ldc, int threads)
{
    if (p < 2) return -1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j) {
            u128 s = 0;
            for (int64_t l = 0; l < k; ++l)
                s += (u128)canon(X[i * ldx + l], p) * canon(Y[j * ldy + l], p);
            C[i * ldc + j] = (uint32_t)(s % p);
        }
    return 0;
}

/* Freivalds: for each of the nvec vectors x (length n, canonical), check
 * Sym(C) x == A (A^T x) mod p, where Sym(C) is the symmetric matrix whose
 * lower triangle (diagonal included) is the lower triangle of C.
 * Returns the number of vectors that FAIL (0 = consistent). */
int orc_freivalds_modp(const int32_t *A, int64_t n, int64_t k, int64_t lda,
                       const int32_t *C, int64_t ldc, uint32_t p,
                       const uint32_t *xs, int nvec, int threads)
{
    int fails = 0;
    uint64_t *t = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(k > 0 ? k : 1));
    uint64_t *lhs = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    if (!t || !lhs) { free(t); free(lhs); return -1; }
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
    for (int v = 0; v < nvec; ++v) {
        const uint32_t *x = xs + (size_t)v * (size_t)n;
        /* t = A^T x */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int64_t l = 0; l < k; ++l) {
            u128 s = 0;
            for (int64_t i = 0; i < n; ++i)
                s += (u128)canon(A[i * lda + l], p) * (x[i] % p);
            t[l] = (uint64_t)(s % p);
        }
        /* lhs = Sym(C) x */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int64_t i = 0; i < n; ++i) {
            u128 s = 0;
            for (int64_t j = 0; j < n; ++j) {
                int64_t c = (j <= i) ? C[i * ldc + j] : C[j * ldc + i];
                s += (u128)canon(c, p) * (x[j] % p);
            }
            lhs[i] = (uint64_t)(s % p);
        }
        /* compare with A t */
        int bad = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(|:bad)
#endif
        for (int64_t i = 0; i < n; ++i) {
            u128 s = 0;
            for (int64_t l = 0; l < k; ++l)
                s += (u128)canon(A[i * lda + l], p) * t[l];
            if ((uint64_t)(s % p) != lhs[i]) bad |= 1;
        }
        fails += bad;
    }
    free(t);
    free(lhs);
    return fails;
}

/* ------------------------------------------------------------------ C */

/* A is n x k complex, interleaved (re, im) doubles, row stride lda complex
 * entries.  For 0 <= j <= i < n:
 *     conj != 0:  C[i,j] = sum_l A[i,l] * conj(A[j,l])   (A A^H)
 *     conj == 0:  C[i,j] = sum_l A[i,l] * A[j,l]         (A A^T)
 * C is interleaved with row stride ldc complex entries. */
int orc_complex_low(const double *A, int64_t n, int64_t k, int64_t lda,
                    int conj, double *C, int64_t ldc, int threads)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t i = n - 1; i >= 0; --i) {
        for (int64_t j = 0; j <= i; ++j) {
            double sr = 0.0, si = 0.0;
            for (int64_t l = 0; l < k; ++l) {
                double ar = A[2 * (i * lda + l)], ai = A[2 * (i * lda + l) + 1];
                double br = A[2 * (j * lda + l)], bi = A[2 * (j * lda + l) + 1];
                if (conj) bi = -bi;
                sr += ar * br - ai * bi;
                si += ar * bi + ai * br;
            }
            C[2 * (i * ldc + j)] = sr;
            C[2 * (i * ldc + j) + 1] = si;
        }
    }
    return 0;
}

/* The same sum at chosen (i, j) pairs; out is interleaved. */
int orc_complex_entries(const double *A, int64_t n, int64_t k, int64_t lda,
                        int conj, const int64_t *ij, int64_t count, double *out,
                        int threads)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(static)
#endif
    for (int64_t t = 0; t < count; ++t) {
        int64_t i = ij[2 * t], j = ij[2 * t + 1];
        double sr = 0.0, si = 0.0;
        if (i >= 0 && i < n && j >= 0 && j < n)
            for (int64_t l = 0; l < k; ++l) {
                double ar = A[2 * (i * lda + l)], ai = A[2 * (i * lda + l) + 1];
                double br = A[2 * (j * lda + l)], bi = A[2 * (j * lda + l) + 1];
                if (conj) bi = -bi;
                sr += ar * br - ai * bi;
                si += ar * bi + ai * br;
            }
        out[2 * t] = sr;
        out[2 * t + 1] = si;
    }
    return 0;
}

/* ------------------------------------------------------- number theory */

/* Primality by trial division: slow, plain, correct for every p < 2^64 it
 * is given time for (used here for p < 2^32). */
int orc_is_prime(uint64_t p)
{
    if (p < 2) return 0;
    if (p < 4) return 1;
    if (p % 2 == 0) return 0;
    for (uint64_t d = 3; d * d <= p; d += 2)
        if (p % d == 0) return 0;
    return 1;
}

/* Legendre symbol (a/p) for an odd prime p by Euler's criterion:
 * a^((p-1)/2) is 1 for a non-zero square, p-1 for a non-square. */
int orc_legendre(int64_t a, uint64_t p)
{
    uint64_t r = canon(a, p);
    if (r == 0) return 0;
    uint64_t e = powmod(r, (p - 1) / 2, p);
    return e == 1 ? 1 : -1;
}

/* Tonelli-Shanks square root modulo an odd prime p.  Writes the root r with
 * r <= p - r into *root and returns 1, or returns 0 when a is not a square. */
int orc_sqrt_mod(int64_t a_in, uint64_t p, uint64_t *root)
{
    uint64_t a = canon(a_in, p);
    if (a == 0) { *root = 0; return 1; }
    if (orc_legendre((int64_t)a, p) != 1) return 0;
    /* p - 1 = q 2^s with q odd */
    uint64_t q = p - 1, s = 0;
    while ((q & 1) == 0) { q >>= 1; ++s; }
    /* z: any non-square */
    uint64_t z = 2;
    while (orc_legendre((int64_t)z, p) != -1) ++z;
    uint64_t m = s;
    uint64_t c = powmod(z, q, p);
    uint64_t t = powmod(a, q, p);
    uint64_t r = powmod(a, (q + 1) / 2, p);
    while (t != 1) {
        /* least i, 0 < i < m, with t^(2^i) == 1 */
        uint64_t i = 0, tt = t;
        while (tt != 1) { tt = mulmod(tt, tt, p); ++i; }
        uint64_t b = c;
        for (uint64_t e = 0; e + 1 < m - i; ++e) b = mulmod(b, b, p);
        m = i;
        c = mulmod(b, b, p);
        t = mulmod(t, c, p);
        r = mulmod(r, b, p);
    }
    if (r > p - r) r = p - r;
    *root = r;
    return 1;
}

/* Algorithm 3 (SoS): (a, b) with a^2 + b^2 == k mod p, p an odd prime.
 * If k is a square, (sqrt(k), 0).  Otherwise let s be the smallest
 * non-residue; s - 1 is then a square c^2, k/s is a square a^2, and
 * k == a^2 s == a^2 (1 + c^2) == a^2 + (a c)^2.  Returns 1 on success. */
int orc_sos_modp(int64_t k_in, uint64_t p, uint64_t *a_out, uint64_t *b_out)
{
    if (p < 3 || !orc_is_prime(p)) return 0;
    uint64_t k = canon(k_in, p);
    if (k == 0) { *a_out = 0; *b_out = 0; return 1; }
    if (orc_legendre((int64_t)k, p) == 1) {
        uint64_t r;
        if (!orc_sqrt_mod((int64_t)k, p, &r)) return 0;
        *a_out = r;
        *b_out = 0;
        return 1;
    }
    uint64_t s = 2;
    while (orc_legendre((int64_t)s, p) == 1) ++s;
    uint64_t c, a;
    if (!orc_sqrt_mod((int64_t)(s - 1), p, &c)) return 0;
    uint64_t sinv = powmod(s, p - 2, p);
    uint64_t r = mulmod(k, sinv, p);
    if (!orc_sqrt_mod((int64_t)r, p, &a)) return 0;
    *a_out = a;
    *b_out = mulmod(a, c, p);
    return 1;
}

/* ------------------------------------------------- Algorithm 1, S blocks */

/* Dense skew-unitary Y (kappa x kappa, row-major, canonical):
 *   ykind 1: Y = i I with i = ya, i^2 == -1            (Sec. 4.2)
 *   ykind 2: Y = [[a, b], [-b, a]] (x) I_{kappa/2}      (Prop. 4.2, pigeonhole)
 * Returns 0 on success. */
int orc_build_y(int ykind, uint32_t ya, uint32_t yb, uint32_t p, int64_t kappa,
                uint32_t *Y)
{
    memset(Y, 0, sizeof(uint32_t) * (size_t)(kappa * kappa));
    if (ykind == 1) {
        for (int64_t j = 0; j < kappa; ++j) Y[j * kappa + j] = ya % p;
        return 0;
    }
    if (ykind == 2) {
        if (kappa % 2) return -1;
        int64_t h = kappa / 2;
        for (int64_t j = 0; j < h; ++j) {
            Y[j * kappa + j] = ya % p;                         /* a I  */
            Y[j * kappa + (j + h)] = yb % p;                   /* b I  */
            Y[(j + h) * kappa + j] = (uint32_t)((p - yb % p) % p); /* -b I */
            Y[(j + h) * kappa + (j + h)] = ya % p;             /* a I  */
        }
        return 0;
    }
    return -1;
}

/* The four additions of Algorithm 1 on A (n x k, n and k even), with
 * A11 = A[0:h, 0:kappa], A12 = A[0:h, kappa:k], A21 = A[h:n, 0:kappa],
 * A22 = A[h:n, kappa:k], h = n/2, kappa = k/2:
 *   S1 = (A21 - A11) Y,  S2 = A22 - A21 Y,  S3 = S1 - A22,  S4 = S3 + A12.
 * Y is applied as a dense kappa x kappa matrix product.  Each S is h x kappa,
 * canonical, row stride kappa. */
int orc_alg1_sblocks(const int32_t *A, int64_t n, int64_t k, int64_t lda,
                     uint32_t p, int ykind, uint32_t ya, uint32_t yb,
                     uint32_t *S1, uint32_t *S2, uint32_t *S3, uint32_t *S4)
{
    if (n % 2 || k % 2) return -1;
    int64_t h = n / 2, kap = k / 2;
    uint32_t *Y = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(kap * kap > 0 ? kap * kap : 1));
    if (!Y) return -2;
    if (orc_build_y(ykind, ya, yb, p, kap, Y)) { free(Y); return -1; }
#define AIJ(r, c) canon(A[(r) * lda + (c)], p)
    for (int64_t i = 0; i < h; ++i) {
        for (int64_t j = 0; j < kap; ++j) {
            u128 s1 = 0, a21y = 0;
            for (int64_t l = 0; l < kap; ++l) {
                uint64_t d = (AIJ(h + i, l) + p - AIJ(i, l)) % p;   /* (A21 - A11)[i,l] */
                s1 += (u128)d * Y[l * kap + j];
                a21y += (u128)AIJ(h + i, l) * Y[l * kap + j];          /* (A21 Y)[i,j] */
            }
            uint64_t v1 = (uint64_t)(s1 % p);
            uint64_t v2 = (AIJ(h + i, kap + j) + p - (uint64_t)(a21y % p)) % p;
            uint64_t v3 = (v1 + p - AIJ(h + i, kap + j)) % p;
            uint64_t v4 = (v3 + AIJ(i, kap + j)) % p;
            S1[i * kap + j] = (uint32_t)v1;
            S2[i * kap + j] = (uint32_t)v2;
            S3[i * kap + j] = (uint32_t)v3;
            S4[i * kap + j] = (uint32_t)v4;
        }
    }
#undef AIJ
    free(Y);
    return 0;
}
