/*
 * oracle.c -- plain, slow, obviously-correct CPU oracle for exact decimal multiplication
 * (Krapivensky, "Speeding up decimal multiplication", arXiv 2011.11524).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its Python
 * binding) may link, import or call this file.  Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline / reference leg use it.  It shares no code, header, table or
 * constant with the GPU path.
 *
 * What is here, and the passage each part follows:
 *   - or_conv_schoolbook   : the convolution c_k = sum_{i+j=k} x_i y_j of the zero-padded limb
 *                            vectors (Sec. 3.1 eq. "star", Sec. 3.2), exact in 128-bit integers.
 *   - or_carry             : the carry recurrence sigma_0 = 0, z_i = (sigma_i + c_i) mod B,
 *                            sigma_{i+1} = (sigma_i + c_i) div B (Sec. 3.2, eq. sigmai_and_zi).
 *   - or_mul_schoolbook    : the product by definition = the two above.
 *   - or_ntt_mul           : an independent slow route for large sizes: number-theoretic
 *                            transform over two primes c*3*2^n+1 below 2^63 (Sec. 3.5, Sec. 4.2
 *                            with l = 2 and 64-bit words, Sec. 4.5), textbook radix-2 DIF/DIT with
 *                            explicit bit reversal (Sec. 5.1-5.3), plain % on 128-bit products
 *                            (no Montgomery, no matrix decomposition), the two-prime CRT formula of
 *                            Sec. 8.2.2 and the carry recurrence.
 *   - or_dft_naive         : the DFT by its definition (Sec. 3.3, eq. dft), O(n^2).
 *   - or_fingerprint       : X mod q of a base-10^9 limb vector by Horner's rule (and
 *                            or_fingerprint_many: the same for many vectors, threaded by vector).
 *   - or_is_prime_mr       : Miller-Rabin with the first 12 primes as bases (Sec. 4.5).
 *   - or_find_primes       : FindPrimesForN / FindPrimes of Sec. 4.5.
 *   - or_transpose         : the out-of-place transpose (definition; Sec. 7.5 row-major order).
 *   - or_permute_rows_rho  : the row permutation rho of Sec. 7.6 (row i -> n*(i mod 2) + i div 2).
 *
 * Every function is single-threaded and uses no blocking or reordering beyond its definition,
 * except or_conv_schoolbook, which may split the output index range across threads (each
 * thread computes whole coefficients by the definition).
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef unsigned __int128 u128;

#define OR_BASE 1000000000u /* B = 10^9: the limb base of the library's I/O format */

/* ------------------------------------------------------------------------------------------ */
/* Sec. 3.1-3.2: c_k = sum over i+j = k of x_i * y_j, k in [0, n+m).  Each c_k is stored as two  */
/* 64-bit words (lo, hi) of an unsigned 128-bit integer.                                        */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    const uint32_t *x, *y;
    size_t n, m, k0, k1;
    uint64_t *c;
} conv_job;

static void *conv_worker(void *arg)
{
    conv_job *J = (conv_job *)arg;
    for (size_t k = J->k0; k < J->k1; ++k) {
        /* i ranges over max(0, k-m+1) .. min(k, n-1) */
        size_t ilo = (k + 1 > J->m) ? k + 1 - J->m : 0;
        size_t ihi = (k < J->n - 1) ? k : J->n - 1;
        u128 s = 0;
        for (size_t i = ilo; i <= ihi && i < J->n; ++i)
            s += (u128)J->x[i] * (u128)J->y[k - i];
        J->c[2 * k] = (uint64_t)s;
        J->c[2 * k + 1] = (uint64_t)(s >> 64);
    }
    return NULL;
}

void or_conv_schoolbook(const uint32_t *x, size_t n, const uint32_t *y, size_t m,
                        uint64_t *c, int nthreads)
{
    size_t L = n + m;
    if (n == 0 || m == 0) {
        memset(c, 0, 2 * L * sizeof(uint64_t));
        return;
    }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    conv_job jobs[256];
    /* split the output range into contiguous blocks of roughly equal work */
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].x = x; jobs[t].y = y; jobs[t].n = n; jobs[t].m = m; jobs[t].c = c;
        jobs[t].k0 = L * (size_t)t / (size_t)nthreads;
        jobs[t].k1 = L * (size_t)(t + 1) / (size_t)nthreads;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, conv_worker, &jobs[t]);
    conv_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* One coefficient c_k of the same convolution, by its definition (for sampled checks). */
void or_conv_at(const uint32_t *x, size_t n, const uint32_t *y, size_t m, size_t k, uint64_t *out2)
{
    u128 s = 0;
    if (n > 0 && m > 0 && k < n + m) {
        size_t ilo = (k + 1 > m) ? k + 1 - m : 0;
        size_t ihi = (k < n - 1) ? k : n - 1;
        for (size_t i = ilo; i <= ihi; ++i) s += (u128)x[i] * (u128)y[k - i];
    }
    out2[0] = (uint64_t)s;
    out2[1] = (uint64_t)(s >> 64);
}

/* Sec. 3.2, eq. sigmai_and_zi.  c is 2 words per coefficient; writes z[0..L).  Returns the   */
/* final carry sigma_L truncated to 64 bits (0 when the product fits in L limbs).            */
uint64_t or_carry(const uint64_t *c, size_t L, uint32_t *z)
{
    u128 sigma = 0;
    for (size_t i = 0; i < L; ++i) {
        u128 ci = ((u128)c[2 * i + 1] << 64) | (u128)c[2 * i];
        u128 t = sigma + ci;
        z[i] = (uint32_t)(t % OR_BASE);
        sigma = t / OR_BASE;
    }
    return (uint64_t)sigma;
}

/* The product by definition: schoolbook convolution then carry.  z has n+m limbs.            */
int or_mul_schoolbook(const uint32_t *x, size_t n, const uint32_t *y, size_t m, uint32_t *z,
                      int nthreads)
{
    size_t L = n + m;
    uint64_t *c = (uint64_t *)malloc(2 * L * sizeof(uint64_t) + 16);
    if (!c) return -1;
    or_conv_schoolbook(x, n, y, m, c, nthreads);
    uint64_t top = or_carry(c, L, z);
    free(c);
    return top == 0 ? 0 : -2;
}

/* ------------------------------------------------------------------------------------------ */
/* Field arithmetic mod a prime p < 2^63 with plain 128-bit % (no Montgomery).                */
/* ------------------------------------------------------------------------------------------ */
static inline uint64_t mulmod(uint64_t a, uint64_t b, uint64_t p) { return (uint64_t)(((u128)a * b) % p); }
static inline uint64_t addmod(uint64_t a, uint64_t b, uint64_t p) { u128 s = (u128)a + b; return (uint64_t)(s % p); }
static inline uint64_t submod(uint64_t a, uint64_t b, uint64_t p) { return a >= b ? a - b : (uint64_t)((u128)a + p - b); }

uint64_t or_powmod(uint64_t a, uint64_t e, uint64_t p)
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

/* Sec. 4.5: Miller-Rabin with the first 12 primes as bases (deterministic below 2^64).      */
int or_is_prime_mr(uint64_t n)
{
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; ++i) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; ++s; }
    for (int i = 0; i < 12; ++i) {
        uint64_t x = or_powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int witness = 1;
        for (int r = 1; r < s; ++r) {
            x = mulmod(x, x, n);
            if (x == n - 1) { witness = 0; break; }
        }
        if (witness) return 0;
    }
    return 1;
}

/* Sec. 4.5, FindPrimesForN(n, pmax, l): the (up to) l largest primes psi*2^n + 1 <= pmax with */
/* psi odd and divisible by 3 (psi = 3c, c odd).  Appends to out, returns how many it found.   */
static int find_primes_for_n(int n, uint64_t pmax, int l, uint64_t *out)
{
    int cnt = 0;
    uint64_t psi = (pmax - 1) >> n;
    if (psi % 2 == 0) {
        if (psi == 0) return 0;
        psi -= 1;
    }
    while (psi > 0 && psi % 3 != 0) psi = psi >= 2 ? psi - 2 : 0;
    while (psi > 0 && cnt < l) {
        uint64_t p = (psi << n) + 1;
        if (or_is_prime_mr(p)) out[cnt++] = p;
        if (psi <= 6) break;
        psi -= 6;
    }
    return cnt;
}

/* Sec. 4.5, FindPrimes(w, n_min, l): the l largest primes c*3*2^n+1 < 2^(w-1), n >= n_min,   */
/* c odd.  Writes them in DESCENDING order.  Returns 0, or -1 when fewer than l exist.         */
int or_find_primes(int w, int n_min, int l, uint64_t *out)
{
    if (w < 4 || w > 64 || l < 1 || l > 16) return -1;
    uint64_t pmax = (w == 64) ? (((uint64_t)1 << 63) - 1) : ((((uint64_t)1) << (w - 1)) - 1);
    uint64_t pool[64 * 16];
    int np = 0;
    for (int n = n_min; n <= w - 2; ++n) {
        uint64_t tmp[16];
        int c = find_primes_for_n(n, pmax, l, tmp);
        for (int i = 0; i < c; ++i) {
            int dup = 0;
            for (int j = 0; j < np; ++j) dup |= (pool[j] == tmp[i]);
            if (!dup) pool[np++] = tmp[i];
        }
    }
    if (np < l) return -1;
    /* selection of the l largest, descending */
    for (int i = 0; i < l; ++i) {
        int best = i;
        for (int j = i + 1; j < np; ++j) if (pool[j] > pool[best]) best = j;
        uint64_t t = pool[i]; pool[i] = pool[best]; pool[best] = t;
        out[i] = pool[i];
    }
    return 0;
}

/* Smallest generator of F_p^* (p prime): g such that g^((p-1)/f) != 1 for every prime f | p-1. */
uint64_t or_primitive_root(uint64_t p)
{
    uint64_t f[64];
    int nf = 0;
    uint64_t r = p - 1;
    for (uint64_t d = 2; d * d <= r; ++d) {
        if (r % d == 0) {
            f[nf++] = d;
            while (r % d == 0) r /= d;
        }
    }
    if (r > 1) f[nf++] = r;
    for (uint64_t g = 2; g < p; ++g) {
        int ok = 1;
        for (int i = 0; i < nf && ok; ++i) ok = (or_powmod(g, (p - 1) / f[i], p) != 1);
        if (ok) return g;
    }
    return 0;
}

/* Sec. 3.3 eq. dft: out[k] = sum_i a[i] * w^(i k) mod p, straight from the definition.        */
void or_dft_naive(const uint64_t *a, size_t n, uint64_t w, uint64_t p, uint64_t *out)
{
    for (size_t k = 0; k < n; ++k) {
        uint64_t wk = or_powmod(w, (uint64_t)k, p);
        uint64_t s = 0, t = 1;
        for (size_t i = 0; i < n; ++i) {
            s = addmod(s, mulmod(a[i], t, p), p);
            t = mulmod(t, wk, p);
        }
        out[k] = s;
    }
}

/* Sec. 5.1: the bit-reversal permutation of a length-2^lg array. */
static void bitrev_permute(uint64_t *A, size_t n, int lg)
{
    for (size_t k = 0; k < n; ++k) {
        size_t r = 0;
        for (int b = 0; b < lg; ++b) r |= ((k >> b) & 1) << (lg - 1 - b);
        if (k < r) { uint64_t t = A[k]; A[k] = A[r]; A[r] = t; }
    }
}

/* tau(A, w): A'[k] = sum_i A[i] w^(ik) for |A| = 2^lg, by radix-2 decimation in frequency      */
/* (Gentleman-Sande butterflies, Sec. 5.3) followed by bit reversal.  w must have order 2^lg.  */
void or_tau_dif(uint64_t *A, int lg, uint64_t w, uint64_t p)
{
    size_t n = (size_t)1 << lg;
    uint64_t *tw = (uint64_t *)malloc((n / 2 + 1) * sizeof(uint64_t));
    for (int s = lg; s >= 1; --s) {
        size_t m = (size_t)1 << s, h = m / 2;
        uint64_t wm = or_powmod(w, (uint64_t)(n / m), p); /* primitive m-th root */
        tw[0] = 1;
        for (size_t j = 1; j < h; ++j) tw[j] = mulmod(tw[j - 1], wm, p);
        for (size_t k = 0; k < n; k += m) {
            for (size_t j = 0; j < h; ++j) {
                uint64_t u = A[k + j], v = A[k + j + h];
                A[k + j] = addmod(u, v, p);
                A[k + j + h] = mulmod(submod(u, v, p), tw[j], p);
            }
        }
    }
    free(tw);
    bitrev_permute(A, n, lg);
}

/* The same tau(A, w) by radix-2 decimation in time (Cooley-Tukey butterflies, Sec. 5.2):     */
/* bit reversal first, then the butterfly levels.                                               */
void or_tau_dit(uint64_t *A, int lg, uint64_t w, uint64_t p)
{
    size_t n = (size_t)1 << lg;
    uint64_t *tw = (uint64_t *)malloc((n / 2 + 1) * sizeof(uint64_t));
    bitrev_permute(A, n, lg);
    for (int s = 1; s <= lg; ++s) {
        size_t m = (size_t)1 << s, h = m / 2;
        uint64_t wm = or_powmod(w, (uint64_t)(n / m), p);
        tw[0] = 1;
        for (size_t j = 1; j < h; ++j) tw[j] = mulmod(tw[j - 1], wm, p);
        for (size_t k = 0; k < n; k += m) {
            for (size_t j = 0; j < h; ++j) {
                uint64_t u = A[k + j], v = mulmod(tw[j], A[k + j + h], p);
                A[k + j] = addmod(u, v, p);
                A[k + j + h] = submod(u, v, p);
            }
        }
    }
    free(tw);
}

/* Cyclic convolution mod p of two length-2^lg vectors by the convolution theorem              */
/* (Sec. 3.3 eq. conv_theorem): f^-1(f(a) . f(b)) with f = tau(., xi) and                      */
/* f^-1 = N^-1 tau(., xi^-1).  a is overwritten with the result; b is destroyed.  a == b means  */
/* a squaring (b is then not touched separately).                                               */
void or_cyclic_conv_mod(uint64_t *a, uint64_t *b, int lg, uint64_t p)
{
    size_t n = (size_t)1 << lg;
    uint64_t g = or_primitive_root(p);
    uint64_t xi = or_powmod(g, (p - 1) >> lg, p);
    uint64_t xi_inv = or_powmod(xi, p - 2, p);
    uint64_t n_inv = or_powmod((uint64_t)(n % p), p - 2, p);
    or_tau_dif(a, lg, xi, p);
    if (b != a) or_tau_dif(b, lg, xi, p);
    for (size_t i = 0; i < n; ++i) a[i] = mulmod(a[i], (b == a) ? a[i] : b[i], p);
    or_tau_dit(a, lg, xi_inv, p);
    for (size_t i = 0; i < n; ++i) a[i] = mulmod(a[i], n_inv, p);
}

/* Independent slow route to the product for sizes where the schoolbook is too slow.           */
/* Primes: FindPrimes(64, 23, 2) sorted ascending (Sec. 4.2 choice l = 2, Sec. 4.5); the       */
/* coefficient bound c_k <= (B-1)^2 min(n, m) < 2^60 * 2^23 < p1 p2 ~ 2^126 (eq. ci_bound, eq.  */
/* product_inequality) makes the two-prime CRT exact.  Transform length: the smallest power of */
/* two >= n + m (Sec. 3.2 padding).  Returns 0 on success.                                      */
int or_ntt_mul(const uint32_t *x, size_t n, const uint32_t *y, size_t m, uint32_t *z)
{
    size_t L = n + m;
    if (n == 0 || m == 0) { memset(z, 0, L * sizeof(uint32_t)); return 0; }
    int lg = 0;
    while (((size_t)1 << lg) < L) ++lg;
    if (lg > 23) return -3; /* the primes' 2-adic order bounds the length (Sec. 3.5) */
    size_t N = (size_t)1 << lg;
    uint64_t P[2];
    if (or_find_primes(64, 23, 2, P) != 0) return -4;
    uint64_t p1 = P[1], p2 = P[0]; /* ascending: p1 < p2 (Sec. 8.2.2) */
    int sq = (x == y && n == m);
    uint64_t *r[2];
    for (int t = 0; t < 2; ++t) {
        uint64_t p = t == 0 ? p1 : p2;
        uint64_t *a = (uint64_t *)calloc(N, sizeof(uint64_t));
        uint64_t *b = sq ? a : (uint64_t *)calloc(N, sizeof(uint64_t));
        if (!a || !b) return -1;
        for (size_t i = 0; i < n; ++i) a[i] = x[i] % p;
        if (!sq) for (size_t i = 0; i < m; ++i) b[i] = y[i] % p;
        or_cyclic_conv_mod(a, b, lg, p);
        if (!sq) free(b);
        r[t] = a;
    }
    /* Sec. 8.2.2: m = a1 + p1 * ((r (a2 - a1)) mod p2), r = p1^-1 mod p2 */
    uint64_t rinv = or_powmod(p1 % p2, p2 - 2, p2);
    uint64_t *c = (uint64_t *)malloc(2 * L * sizeof(uint64_t));
    if (!c) return -1;
    for (size_t k = 0; k < L; ++k) {
        uint64_t a1 = r[0][k], a2 = r[1][k];
        uint64_t psi = submod(a2 % p2, a1 % p2, p2);
        uint64_t phi = mulmod(rinv, psi, p2);
        u128 v = (u128)a1 + (u128)p1 * phi;
        c[2 * k] = (uint64_t)v;
        c[2 * k + 1] = (uint64_t)(v >> 64);
    }
    free(r[0]); free(r[1]);
    uint64_t top = or_carry(c, L, z);
    free(c);
    return top == 0 ? 0 : -2;
}

/* X mod q for X = sum_i limbs[i] * 10^(9 i), by Horner's rule from the top limb. */
uint64_t or_fingerprint(const uint32_t *limbs, size_t n, uint64_t q)
{
    u128 acc = 0;
    for (size_t i = n; i-- > 0;) acc = (acc * OR_BASE + limbs[i]) % q;
    return (uint64_t)acc;
}

/* The same fingerprint for many limb vectors and moduli: out[v * nq + j] = X_v mod q_j.  Each   */
/* thread takes whole vectors (the work is split by vector, never inside one Horner chain).     */
typedef struct {
    const uint64_t *ptrs, *lens, *qs;
    size_t count, nq, next;
    uint64_t *out;
    pthread_mutex_t *mu;
} fp_job;

static void *fp_worker(void *arg)
{
    fp_job *J = (fp_job *)arg;
    for (;;) {
        pthread_mutex_lock(J->mu);
        size_t v = J->next++;
        pthread_mutex_unlock(J->mu);
        if (v >= J->count) break;
        const uint32_t *limbs = (const uint32_t *)(uintptr_t)J->ptrs[v];
        for (size_t j = 0; j < J->nq; ++j) J->out[v * J->nq + j] = or_fingerprint(limbs, J->lens[v], J->qs[j]);
    }
    return NULL;
}

void or_fingerprint_many(const uint64_t *ptrs, const uint64_t *lens, size_t count, const uint64_t *qs,
                         size_t nq, uint64_t *out, int nthreads)
{
    pthread_mutex_t mu = PTHREAD_MUTEX_INITIALIZER;
    fp_job J = {ptrs, lens, qs, count, nq, 0, out, &mu};
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, fp_worker, &J);
    fp_worker(&J);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* Out-of-place transpose of a rows x cols row-major matrix (Sec. 7: row-major convention). */
void or_transpose(const uint32_t *in, size_t rows, size_t cols, uint32_t *out)
{
    for (size_t i = 0; i < rows; ++i)
        for (size_t j = 0; j < cols; ++j) out[j * rows + i] = in[i * cols + j];
}

/* Sec. 7.6: the permutation rho sends row i (0 <= i < 2n) of a 2n-row matrix to row          */
/* n*(i mod 2) + (i div 2).  Applied to the rows of a (2n) x cols row-major matrix.            */
void or_permute_rows_rho(const uint32_t *in, size_t n, size_t cols, uint32_t *out)
{
    for (size_t i = 0; i < 2 * n; ++i) {
        size_t dst = n * (i % 2) + i / 2;
        memcpy(out + dst * cols, in + i * cols, cols * sizeof(uint32_t));
    }
}
