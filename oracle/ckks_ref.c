/*
 * Oracle scalar primitives -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct modular arithmetic on polynomial rows used by
 * the CPU oracle (oracle/ckks.py, oracle/hercules.py).  Only tests/, the smoke
 * check and the benchmark's CPU-baseline leg may load this library; the product
 * path never does.  It shares no code with the CUDA library.
 *
 * Every modular product is computed as ((unsigned __int128)a*b) % q: no
 * Shoup/Barrett/Montgomery tricks, so a reader can check each line by eye.
 *
 * Ring: R_q = Z_q[X]/(X^N+1) with q prime, q = 1 mod 2N (the RNS ring of the
 * paper's MCKKS section, Sec. 2.2).  A "row" is one polynomial modulo one
 * prime: n consecutive uint64 residues.  Functions taking `rows` process
 * `rows` consecutive rows, row r using modulus q[r].
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a * b) % q); }
static uint64_t addmod(uint64_t a, uint64_t b, uint64_t q) { u128 s = (u128)a + b; return (uint64_t)(s % q); }
static uint64_t submod(uint64_t a, uint64_t b, uint64_t q) { return a >= b ? a - b : (uint64_t)(((u128)a + q - b) % q); }

uint64_t ref_powmod(uint64_t a, uint64_t e, uint64_t q)
{
    uint64_t r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

static unsigned bitrev(unsigned x, int bits)
{
    unsigned r = 0;
    for (int i = 0; i < bits; i++) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

/* Definition of the forward transform (used only to pin the fast one):
 *   out[j] = sum_i a[i] * psi^((2*brv(j)+1)*i)  (mod q),  psi a primitive 2N-th root. */
void ref_ntt_direct(uint64_t *out, const uint64_t *a, int logn, uint64_t q, uint64_t psi)
{
    const unsigned n = 1u << logn;
    for (unsigned j = 0; j < n; j++) {
        uint64_t e = 2ull * bitrev(j, logn) + 1;
        uint64_t x = ref_powmod(psi, e, q);  /* evaluation point psi^(2brv(j)+1) */
        uint64_t acc = 0, xp = 1;
        for (unsigned i = 0; i < n; i++) {
            acc = addmod(acc, mulmod(a[i], xp, q), q);
            xp = mulmod(xp, x, q);
        }
        out[j] = acc;
    }
}

/* Textbook radix-2 Cooley-Tukey negacyclic NTT with the psi powers merged
 * into the butterflies; natural-order input, bit-reversed-order output, so
 * that out[j] = a(psi^(2brv(j)+1)) as in ref_ntt_direct. */
static void ntt_forward_one(uint64_t *a, int logn, uint64_t q, uint64_t psi)
{
    const unsigned n = 1u << logn;
    uint64_t *w = (uint64_t *)malloc(sizeof(uint64_t) * n);
    for (unsigned k = 0; k < n; k++) w[k] = ref_powmod(psi, bitrev(k, logn), q);
    for (unsigned m = 1, t = n / 2; m < n; m *= 2, t /= 2) {
        for (unsigned i = 0; i < m; i++) {
            uint64_t s = w[m + i];
            for (unsigned j = 2 * i * t; j < 2 * i * t + t; j++) {
                uint64_t u = a[j], v = mulmod(a[j + t], s, q);
                a[j] = addmod(u, v, q);
                a[j + t] = submod(u, v, q);
            }
        }
    }
    free(w);
}

/* Gentleman-Sande inverse of ntt_forward_one, followed by the factor N^-1. */
static void ntt_inverse_one(uint64_t *a, int logn, uint64_t q, uint64_t psi)
{
    const unsigned n = 1u << logn;
    uint64_t psi_inv = ref_powmod(psi, q - 2, q);
    uint64_t *w = (uint64_t *)malloc(sizeof(uint64_t) * n);
    for (unsigned k = 0; k < n; k++) w[k] = ref_powmod(psi_inv, bitrev(k, logn), q);
    for (unsigned m = n / 2, t = 1; m >= 1; m /= 2, t *= 2) {
        for (unsigned i = 0; i < m; i++) {
            uint64_t s = w[m + i];
            for (unsigned j = 2 * i * t; j < 2 * i * t + t; j++) {
                uint64_t u = a[j], v = a[j + t];
                a[j] = addmod(u, v, q);
                a[j + t] = mulmod(submod(u, v, q), s, q);
            }
        }
    }
    uint64_t n_inv = ref_powmod(n % q, q - 2, q);
    for (unsigned j = 0; j < n; j++) a[j] = mulmod(a[j], n_inv, q);
    free(w);
}

void ref_ntt_forward_rows(uint64_t *a, int rows, int logn, const uint64_t *q, const uint64_t *psi)
{
#pragma omp parallel for schedule(dynamic)
    for (int r = 0; r < rows; r++) ntt_forward_one(a + ((size_t)r << logn), logn, q[r], psi[r]);
}

void ref_ntt_inverse_rows(uint64_t *a, int rows, int logn, const uint64_t *q, const uint64_t *psi)
{
#pragma omp parallel for schedule(dynamic)
    for (int r = 0; r < rows; r++) ntt_inverse_one(a + ((size_t)r << logn), logn, q[r], psi[r]);
}

/* Schoolbook product in Z_q[X]/(X^N+1): X^N = -1 folds the upper half back
 * with a minus sign.  Used only to pin the NTT-based product. */
void ref_negacyclic_schoolbook(uint64_t *out, const uint64_t *a, const uint64_t *b, int n, uint64_t q)
{
    for (int k = 0; k < n; k++) out[k] = 0;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            uint64_t p = mulmod(a[i], b[j], q);
            int k = i + j;
            if (k < n) out[k] = addmod(out[k], p, q);
            else out[k - n] = submod(out[k - n], p, q);
        }
}

void ref_rows_add(uint64_t *out, const uint64_t *a, const uint64_t *b, int rows, int n, const uint64_t *q)
{
    for (int r = 0; r < rows; r++)
        for (int i = 0; i < n; i++) { size_t k = (size_t)r * n + i; out[k] = addmod(a[k], b[k], q[r]); }
}

void ref_rows_sub(uint64_t *out, const uint64_t *a, const uint64_t *b, int rows, int n, const uint64_t *q)
{
    for (int r = 0; r < rows; r++)
        for (int i = 0; i < n; i++) { size_t k = (size_t)r * n + i; out[k] = submod(a[k], b[k], q[r]); }
}

void ref_rows_neg(uint64_t *out, const uint64_t *a, int rows, int n, const uint64_t *q)
{
    for (int r = 0; r < rows; r++)
        for (int i = 0; i < n; i++) { size_t k = (size_t)r * n + i; out[k] = submod(0, a[k], q[r]); }
}

void ref_rows_mul(uint64_t *out, const uint64_t *a, const uint64_t *b, int rows, int n, const uint64_t *q)
{
#pragma omp parallel for
    for (int r = 0; r < rows; r++)
        for (int i = 0; i < n; i++) { size_t k = (size_t)r * n + i; out[k] = mulmod(a[k], b[k], q[r]); }
}

/* out = a * s[r] (one scalar residue per row) */
void ref_rows_mul_scalar(uint64_t *out, const uint64_t *a, const uint64_t *s, int rows, int n, const uint64_t *q)
{
    for (int r = 0; r < rows; r++)
        for (int i = 0; i < n; i++) { size_t k = (size_t)r * n + i; out[k] = mulmod(a[k], s[r], q[r]); }
}

/* out = a + s[r] */
void ref_rows_add_scalar(uint64_t *out, const uint64_t *a, const uint64_t *s, int rows, int n, const uint64_t *q)
{
    for (int r = 0; r < rows; r++)
        for (int i = 0; i < n; i++) { size_t k = (size_t)r * n + i; out[k] = addmod(a[k], s[r], q[r]); }
}

/* out = x mod q[r] for arbitrary 64-bit x */
void ref_rows_reduce(uint64_t *out, const uint64_t *x, int rows, int n, const uint64_t *q)
{
    for (int r = 0; r < rows; r++)
        for (int i = 0; i < n; i++) { size_t k = (size_t)r * n + i; out[k] = x[k] % q[r]; }
}

/* Automorphism sigma_g : a(X) -> a(X^g), g odd, on rows in the NTT (evaluation)
 * representation out[j] = a(psi^(2brv(j)+1)):
 *   sigma_g(a)(psi^e) = a(psi^(e*g)), so out[j] = in[j'] with
 *   2brv(j')+1 = (2brv(j)+1)*g mod 2N. */
void ref_automorphism_ntt(uint64_t *out, const uint64_t *in, int rows, int logn, uint64_t g)
{
    const unsigned n = 1u << logn;
    const uint64_t two_n = 2ull * n;
    for (unsigned j = 0; j < n; j++) {
        uint64_t e = ((2ull * bitrev(j, logn) + 1) * (g % two_n)) % two_n;
        unsigned jp = bitrev((unsigned)((e - 1) / 2), logn);
        for (int r = 0; r < rows; r++) out[(size_t)r * n + j] = in[(size_t)r * n + jp];
    }
}

/* Same automorphism on the coefficient representation: coefficient i moves
 * to i*g mod 2N; landing in [N, 2N) means X^N = -1 flips its sign. */
void ref_automorphism_coef(uint64_t *out, const uint64_t *in, int rows, int logn, uint64_t g, const uint64_t *q)
{
    const unsigned n = 1u << logn;
    const uint64_t two_n = 2ull * n;
    for (int r = 0; r < rows; r++)
        for (unsigned i = 0; i < n; i++) {
            uint64_t d = ((uint64_t)i * (g % two_n)) % two_n;
            uint64_t v = in[(size_t)r * n + i];
            if (d < n) out[(size_t)r * n + d] = v;
            else out[(size_t)r * n + (d - n)] = submod(0, v, q[r]);
        }
}

/* Fast basis conversion of Han-Ki hybrid key switching (no correction term):
 * for each destination prime t,
 *   out_t = sum_i [ x_i * qhat_inv_i ]_{q_i} * (qhat_i mod t)   (mod t)
 * where the x_i are the residues of one integer modulo the source primes q_i.
 * qhat_mod_dst is laid out [n_src][n_dst]. */
void ref_basis_convert(uint64_t *out, const uint64_t *in, int n, int n_src, const uint64_t *src_q,
                       const uint64_t *qhat_inv, int n_dst, const uint64_t *dst_q, const uint64_t *qhat_mod_dst)
{
    uint64_t *y = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n_src * n);
    for (int i = 0; i < n_src; i++)
        for (int c = 0; c < n; c++) y[(size_t)i * n + c] = mulmod(in[(size_t)i * n + c], qhat_inv[i], src_q[i]);
#pragma omp parallel for
    for (int t = 0; t < n_dst; t++)
        for (int c = 0; c < n; c++) {
            uint64_t acc = 0;
            for (int i = 0; i < n_src; i++)
                acc = addmod(acc, mulmod(y[(size_t)i * n + c] % dst_q[t], qhat_mod_dst[(size_t)i * n_dst + t], dst_q[t]), dst_q[t]);
            out[(size_t)t * n + c] = acc;
        }
    free(y);
}
