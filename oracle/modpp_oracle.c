/*
 * Test oracle for the Mod-PP-MM hot path of "Fast Homomorphic Linear Algebra
 * with BLAS" (Bae, Cheon, Hanrot, Park, Stehle; arXiv 2503.16080).
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  The product library never
 * links, loads or calls it, and it shares no code with the CUDA path.
 *
 * Everything here is the plain definition, written for a reader to check by
 * eye: 128-bit integer accumulation, one '%' per reduction, schoolbook loops.
 * Speed is a non-goal; OpenMP over output rows is the only concession.
 *
 * Contents (paper section in brackets):
 *   or_mod_pp_mm_i32   Mod-PP-MM, C = U*A mod q, U small signed integers
 *                      [Sec. 5 notation ModPPMM; Thm th:pcmm]
 *   or_mod_pp_mm_res   Mod-PP-MM with both operands residues mod q [Alg. 8 step 2]
 *   or_negacyclic_*    products in R_q = Z_q[X]/(X^N+1) [Sec. 2, ring R_{q,N}]
 *   or_ckks_encode     Ecd_coeff: floor(Delta*z + 1/2) [Sec. 2.2, Encoding]
 *   or_rlwe_*          symmetric RLWE encryption / decryption a*s + b [Sec. 2.1, 2.2]
 *   or_crt2_centered   two-prime CRT to a centred integer
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef __int128 i128;
typedef unsigned __int128 u128;

/* ---- scalar modular helpers (definitions) ---------------------------- */

static uint64_t red_i128(i128 x, uint64_t q) {
    i128 r = x % (i128)q;
    if (r < 0) r += (i128)q;
    return (uint64_t)r;
}
static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) {
    return (uint64_t)(((u128)a * (u128)b) % (u128)q);
}
static uint64_t addmod(uint64_t a, uint64_t b, uint64_t q) {
    return (uint64_t)(((u128)a + (u128)b) % (u128)q);
}
static uint64_t submod(uint64_t a, uint64_t b, uint64_t q) {
    return a >= b ? a - b : (uint64_t)((u128)a + q - b);
}
static uint64_t powmod(uint64_t b, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    b %= q;
    while (e) {
        if (e & 1) r = mulmod(r, b, q);
        b = mulmod(b, b, q);
        e >>= 1;
    }
    return r;
}
/* inverse of a modulo a prime q (Fermat) */
static uint64_t invmod_prime(uint64_t a, uint64_t q) { return powmod(a, q - 2, q); }

uint64_t or_mulmod(uint64_t a, uint64_t b, uint64_t q) { return mulmod(a, b, q); }
uint64_t or_powmod(uint64_t b, uint64_t e, uint64_t q) { return powmod(b, e, q); }

/* ---- Mod-PP-MM ----------------------------------------------------------
 * C[r][c] = ( sum_t U[r][t] * A[t][c] ) mod q, canonical in [0, q).
 * U: d x k signed 32-bit, row-major with leading dimension ldu.
 * A: k x n residues, row-major with leading dimension lda.
 * The sum is kept exactly in a signed 128-bit accumulator: |U| < 2^31 and
 * A < 2^63 give |term| < 2^94, so k < 2^32 terms cannot overflow.
 * Returns 0, or -1 on a bad argument. */
int or_mod_pp_mm_i32(int64_t d, int64_t k, int64_t n, const int32_t *U, int64_t ldu,
                     const uint64_t *A, int64_t lda, uint64_t *C, int64_t ldc, uint64_t q) {
    if (d < 0 || k < 0 || n < 0 || q < 2 || k >= ((int64_t)1 << 32)) return -1;
    int bad = 0;
#pragma omp parallel
    {
        i128 *acc = (i128 *)malloc(sizeof(i128) * (size_t)(n > 0 ? n : 1));
        if (!acc) {
#pragma omp atomic write
            bad = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t r = 0; r < d; ++r) {
            if (!acc) continue;
            for (int64_t c = 0; c < n; ++c) acc[c] = 0;
            for (int64_t t = 0; t < k; ++t) {
                const int64_t u = U[r * ldu + t];
                if (u == 0) continue;
                const uint64_t *arow = A + t * lda;
                for (int64_t c = 0; c < n; ++c) acc[c] += (i128)u * (i128)arow[c];
            }
            for (int64_t c = 0; c < n; ++c) C[r * ldc + c] = red_i128(acc[c], q);
        }
        free(acc);
    }
    return bad ? -1 : 0;
}

/* Mod-PP-MM with both operands residues mod q (the ciphertext-ciphertext
 * product of Alg. 8, step 2).  Each product is reduced before it is added. */
int or_mod_pp_mm_res(int64_t d, int64_t k, int64_t n, const uint64_t *U, int64_t ldu,
                     const uint64_t *A, int64_t lda, uint64_t *C, int64_t ldc, uint64_t q) {
    if (d < 0 || k < 0 || n < 0 || q < 2) return -1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < d; ++r) {
        for (int64_t c = 0; c < n; ++c) C[r * ldc + c] = 0;
        for (int64_t t = 0; t < k; ++t) {
            const uint64_t u = U[r * ldu + t] % q;
            if (u == 0) continue;
            const uint64_t *arow = A + t * lda;
            for (int64_t c = 0; c < n; ++c)
                C[r * ldc + c] = addmod(C[r * ldc + c], mulmod(u, arow[c] % q, q), q);
        }
    }
    return 0;
}

/* ---- ring arithmetic in R_q = Z_q[X]/(X^N + 1) ----------------------- */

/* Schoolbook negacyclic product: X^N = -1, so a term landing at degree
 * i + j >= N wraps to i + j - N with a minus sign. */
int or_negacyclic_mul_schoolbook(int64_t N, const uint64_t *a, const uint64_t *b, uint64_t *c,
                                 uint64_t q) {
    if (N <= 0 || q < 2) return -1;
    uint64_t *t = (uint64_t *)calloc((size_t)N, sizeof(uint64_t));
    if (!t) return -1;
    for (int64_t i = 0; i < N; ++i) {
        if (a[i] % q == 0) continue;
        for (int64_t j = 0; j < N; ++j) {
            uint64_t p = mulmod(a[i], b[j], q);
            int64_t dgr = i + j;
            if (dgr < N) t[dgr] = addmod(t[dgr], p, q);
            else t[dgr - N] = submod(t[dgr - N], p, q);
        }
    }
    memcpy(c, t, sizeof(uint64_t) * (size_t)N);
    free(t);
    return 0;
}

/* A primitive 2N-th root of unity psi mod prime q (needs q = 1 mod 2N):
 * psi = g^((q-1)/2N) for the first g with psi^N = -1. Returns 0 if none. */
uint64_t or_find_psi(uint64_t q, int64_t N) {
    if (N <= 0 || (q - 1) % (uint64_t)(2 * N) != 0) return 0;
    for (uint64_t g = 2; g < 1000; ++g) {
        uint64_t x = powmod(g, (q - 1) / (uint64_t)(2 * N), q);
        if (powmod(x, (uint64_t)N, q) == q - 1) return x;
    }
    return 0;
}

/* Textbook iterative radix-2 cyclic NTT of length N (power of two) with a
 * primitive N-th root w: out[k] = sum_i a[i] w^(ik). Bit-reversal first. */
static void ntt_cyclic(uint64_t *a, int64_t N, uint64_t w, uint64_t q) {
    for (int64_t i = 1, j = 0; i < N; ++i) {
        int64_t bit = N >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { uint64_t t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (int64_t len = 2; len <= N; len <<= 1) {
        uint64_t wl = powmod(w, (uint64_t)(N / len), q);
        for (int64_t i = 0; i < N; i += len) {
            uint64_t x = 1;
            for (int64_t j = 0; j < len / 2; ++j) {
                uint64_t u = a[i + j], v = mulmod(a[i + j + len / 2], x, q);
                a[i + j] = addmod(u, v, q);
                a[i + j + len / 2] = submod(u, v, q);
                x = mulmod(x, wl, q);
            }
        }
    }
}

/* Negacyclic product through the NTT: twist by psi^i, cyclic convolution
 * with w = psi^2, untwist by psi^-i and scale by N^-1.  Requires q prime,
 * q = 1 mod 2N and N a power of two; falls back to schoolbook otherwise. */
int or_negacyclic_mul(int64_t N, const uint64_t *a, const uint64_t *b, uint64_t *c, uint64_t q) {
    if (N <= 0 || q < 2) return -1;
    uint64_t psi = ((N & (N - 1)) == 0) ? or_find_psi(q, N) : 0;
    if (psi == 0) return or_negacyclic_mul_schoolbook(N, a, b, c, q);
    uint64_t *x = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    uint64_t *y = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    if (!x || !y) { free(x); free(y); return -1; }
    uint64_t pw = 1;
    for (int64_t i = 0; i < N; ++i) {
        x[i] = mulmod(a[i] % q, pw, q);
        y[i] = mulmod(b[i] % q, pw, q);
        pw = mulmod(pw, psi, q);
    }
    uint64_t w = mulmod(psi, psi, q);
    ntt_cyclic(x, N, w, q);
    ntt_cyclic(y, N, w, q);
    for (int64_t i = 0; i < N; ++i) x[i] = mulmod(x[i], y[i], q);
    ntt_cyclic(x, N, invmod_prime(w, q), q);
    uint64_t ninv = invmod_prime((uint64_t)N % q, q), psi_inv = invmod_prime(psi, q);
    pw = ninv;
    for (int64_t i = 0; i < N; ++i) {
        c[i] = mulmod(x[i], pw, q);
        pw = mulmod(pw, psi_inv, q);
    }
    free(x);
    free(y);
    return 0;
}

/* ---- CKKS coefficient encoding and symmetric RLWE --------------------- */

/* Ecd_coeff: m_i = floor(Delta * z_i + 1/2) (ties go toward +infinity).
 * x = Delta*z is exact when Delta is a power of two.  x + 1/2 is not always
 * representable, so the rounding is taken from the exact split
 * x = floor(x) + frac with frac = x - floor(x) in [0, 1). */
static int64_t round_half_up(double x) {
    double f = floor(x);
    double frac = x - f; /* exact */
    return (int64_t)f + (frac >= 0.5 ? 1 : 0);
}
void or_ckks_encode(int64_t n, const double *z, double delta, int64_t *m) {
    for (int64_t i = 0; i < n; ++i) m[i] = round_half_up(delta * z[i]);
}

/* Dcd_coeff of a centred integer: p / Delta. */
void or_ckks_decode(int64_t n, const int64_t *p, double delta, double *z) {
    for (int64_t i = 0; i < n; ++i) z[i] = (double)p[i] / delta;
}

static uint64_t lift_signed(int64_t v, uint64_t q) { return red_i128((i128)v, q); }

/* Symmetric RLWE encryption of `rows` plaintexts (one per row), for each of
 * the P primes: b = -(a * s) + m + e  mod q_j, so that a*s + b = m + e.
 * a, b: [P][rows][N] residues; s: [N] small signed; m, e: [rows][N].
 * The randomness (a, s, e) is an input. */
int or_rlwe_encrypt_rows(int64_t rows, int64_t N, int P, const uint64_t *primes, const uint64_t *a,
                         const int64_t *s, const int64_t *m, const int64_t *e, uint64_t *b) {
    if (rows < 0 || N <= 0 || P <= 0) return -1;
    int bad = 0;
    for (int j = 0; j < P; ++j) {
        const uint64_t q = primes[j];
        uint64_t *sq = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
        if (!sq) return -1;
        for (int64_t i = 0; i < N; ++i) sq[i] = lift_signed(s[i], q);
#pragma omp parallel
        {
            uint64_t *as = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
#pragma omp for schedule(dynamic, 4)
            for (int64_t r = 0; r < rows; ++r) {
                const uint64_t *ar = a + ((int64_t)j * rows + r) * N;
                uint64_t *br = b + ((int64_t)j * rows + r) * N;
                if (!as || or_negacyclic_mul(N, ar, sq, as, q) != 0) {
#pragma omp atomic write
                    bad = 1;
                    continue;
                }
                for (int64_t i = 0; i < N; ++i) {
                    uint64_t me = lift_signed(m[r * N + i], q);
                    me = addmod(me, lift_signed(e[r * N + i], q), q);
                    br[i] = submod(me, as[i], q);
                }
            }
            free(as);
        }
        free(sq);
    }
    return bad ? -1 : 0;
}

/* Decryption a*s + b mod q_j for each row and prime. out: [P][rows][N]. */
int or_rlwe_decrypt_rows(int64_t rows, int64_t N, int P, const uint64_t *primes, const uint64_t *a,
                         const uint64_t *b, const int64_t *s, uint64_t *out) {
    if (rows < 0 || N <= 0 || P <= 0) return -1;
    int bad = 0;
    for (int j = 0; j < P; ++j) {
        const uint64_t q = primes[j];
        uint64_t *sq = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
        if (!sq) return -1;
        for (int64_t i = 0; i < N; ++i) sq[i] = lift_signed(s[i], q);
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t r = 0; r < rows; ++r) {
            const int64_t off = ((int64_t)j * rows + r) * N;
            if (or_negacyclic_mul(N, a + off, sq, out + off, q) != 0) {
#pragma omp atomic write
                bad = 1;
                continue;
            }
            for (int64_t i = 0; i < N; ++i) out[off + i] = addmod(out[off + i], b[off + i] % q, q);
        }
        free(sq);
    }
    return bad ? -1 : 0;
}

/* Two-prime CRT (Garner) to the centred representative in (-q0q1/2, q0q1/2].
 * out[i] receives it when it fits in int64; overflow[i] is set otherwise. */
void or_crt2_centered(int64_t n, const uint64_t *r0, const uint64_t *r1, uint64_t q0, uint64_t q1,
                      int64_t *out, int32_t *overflow) {
    const uint64_t q0inv = invmod_prime(q0 % q1, q1);
    const i128 Q = (i128)q0 * (i128)q1;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t h = mulmod(submod(r1[i] % q1, r0[i] % q1, q1), q0inv, q1);
        i128 x = (i128)r0[i] + (i128)q0 * (i128)h; /* in [0, Q) */
        if (2 * x > Q) x -= Q;
        int ovf = (x > (i128)INT64_MAX || x < (i128)INT64_MIN);
        overflow[i] = ovf;
        out[i] = ovf ? 0 : (int64_t)x;
    }
}
