/*
 * Test oracle, part 2: the ring operations that the ciphertext-ciphertext
 * matrix product (Alg. 8) performs around its Mod-PP-MMs.
 *
 * THIS FILE IS TEST INFRASTRUCTURE (see modpp_oracle.c).  Plain loops, one
 * operation per function, in the order the paper states them:
 *
 *   or_monomial_mul     X^t * m in R_q (Sec. 2; PCMult by a monomial, Sec. 2.2)
 *   or_automorphism     m(X) -> m(X^l), l odd (Aut, Sec. 2.2)
 *   or_tweak_def        ct'_j = sum_{i<n} X^(2ijN/n) ct_i (the definition, Alg. 3 ENSURE)
 *   or_tweak_alg        the recursion of Alg. 3 (Tweak)
 *   or_ks_keygen_g      RNS switching keys (SWKGen, Sec. 2.2, with an RNS gadget of D digits)
 *   or_keyswitch_g      KeySwitch with the same gadget and K special primes
 *   or_ks_keygen, or_keyswitch   the same with D = L digits and one special prime
 *   or_rescale          Rescale by the last prime of the RNS chain (Sec. 2.2)
 *
 * Ciphertext layout: ct[part][plane][coef], part 0 = a, part 1 = b; `L`
 * planes, one per prime of the chain q_0 .. q_{L-1}.  Key layout:
 * key[digit][part][plane][coef] with L+K planes (the special primes, whose
 * product is P, last).
 *
 * RNS gadget (SWKGen with gadget rank D, the decomposition number of the
 * footnote of Sec. 2.2): the chain primes fall into D digits of consecutive
 * primes; digit d of a ciphertext's a-part is its residue modulo Q_d, the
 * product of the digit's primes.  Key d encrypts P * g_d * s_old under s_new
 * modulo P*Q, where g_d = (Q/Q_d) * ((Q/Q_d)^-1 mod Q_d), so g_d = 1 mod the
 * digit's primes and 0 mod the other q_k.  KeySwitch sums digit_d * key_d over
 * P*Q and divides by P with rounding.  D = L, K = 1 is one digit per prime.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;
typedef unsigned __int128 u128;

int or_negacyclic_mul(int64_t N, const uint64_t *a, const uint64_t *b, uint64_t *c, uint64_t q);

static uint64_t mmul(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a * b) % q); }
static uint64_t madd(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a + b) % q); }
static uint64_t msub(uint64_t a, uint64_t b, uint64_t q) { return a >= b ? a - b : (uint64_t)((u128)a + q - b); }
static uint64_t mneg(uint64_t a, uint64_t q) { return a == 0 ? 0 : q - a; }
static uint64_t mlift(int64_t v, uint64_t q) {
    i128 r = (i128)v % (i128)q;
    if (r < 0) r += q;
    return (uint64_t)r;
}
static uint64_t mpow(uint64_t b, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    b %= q;
    while (e) {
        if (e & 1) r = mmul(r, b, q);
        b = mmul(b, b, q);
        e >>= 1;
    }
    return r;
}
static uint64_t minv(uint64_t a, uint64_t q) { return mpow(a % q, q - 2, q); }

/* X^t * m in Z_q[X]/(X^N + 1): coefficient i moves to i + t; X^N = -1. */
void or_monomial_mul(int64_t N, int64_t t, const uint64_t *m, uint64_t *out, uint64_t q) {
    int64_t tt = ((t % (2 * N)) + 2 * N) % (2 * N);
    for (int64_t i = 0; i < N; ++i) {
        int64_t p = i + tt;
        int neg = 0;
        while (p >= N) {
            p -= N;
            neg ^= 1;
        }
        out[p] = neg ? mneg(m[i], q) : m[i] % q;
    }
}

/* m(X) -> m(X^l) for odd l: X^i maps to X^(i*l mod 2N), with X^N = -1. */
void or_automorphism(int64_t N, int64_t l, const uint64_t *m, uint64_t *out, uint64_t q) {
    for (int64_t i = 0; i < N; ++i) {
        int64_t p = (int64_t)(((i128)i * l) % (2 * N));
        if (p < 0) p += 2 * N;
        if (p < N) out[p] = m[i] % q;
        else out[p - N] = mneg(m[i], q);
    }
}

/* Tweak by its definition: ct'_j = sum_{i<n} X^(2 i j N/n) ct_i, for j < n.
 * cts: n ciphertexts of W = 2*L*N words each, contiguous. */
void or_tweak_def(int64_t n, int64_t N, int L, const uint64_t *primes, const uint64_t *in,
                  uint64_t *out) {
    const int64_t W = 2 * (int64_t)L * N;
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    for (int64_t j = 0; j < n; ++j) {
        uint64_t *o = out + j * W;
        memset(o, 0, sizeof(uint64_t) * (size_t)W);
        for (int64_t i = 0; i < n; ++i) {
            const int64_t t = 2 * i * j * N / n; /* exact for n | 2N */
            for (int part = 0; part < 2; ++part)
                for (int pl = 0; pl < L; ++pl) {
                    const uint64_t q = primes[pl];
                    const int64_t off = ((int64_t)part * L + pl) * N;
                    or_monomial_mul(N, t, in + i * W + off, tmp, q);
                    for (int64_t c = 0; c < N; ++c) o[off + c] = madd(o[off + c], tmp[c], q);
                }
        }
    }
    free(tmp);
}

/* X^t * ct for every part and plane. */
static void ct_monomial(int64_t N, int L, const uint64_t *primes, int64_t t, const uint64_t *ct,
                        uint64_t *out) {
    for (int part = 0; part < 2; ++part)
        for (int pl = 0; pl < L; ++pl) {
            const int64_t off = ((int64_t)part * L + pl) * N;
            or_monomial_mul(N, t, ct + off, out + off, primes[pl]);
        }
}

/* Alg. 3 (Tweak): in[idx[i]], i < n, are the input ciphertexts. */
static void tweak_rec(int64_t n, int64_t N, int L, const uint64_t *primes, const uint64_t *in,
                      const int64_t *idx, uint64_t *out) {
    const int64_t W = 2 * (int64_t)L * N;
    if (n == 1) {
        memcpy(out, in + idx[0] * W, sizeof(uint64_t) * (size_t)W);
        return;
    }
    memcpy(out, in + idx[0] * W, sizeof(uint64_t) * (size_t)W); /* ct'_0 = ct_0 */
    uint64_t *tw = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)W);
    for (int64_t half = 1; half < n; half <<= 1) { /* half = 2^l */
        /* aux = Tweak((ct_{(2j+1) n / 2^(l+1)})_{j < 2^l}) */
        int64_t *sub = (int64_t *)malloc(sizeof(int64_t) * (size_t)half);
        for (int64_t j = 0; j < half; ++j) sub[j] = idx[(2 * j + 1) * (n / (2 * half))];
        uint64_t *aux = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(half * W));
        tweak_rec(half, N, L, primes, in, sub, aux);
        for (int64_t j = 0; j < half; ++j) {
            ct_monomial(N, L, primes, (N / half) * j, aux + j * W, tw); /* X^{(N/2^l) j} aux_j */
            uint64_t *lo = out + j * W, *hi = out + (j + half) * W;
            for (int part = 0; part < 2; ++part)
                for (int pl = 0; pl < L; ++pl) {
                    const uint64_t q = primes[pl];
                    const int64_t off = ((int64_t)part * L + pl) * N;
                    for (int64_t c = 0; c < N; ++c) {
                        hi[off + c] = msub(lo[off + c], tw[off + c], q);
                        lo[off + c] = madd(lo[off + c], tw[off + c], q);
                    }
                }
        }
        free(aux);
        free(sub);
    }
    free(tw);
}

void or_tweak_alg(int64_t n, int64_t N, int L, const uint64_t *primes, const uint64_t *in,
                  uint64_t *out) {
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) idx[i] = i;
    tweak_rec(n, N, L, primes, in, idx, out);
    free(idx);
}

/* Digit d of the RNS gadget with D digits over L chain primes holds the
 * primes [d * alpha, min(L, (d + 1) * alpha)), alpha = ceil(L / D). */
static int digit_lo(int L, int D, int d) { return d * ((L + D - 1) / D); }
static int digit_hi(int L, int D, int d) {
    const int hi = (d + 1) * ((L + D - 1) / D);
    return hi < L ? hi : L;
}

/* The gadget's limits here: every digit non-empty, and at most two primes per
 * digit and two special primes, so that Q_d and P fit in 128 bits. */
static int gadget_ok(int L, int K, int D) {
    if (L < 1 || D < 1 || D > L || K < 1 || K > 2) return 0;
    const int alpha = (L + D - 1) / D;
    return alpha <= 2 && (D - 1) * alpha < L;
}

/* Exact CRT lift of residues r[0..m) modulo the primes p[0..m) (m <= 2,
 * product M < 2^126) to the integer x in [0, M):
 * x = sum_j [r_j * (M/p_j)^-1]_{p_j} * (M/p_j) mod M. */
static u128 crt_lift(int m, const uint64_t *r, const uint64_t *p, u128 *M_out) {
    u128 M = 1;
    for (int j = 0; j < m; ++j) M *= p[j];
    u128 x = 0;
    for (int j = 0; j < m; ++j) {
        u128 Mj = M / p[j];
        const uint64_t t = mmul(r[j] % p[j], minv((uint64_t)(Mj % p[j]), p[j]), p[j]);
        x = (x + (u128)t * Mj) % M;
    }
    if (M_out) *M_out = M;
    return x;
}

/* Switching keys from s_old to s_new modulo P*Q, P the product of the K
 * special primes primes[L .. L+K-1], with the RNS gadget of D digits (SWKGen
 * of Sec. 2.2 with gadget rank D, the decomposition number of the footnote).
 * Key d encrypts P * g_d * s_old under s_new, g_d = (Q/Q_d) [(Q/Q_d)^-1]_{Q_d}
 * with Q_d the product of digit d's primes: g_d = 1 mod those primes and 0
 * mod every other chain prime, and P * g_d = 0 mod the special primes.
 * a: [D][L+K][N] uniform residues; e: [D][N] small errors (the randomness).
 * key: [D][2][L+K][N]; part 0 = a_d, part 1 = -a_d s_new + e_d + P g_d s_old. */
int or_ks_keygen_g(int64_t N, int L, int K, int D, const uint64_t *primes, const int64_t *s_old,
                   const int64_t *s_new, const uint64_t *a, const int64_t *e, uint64_t *key) {
    if (!gadget_ok(L, K, D)) return -2;
    const int Lp = L + K;
    uint64_t *sn = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    uint64_t *prod = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    if (!sn || !prod) return -1;
    for (int d = 0; d < D; ++d)
        for (int k = 0; k < Lp; ++k) {
            const uint64_t q = primes[k];
            const uint64_t *ad = a + ((int64_t)d * Lp + k) * N;
            uint64_t *ka = key + (((int64_t)d * 2 + 0) * Lp + k) * N;
            uint64_t *kb = key + (((int64_t)d * 2 + 1) * Lp + k) * N;
            for (int64_t c = 0; c < N; ++c) sn[c] = mlift(s_new[c], q);
            if (or_negacyclic_mul(N, ad, sn, prod, q) != 0) return -1;
            uint64_t Pg = 0; /* P * g_d mod q_k */
            if (k >= digit_lo(L, D, d) && k < digit_hi(L, D, d)) {
                Pg = 1;
                for (int t = 0; t < K; ++t) Pg = mmul(Pg, primes[L + t] % q, q);
            }
            for (int64_t c = 0; c < N; ++c) {
                ka[c] = ad[c] % q;
                uint64_t v = msub(mlift(e[(int64_t)d * N + c], q), prod[c], q);
                v = madd(v, mmul(Pg, mlift(s_old[c], q), q), q);
                kb[c] = v;
            }
        }
    free(sn);
    free(prod);
    return 0;
}

/* KeySwitch of ct (L chain planes) with a key of D digits over L+K planes:
 *  1. digit d of the a-part is [a]_{Q_d}, the exact CRT lift of a's residues
 *     on digit d's primes to [0, Q_d), reduced mod every prime of P*Q;
 *  2. u = sum_d digit_d * key_d mod P*Q (both parts);
 *  3. u' = round(u / P) mod Q: r = [u]_P centred in (-P/2, P/2] (the exact
 *     CRT lift of u's special residues), u'_k = (u_k - r) * P^-1 mod q_k;
 *  4. out = (u'_a, b + u'_b).
 * With D = L and K = 1 the digits are the residues a mod q_i themselves. */
int or_keyswitch_g(int64_t N, int L, int K, int D, const uint64_t *primes, const uint64_t *key,
                   const uint64_t *ct, uint64_t *out) {
    if (!gadget_ok(L, K, D)) return -2;
    const int Lp = L + K;
    uint64_t *u = (uint64_t *)calloc((size_t)(2 * Lp * N), sizeof(uint64_t));
    u128 *x = (u128 *)malloc(sizeof(u128) * (size_t)N);
    uint64_t *dk = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    uint64_t *prod = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    if (!u || !x || !dk || !prod) return -1;
    for (int d = 0; d < D; ++d) {
        const int lo = digit_lo(L, D, d), m = digit_hi(L, D, d) - lo;
        for (int64_t c = 0; c < N; ++c) {
            uint64_t r[2];
            for (int j = 0; j < m; ++j) r[j] = ct[(0 * L + lo + j) * N + c]; /* a-part */
            x[c] = crt_lift(m, r, primes + lo, NULL);
        }
        for (int k = 0; k < Lp; ++k) {
            const uint64_t q = primes[k];
            for (int64_t c = 0; c < N; ++c) dk[c] = (uint64_t)(x[c] % q);
            for (int part = 0; part < 2; ++part) {
                const uint64_t *kp = key + (((int64_t)d * 2 + part) * Lp + k) * N;
                if (or_negacyclic_mul(N, dk, kp, prod, q) != 0) return -1;
                uint64_t *up = u + ((int64_t)part * Lp + k) * N;
                for (int64_t c = 0; c < N; ++c) up[c] = madd(up[c], prod[c], q);
            }
        }
    }
    for (int part = 0; part < 2; ++part) {
        for (int64_t c = 0; c < N; ++c) {
            uint64_t r[2];
            for (int t = 0; t < K; ++t) r[t] = u[((int64_t)part * Lp + L + t) * N + c];
            u128 P;
            const u128 uP = crt_lift(K, r, primes + L, &P);
            const int neg = uP > P / 2; /* P odd: centred value uP - P */
            const u128 mag = neg ? P - uP : uP;
            for (int k = 0; k < L; ++k) {
                const uint64_t q = primes[k];
                const uint64_t rk = neg ? mneg((uint64_t)(mag % q), q) : (uint64_t)(mag % q);
                const uint64_t pinv = minv((uint64_t)(P % q), q);
                const uint64_t uk = u[((int64_t)part * Lp + k) * N + c];
                const uint64_t v = mmul(msub(uk, rk, q), pinv, q);
                const uint64_t b = ct[((int64_t)1 * L + k) * N + c];
                out[((int64_t)part * L + k) * N + c] = part == 0 ? v : madd(b % q, v, q);
            }
        }
    }
    free(u);
    free(x);
    free(dk);
    free(prod);
    return 0;
}

/* The gadget of one digit per chain prime and one special prime. */
int or_ks_keygen(int64_t N, int L, const uint64_t *primes, const int64_t *s_old,
                 const int64_t *s_new, const uint64_t *a, const int64_t *e, uint64_t *key) {
    return or_ks_keygen_g(N, L, 1, L, primes, s_old, s_new, a, e, key);
}
int or_keyswitch(int64_t N, int L, const uint64_t *primes, const uint64_t *key, const uint64_t *ct,
                 uint64_t *out) {
    return or_keyswitch_g(N, L, 1, L, primes, key, ct, out);
}

/* Rescale by q_{L-1}: each coefficient x (residues x_0 .. x_{L-1}) becomes
 * round(x / q_{L-1}) = (x - r) / q_{L-1} with r = [x]_{q_{L-1}} centred;
 * in RNS: (x_k - r) * q_{L-1}^-1 mod q_k for k < L-1.  out has L-1 planes. */
void or_rescale(int64_t N, int L, const uint64_t *primes, const uint64_t *ct, uint64_t *out) {
    const uint64_t ql = primes[L - 1];
    for (int part = 0; part < 2; ++part) {
        const uint64_t *xl = ct + ((int64_t)part * L + (L - 1)) * N;
        for (int k = 0; k < L - 1; ++k) {
            const uint64_t q = primes[k];
            const uint64_t inv = minv(ql % q, q);
            const uint64_t *xk = ct + ((int64_t)part * L + k) * N;
            uint64_t *o = out + ((int64_t)part * (L - 1) + k) * N;
            for (int64_t c = 0; c < N; ++c) {
                const int64_t r = xl[c] > ql / 2 ? (int64_t)xl[c] - (int64_t)ql : (int64_t)xl[c];
                o[c] = mmul(msub(xk[c] % q, mlift(r, q), q), inv, q);
            }
        }
    }
}
