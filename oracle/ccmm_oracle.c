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
 *   or_ks_keygen        RNS switching keys (SWKGen, Sec. 2.2, with an RNS gadget)
 *   or_keyswitch        KeySwitch with the same gadget and a special prime
 *   or_rescale          Rescale by the last prime of the RNS chain (Sec. 2.2)
 *
 * Ciphertext layout: ct[part][plane][coef], part 0 = a, part 1 = b; `L`
 * planes, one per prime of the chain q_0 .. q_{L-1}.  Key layout:
 * key[digit][part][plane][coef] with L+1 planes (the special prime P last).
 *
 * RNS gadget (SWKGen with gadget rank L, the decomposition allowed by the
 * footnote of Sec. 2.2): digit i of a ciphertext's a-part is its residue mod
 * q_i.  Key i encrypts P * g_i * s_old under s_new modulo P*Q, where
 * g_i = (Q/q_i) * ((Q/q_i)^-1 mod q_i), so g_i = 1 mod q_i and 0 mod the other
 * q_k.  KeySwitch sums digit_i * key_i over P*Q and divides by P with rounding.
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

/* Switching keys from s_old to s_new modulo P*Q (P = primes[L]).
 * a: [L][L+1][N] uniform residues; e: [L][N] small errors (the randomness).
 * key: [L][2][L+1][N]; part 0 = a_i, part 1 = b_i = -a_i s_new + e_i + P g_i s_old. */
int or_ks_keygen(int64_t N, int L, const uint64_t *primes, const int64_t *s_old,
                 const int64_t *s_new, const uint64_t *a, const int64_t *e, uint64_t *key) {
    const int Lp = L + 1;
    const uint64_t P = primes[L];
    uint64_t *sn = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    uint64_t *prod = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    for (int i = 0; i < L; ++i)
        for (int k = 0; k < Lp; ++k) {
            const uint64_t q = primes[k];
            const uint64_t *ai = a + ((int64_t)i * Lp + k) * N;
            uint64_t *ka = key + (((int64_t)i * 2 + 0) * Lp + k) * N;
            uint64_t *kb = key + (((int64_t)i * 2 + 1) * Lp + k) * N;
            for (int64_t c = 0; c < N; ++c) sn[c] = mlift(s_new[c], q);
            if (or_negacyclic_mul(N, ai, sn, prod, q) != 0) return -1;
            const uint64_t Pg = (k == i) ? P % q : 0; /* P * g_i mod q_k (0 mod P itself) */
            for (int64_t c = 0; c < N; ++c) {
                ka[c] = ai[c] % q;
                uint64_t v = msub(mlift(e[(int64_t)i * N + c], q), prod[c], q);
                v = madd(v, mmul(Pg, mlift(s_old[c], q), q), q);
                kb[c] = v;
            }
        }
    free(sn);
    free(prod);
    return 0;
}

/* KeySwitch of ct (L planes) with key (L+1 planes): digits d_i = a mod q_i,
 * u = sum_i d_i * key_i mod P*Q, then u' = round(u / P) mod Q:
 * r = [u]_P centred in (-P/2, P/2], u'_k = (u_k - r) * P^-1 mod q_k.
 * out = (u'_a, b + u'_b). */
int or_keyswitch(int64_t N, int L, const uint64_t *primes, const uint64_t *key, const uint64_t *ct,
                 uint64_t *out) {
    const int Lp = L + 1;
    const uint64_t P = primes[L];
    uint64_t *u = (uint64_t *)calloc((size_t)(2 * Lp * N), sizeof(uint64_t));
    uint64_t *dk = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    uint64_t *prod = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    if (!u || !dk || !prod) return -1;
    for (int i = 0; i < L; ++i) {
        const uint64_t *di = ct + (0 * L + i) * N; /* residues of a mod q_i, in [0, q_i) */
        for (int k = 0; k < Lp; ++k) {
            const uint64_t q = primes[k];
            for (int64_t c = 0; c < N; ++c) dk[c] = di[c] % q;
            for (int part = 0; part < 2; ++part) {
                const uint64_t *kp = key + (((int64_t)i * 2 + part) * Lp + k) * N;
                if (or_negacyclic_mul(N, dk, kp, prod, q) != 0) return -1;
                uint64_t *up = u + ((int64_t)part * Lp + k) * N;
                for (int64_t c = 0; c < N; ++c) up[c] = madd(up[c], prod[c], q);
            }
        }
    }
    for (int part = 0; part < 2; ++part) {
        const uint64_t *uP = u + ((int64_t)part * Lp + L) * N;
        for (int k = 0; k < L; ++k) {
            const uint64_t q = primes[k];
            const uint64_t pinv = minv(P % q, q);
            const uint64_t *uk = u + ((int64_t)part * Lp + k) * N;
            uint64_t *o = out + ((int64_t)part * L + k) * N;
            const uint64_t *b = ct + ((int64_t)1 * L + k) * N;
            for (int64_t c = 0; c < N; ++c) {
                const int64_t r = uP[c] > P / 2 ? (int64_t)uP[c] - (int64_t)P : (int64_t)uP[c];
                uint64_t v = mmul(msub(uk[c], mlift(r, q), q), pinv, q);
                o[c] = part == 0 ? v : madd(b[c] % q, v, q);
            }
        }
    }
    free(u);
    free(dk);
    free(prod);
    return 0;
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
