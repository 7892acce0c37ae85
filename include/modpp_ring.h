/*
 * modpp_ring.h -- C ABI of the ciphertext-ciphertext matrix product (CC-MM,
 * Alg. 8 of "Fast Homomorphic Linear Algebra with BLAS", arXiv 2503.16080)
 * and the ring operations it is built from: Tweak (Alg. 3), Transpose
 * (Alg. 4), KeySwitch with special primes (Sec. 2.2), and Rescale.
 *
 * Ring and ciphertexts
 * --------------------
 * R_q = Z_q[X]/(X^N + 1), N a power of two, 2 <= N <= 16384.  The RNS chain
 * is q_0 .. q_{L-1} (the ciphertext modulus Q is their product) and key
 * switching uses K special primes p_0 .. p_{K-1} (K = 1 or 2) whose product
 * is P.  Every prime is odd, < 2^62, congruent to 1 mod 2N (the negacyclic
 * NTT needs a primitive 2N-th root of unity), and all L+K primes are
 * distinct.
 *
 * A batch of n ciphertexts is stored part-major, [2][L][n][N] uint64:
 * element ((part * L + j) * n + c) * N + m is coefficient m of part `part`
 * (0 = a, 1 = b) of ciphertext c, modulo q_j, canonical in [0, q_j).  A
 * ciphertext (a, b) decrypts to b + a*s (Sec. 2.2).  For a batch of N
 * ciphertexts the a-part plane j is an N x N matrix whose row c is ciphertext
 * c: the column-wise and row-wise formats of a ciphertext matrix (Sec. 6) are
 * the same storage read along the other axis.
 *
 * Gadget (SWKGen with gadget rank D, the decomposition number of Sec. 2.2's
 * footnote; the paper's experiments use D = 2): the chain primes fall into
 * D digits of alpha = ceil(L / D) consecutive primes (the last digit may be
 * shorter; alpha <= 2), digit d holding q_j for d*alpha <= j <
 * min(L, (d+1)*alpha), with product Q_d.  Switching keys: [D][2][L+K][N]
 * uint64 per key (digit d, part, plane over q_0 .. q_{L-1}, p_0 .. p_{K-1},
 * coefficient).  Key d encrypts P * g_d * s_old under s_new modulo P*Q with
 * g_d = (Q/Q_d) * ((Q/Q_d)^-1 mod Q_d), which is 1 mod the digit's primes and
 * 0 mod the other q_k: key[d][1] = -key[d][0] * s_new + e_d + P * g_d * s_old.
 * KeySwitch of (a, b) computes (round(sum_d [a]_{Q_d} * key[d][0] / P),
 * b + round(sum_d [a]_{Q_d} * key[d][1] / P)), [a]_{Q_d} the exact lift of
 * a's residues on the digit's primes to [0, Q_d), with the division by P
 * rounded as x -> (x - [x]_P) / P, [x]_P centred in (-P/2, P/2].  The
 * default ring (modpp_ring_create) has D = L one-prime digits and K = 1.
 * Keys are generated outside the library (the server never sees secrets)
 * and converted once, in place, by modpp_ring_prepare_keys.
 *
 * Conventions are those of modpp.h: device pointers owned by the caller,
 * asynchronous calls on `stream`, host-side argument checks returning a
 * negative modpp_status before anything is enqueued, caller workspaces
 * (256-byte aligned) sized by the *_workspace queries, no device allocation
 * on the call path, outputs that do not overlap inputs unless stated.
 * Ciphertext, key and output pointers must be 16-byte aligned (the kernels
 * move neighbouring coefficient pairs in 16-byte accesses); a misaligned
 * pointer returns MODPP_ERR_ARG before anything is enqueued.
 */
#ifndef MODPP_RING_H
#define MODPP_RING_H

#include "modpp.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct modpp_ring_s *modpp_ring;

/* Device bytes of the ring tables for degree N, L chain primes, K special
 * primes and D = dnum gadget digits (0 for invalid sizes); modpp_ring_bytes
 * is the same with K = 1, D = L. */
size_t modpp_ring_bytes_ks(int64_t N, int L, int K, int dnum);
size_t modpp_ring_bytes(int64_t N, int L);

/*
 * Writes the NTT tables (powers of a primitive 2N-th root psi of every
 * prime in bit-reversed order and their Shoup quotients), the RNS constants
 * (P^-1 mod q_k, q_{L-1}^-1 mod q_k, N^-1 mod q_k) and the index tables of
 * Alg. 4, and the gadget's constants (Garner's lift of two-prime digits,
 * the CRT lift of [x]_P for two special primes) into `mem` (device,
 * modpp_ring_bytes_ks(N, L, K, dnum) bytes, owned by the caller and kept
 * alive until modpp_ring_destroy), and returns a host handle in *ring.
 * primes_host: L+K primes, the chain q_0 .. q_{L-1} then the special primes.
 * 1 <= L <= 16, K in {1, 2}, 1 <= dnum <= L with ceil(L / dnum) <= 2 and
 * every digit non-empty.  Synchronises `stream` once (the tables are copied
 * from host memory).  Errors: MODPP_ERR_ARG (sizes, gadget, null pointers),
 * MODPP_ERR_PRIME (a prime that is even, >= 2^62, not 1 mod 2N, or
 * repeated), MODPP_ERR_WORKSPACE (mem too small or misaligned),
 * MODPP_ERR_CUDA.  modpp_ring_create is the same with K = 1 and dnum = L
 * (primes_host: L+1 primes, the chain then P).
 */
int modpp_ring_create_ks(int64_t N, int L, int K, int dnum, const uint64_t *primes_host, void *mem,
                         size_t mem_bytes, void *stream, modpp_ring *ring);
int modpp_ring_create(int64_t N, int L, const uint64_t *primes_host, void *mem, size_t mem_bytes,
                      void *stream, modpp_ring *ring);
int modpp_ring_destroy(modpp_ring ring);

/*
 * Converts `count` switching keys ([count][D][2][L+K][N], contiguous) in
 * place from coefficients to the form the key-switching kernels read: the
 * negacyclic NTT of every polynomial, multiplied by 2^64 mod its prime
 * (Montgomery form).  Apply once per key; the other calls take prepared keys.
 */
int modpp_ring_prepare_keys(modpp_ring ring, uint64_t *keys, int64_t count, void *stream);

/*
 * KeySwitch (Sec. 2.2) of a batch of n ciphertexts with one prepared key:
 * out = KeySwitch(ct).  ct and out are [2][L][n][N]; out may equal ct.
 */
size_t modpp_keyswitch_workspace(modpp_ring ring, int64_t n);
int modpp_keyswitch(modpp_ring ring, const uint64_t *ct, uint64_t *out, int64_t n,
                    const uint64_t *key, void *ws, size_t ws_bytes, void *stream);

/*
 * KeySwitch (Sec. 2.2) of a batch of n ciphertexts, each with its own key:
 * ciphertext c is switched with keys[key_index[c]] (prepared keys,
 * [count][D][2][L+K][N]); key_index[c] < 0 copies ciphertext c unchanged.
 * This is the key switch that follows each automorphism in Alg. 4 (steps
 * 2-5), where ciphertext j needs the key of s(X^(2j+1)) -> s.
 *   key_index  DEVICE array of n int32, read by the kernels; every
 *              non-negative entry must be a valid key index (not checked).
 * Workspace: modpp_keyswitch_workspace(ring, n).  out may equal ct.
 * n = 1 runs the single-key kernel; n >= 2 the streaming key-product kernels
 * that modpp_transpose uses.
 */
int modpp_keyswitch_indexed(modpp_ring ring, const uint64_t *ct, uint64_t *out, int64_t n,
                            const uint64_t *keys, const int *key_index, void *ws, size_t ws_bytes,
                            void *stream);

/*
 * Tweak (Alg. 3): out_j = sum_{i<n} X^(2 i j N / n) * ct_i for a batch of n
 * ciphertexts, n a power of two dividing 2N (an n-point DFT over R_q with
 * root X^(2N/n)), computed by log2(n) radix-2 stages.  [2][L][n][N]; out must
 * not overlap ct.
 */
size_t modpp_tweak_workspace(modpp_ring ring, int64_t n);
int modpp_tweak(modpp_ring ring, const uint64_t *ct, uint64_t *out, int64_t n, void *ws,
                size_t ws_bytes, void *stream);

/*
 * Transpose (Alg. 4) of `groups` independent ciphertext matrices, each N
 * ciphertexts (a batch of groups * N ciphertexts, [2][L][groups*N][N]):
 * turns an encryption of the rows of an N x N matrix into one of its columns
 * and conversely.  aut_keys: N prepared keys, key j switching
 * s(X^(2j+1)) -> s (key 0 is never read).  The last step (j = N of the
 * algorithm, column 0) is taken as ct'_0 = +ct''_0: the trace identity
 * behind the others, -Tr(X^j m)/N = m_{N-j}, holds for 1 <= j < N only.
 * out must not overlap ct.
 */
size_t modpp_transpose_workspace(modpp_ring ring, int64_t groups);
int modpp_transpose(modpp_ring ring, const uint64_t *ct, uint64_t *out, int64_t groups,
                    const uint64_t *aut_keys, void *ws, size_t ws_bytes, void *stream);

/*
 * Rescale by the last chain prime: x -> round(x / q_{L-1}) on every
 * coefficient, [2][L][n][N] -> [2][L-1][n][N].  Needs L >= 2.
 */
int modpp_rescale(modpp_ring ring, const uint64_t *ct, uint64_t *out, int64_t n, void *stream);

/*
 * CC-MM (Alg. 8).  ct1, ct2: column-wise encryptions of two N x N matrices
 * (ciphertext j encrypts column j), [2][L][N][N].  Computes
 *   1. the row-wise encryption of M2 by Transpose,
 *   2. C = [A; B] * [A~' B~'] mod q_j for every prime: the four N x N blocks
 *      C00, C01, C10, C11, as two Mod-PP-MMs of residue matrices
 *      (modpp_mm_wide),
 *   3-4. Transpose((C00, 0)) = (D0, D1) and Transpose((C10, 0)) = (D2, D3)
 *      as one batch of two matrices,
 *   5. Relin(D0, 0) + (D1 + D2 + C01, D3 + C11) with column j of C01 and C11
 *      added to ciphertext j, then Rescale by q_{L-1}.
 * out: [2][L-1][N][N], the column-wise encryption of M1 * M2 at scale
 * Delta^2 / q_{L-1}.  aut_keys as modpp_transpose; relin_key: one prepared
 * key switching s^2 -> s.  Needs L >= 2.
 */
size_t cc_mm_workspace(modpp_ring ring);
int cc_mm(modpp_ring ring, const uint64_t *ct1, const uint64_t *ct2, const uint64_t *aut_keys,
          const uint64_t *relin_key, uint64_t *out, void *ws, size_t ws_bytes, void *stream);

/*
 * CC-MM with a choice of encoding for the right operand (the remark on row
 * or column encodings after Thm th:ccmm, Sec. 5):
 *   flags = 0: as cc_mm; n must equal N.
 *   flags = MODPP_CC_M2_ROWWISE: ct2 is a ROW-wise encryption of an n x N
 *     matrix M2 (ciphertext t encrypts row t; [2][L][n][N]) and ct1 the
 *     column-wise encryption of an N x n matrix M1 (ciphertext j encrypts
 *     column j; [2][L][n][N]), 1 <= n <= N.  Step 1 of Alg. 8 (the
 *     Transpose of ct2) is skipped: two Transposes instead of three, and the
 *     wide products have inner dimension n.
 * out: [2][L-1][N][N], the column-wise encryption of M1 * M2 (N x N).
 * out_scale_mult (host, may be null) receives 1 / q_{L-1}: the output's
 * scale is the product of the inputs' scales times this factor (Delta^2 /
 * q_{L-1} for two inputs at scale Delta).  Workspace: cc_mm_ex_workspace
 * (0 for an invalid n or flags).  Other conventions as cc_mm.
 */
#define MODPP_CC_M2_ROWWISE 1
size_t cc_mm_ex_workspace(modpp_ring ring, int64_t n, int flags);
int cc_mm_ex(modpp_ring ring, int64_t n, const uint64_t *ct1, const uint64_t *ct2,
             const uint64_t *aut_keys, const uint64_t *relin_key, int flags, uint64_t *out,
             double *out_scale_mult, void *ws, size_t ws_bytes, void *stream);

/*
 * CP-MM with precomputation (Alg. 7, Thm th:pcmm-with-precomp), followed by
 * the key switches back to one secret (before the optional Rescale, the
 * order the remark after Thm th:pcmm-with-precomp recommends for precision).
 *
 * Input: a shared-a encryption of an N x d2 matrix M: d2 ciphertexts
 * (a, b_j) with ONE common a-part, ciphertext j encrypting column j of M
 * under its own secret s_j (column j of S): Toep(a) * S + B = Delta M + E.
 * U (d2 x d3, int8) is the plaintext known beforehand; key k (prepared)
 * switches s'_k = sum_j U[j][k] s_j (column k of S * U) to the target
 * secret s -- the precomputation of Alg. 7.
 *   1. B' = B * U mod q_j: ONE Mod-PP-MM per chain prime (Alg. 6 needs two);
 *      (a, column k of B') encrypts column k of M * U under s'_k.
 *   2. KeySwitch of (a, b'_k) with key k for every k < d3.  The a-part is
 *      shared, so its digits and their forward transforms are computed once
 *      for the whole batch.
 *   3. with MODPP_PRECOMP_RESCALE: Rescale by q_{L-1}.
 *   Ut    d3 x d2 int8, contiguous: row k is column k of U.
 *   a     [L][N], the shared a-part.
 *   B     [L][d2][N]: the b-parts, row j = b_j (the b-part planes of a batch).
 *   keys  [d3][D][2][L+K][N], prepared (modpp_ring_prepare_keys).
 *   out   [2][L][d3][N] (with Rescale: [2][L-1][d3][N]): ciphertext k
 *         encrypts column k of M * U under s (at scale Delta * scale(U),
 *         divided by q_{L-1} with Rescale).
 * 1 <= d2 <= 2^20, 1 <= d3 < 2^31.  Workspace: pc_mm_precomp_workspace.
 */
#define MODPP_PRECOMP_RESCALE 1
size_t pc_mm_precomp_workspace(modpp_ring ring, int64_t d2, int64_t d3, int flags);
int pc_mm_precomp(modpp_ring ring, int64_t d2, int64_t d3, const int8_t *Ut, const uint64_t *a,
                  const uint64_t *B, const uint64_t *keys, int flags, uint64_t *out, void *ws,
                  size_t ws_bytes, void *stream);

/*
 * Waits for `stream`, then reads and clears the ring's status word (a word
 * in the ring's table memory): MODPP_OK, or MODPP_ERR_RANGE when, in debug
 * mode (modpp_set_debug_checks), an entry point of this ring was given a
 * ciphertext coefficient or key coefficient not below its prime since the
 * last read.  The word is sticky until read.  Device waits of the wide
 * products inside cc_mm report in the status word at the start of cc_mm's
 * workspace (modpp_status_read).
 */
int modpp_ring_status_read(modpp_ring ring, void *stream);

/* Device time (ms) of the stages of the last cc_mm call on this ring, when
 * timing is switched on with modpp_profile_enable(1); stage 0 = transpose of
 * ct2, 1 = the two Mod-PP-MMs, 2 = transpose of C00 | C10, 3 = relin and
 * finish.  Synchronises with the events of the last call. */
int cc_mm_stage_ms(modpp_ring ring, double ms[4]);

#ifdef __cplusplus
}
#endif

#endif /* MODPP_RING_H */
