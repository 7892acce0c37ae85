// Internal declarations of the ring kernels (NTT, automorphism, key
// switching, Tweak stages, Rescale) used by the ciphertext-ciphertext product.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace modpp {

// Per-prime constants and tables of the negacyclic NTT of degree N.
struct NttPlane {
    uint64_t q;
    uint64_t mu;        // floor(2^64 / q), Barrett
    uint64_t qinv_neg;  // -q^-1 mod 2^64, Montgomery
    uint64_t ninv, ninv_s;  // N^-1 mod q and its Shoup quotient
    uint64_t r64, r64_s;    // 2^64 mod q (Montgomery form factor) and its Shoup quotient
    const uint64_t *fwd;    // psi^bitrev(i), i < N
    const uint64_t *fwd_s;
    const uint64_t *inv;    // psi^-bitrev(i)
    const uint64_t *inv_s;
    const ulonglong2 *fwd2; // (fwd[i], fwd_s[i]) pairs: one 16-byte load per twiddle
    const ulonglong2 *inv2;
};

// Gadget of the ring's key switching (SWKGen with gadget rank D, Sec. 2.2):
// the L chain primes fall into D digits of at most two consecutive primes
// (digit d: primes d * alpha .. min(L, (d + 1) * alpha) - 1), and K <= 2
// special primes, whose product is P, follow the chain (planes L .. L+K-1).
// Digit d of an a-part is its residue modulo the product Q_d of the digit's
// primes.  Switching keys: [count][D][2][L+K][N].  Device pointers point into
// the ring's tables.
constexpr int kMaxGadgetDigits = 16;
struct KsGadget {
    int L, K, D, alpha;
    uint64_t chain_max;  // largest chain prime: bound of an unreduced one-prime digit
    // ModUp of a two-prime digit (primes j0 and j1 = j0 + 1): the digit is
    // the integer v0 + q_j0 * v1 in [0, q_j0 q_j1), v0 = a_j0 and
    // v1 = (a_j1 - v0) * q_j0^-1 mod q_j1 (Garner's mixed radix).
    uint64_t ginv[kMaxGadgetDigits], ginv_s[kMaxGadgetDigits];  // q_j0^-1 mod q_j1, Shoup quotient
    const uint64_t *cq, *cq_s;                      // [D][L+K]: q_j0 mod q_k, Shoup quotient
    // ModDown with two special primes p0, p1: [u]_P = v0 + p0 * v1 with
    // v0 = u mod p0, v1 = (u_p1 - v0) * p0^-1 mod p1; the centred value is
    // [u]_P - P when (v1, v0) >= (m1, h0) lexicographically, i.e. when
    // [u]_P >= (P + 1) / 2 = h0 + p0 * m1.
    uint64_t p0inv, p0inv_s, m1, h0;
    const uint64_t *p0k, *p0k_s;  // [L]: p0 mod q_k, Shoup quotient
    const uint64_t *Pk;           // [L]: P mod q_k
};

// Per-ciphertext tables of a gather: every table has period `per` over the
// batch (ciphertext c reads entry c mod per; source indices are relative to
// the period block of c, and per is a power of two).  Null tables mean
// identity source and ell 1.
struct GatherTables {
    const int *src;
    const int *ellinv;        // ell^-1 mod 2N of the automorphism, or null (ell = 1)
    const uint64_t *scale;    // per plane, or null
    const uint64_t *scale_s;
    int per;
};

// Negacyclic NTT of npolys polynomials in place; polynomial p uses the
// tables of plane (p / inner) % nplanes.  N >= 1024 runs the register-blocked
// kernel of ntt_kernels.cu, smaller N the per-stage kernel.
cudaError_t launch_ntt(uint64_t *polys, int64_t npolys, int N, int64_t inner, int nplanes,
                       const NttPlane *tab, bool inverse, cudaStream_t s);
bool ntt_fast_supported(int N);
cudaError_t launch_ntt_fast(uint64_t *polys, int64_t npolys, int N, int64_t inner, int nplanes,
                            const NttPlane *tab, bool inverse, cudaStream_t s);
// Garner digits of the two-prime gadget digits of ciphertexts [c0, c0 + nb):
// V[c][d][m] = (a_j1 - a_j0) * q_j0^-1 mod q_j1 at coefficient m (rows of
// one-prime digits are left untouched).  Every digit source below takes V
// (null when every digit has one prime).
cudaError_t launch_ks_garner(const uint64_t *ct, int64_t n, int N, int64_t c0, int64_t nb,
                             const NttPlane *tab, const KsGadget &g, uint64_t *V, cudaStream_t s);
// Key switching's digits, NTTs, key products and inverse NTTs in one kernel
// (1024 <= N <= 8192): U[c][part][k] = sum_d digit_d * key_d[part] mod q_k
// (coefficients), k < L + K.
bool ks_fused_supported(int N);
cudaError_t launch_ks_fused(const uint64_t *ct, int64_t n, int N, int64_t c0, int64_t nb,
                            const NttPlane *tab, const KsGadget &g, const uint64_t *V,
                            const uint64_t *keys, const int *kid, int kper, uint64_t *U,
                            cudaStream_t s);
// Digits of key switching fused with their forward NTT (N >= 1024):
// D[c][d][k] = NTT_k(digit d of the a-part of ciphertext c0 + c, mod q_k), c < nb.
cudaError_t launch_ks_digits_ntt(const uint64_t *ct, int64_t n, int N, int64_t c0, int64_t nb,
                                 const NttPlane *tab, const KsGadget &g, const uint64_t *V,
                                 uint64_t *D, cudaStream_t s);
cudaError_t launch_to_montgomery(uint64_t *polys, int64_t npolys, int N, int64_t inner,
                                 int nplanes, const NttPlane *tab, cudaStream_t s);
// The digits alone (coefficients), D[c][d][k] as above.
cudaError_t launch_ks_decompose(const uint64_t *ct, int64_t n, int N, int64_t c0, int64_t nb,
                                const NttPlane *tab, const KsGadget &g, const uint64_t *V,
                                uint64_t *D, cudaStream_t s);
// kid null: ciphertext c takes key c.  d_shared: one set of digits D[0] for
// every ciphertext (a batch sharing one a-part).
cudaError_t launch_ks_multacc(const uint64_t *D, const uint64_t *keys, const int *kid, int kper,
                              const KsGadget &g, int N, int64_t c0, int64_t nb,
                              const NttPlane *tab, uint64_t *U, cudaStream_t s,
                              int d_shared = 0);
// Writes ciphertext c0 + c of the chunk to plane stride n_out of `out`; kid
// null: no ciphertext is copied unchanged.  pinv: P^-1 mod q_k (Shoup).
cudaError_t launch_ks_moddown(const uint64_t *U, const uint64_t *ct, int64_t n, int N, int64_t c0,
                              int64_t nb, const int *kid, int kper, int b_zero,
                              const NttPlane *tab, const KsGadget &g, const uint64_t *pinv,
                              const uint64_t *pinv_s, uint64_t *out, int64_t n_out,
                              cudaStream_t s);
// parts = 2: both parts of every ciphertext; 1: the a-parts only.
cudaError_t launch_ct_gather(const uint64_t *in, uint64_t *out, int64_t n, int L, int N,
                             const GatherTables &t, const NttPlane *tab, cudaStream_t s,
                             int parts = 2);
// Input and output maps of a Tweak pass, folding the gathers around the
// Tweaks of Alg. 4 into the first and last passes:
//   in_bits > 0: input ciphertext i of each group of 2^in_bits is read from
//     the bit-reversed index si of the group, times X^si when in_shift
//     (Alg. 4 step 1: aux = Tweak((X^i ct_i)_i) with the stages' input in
//     bit-reversed order);
//   out_t3: output ciphertext i of each group of N is written as ciphertext
//     (N - i) mod N times X^(N + i) for i > 0 (Alg. 4 steps 7-9:
//     ct'_j = X^(2N - j) ct''_(N - j), ct'_0 = ct''_0).
struct TweakMap {
    int in_bits = 0;
    int in_shift = 0;
    int out_t3 = 0;
};
cudaError_t launch_tweak_stage(const uint64_t *in, uint64_t *out, int64_t n, int L, int N,
                               int64_t half, const NttPlane *tab, cudaStream_t s, int parts = 2,
                               const TweakMap &mp = TweakMap{});
// Stages half and 2 half in one pass (4 half <= N, n a multiple of 4 half).
cudaError_t launch_tweak_radix4(const uint64_t *in, uint64_t *out, int64_t n, int L, int N,
                                int64_t half, const NttPlane *tab, cudaStream_t s, int parts = 2,
                                const TweakMap &mp = TweakMap{});
// Stages half, 2 half and 4 half in one pass (8 half <= N, n a multiple of 8 half).
cudaError_t launch_tweak_radix8(const uint64_t *in, uint64_t *out, int64_t n, int L, int N,
                                int64_t half, const NttPlane *tab, cudaStream_t s, int parts = 2,
                                const TweakMap &mp = TweakMap{});
cudaError_t launch_add_planes(const uint64_t *x, const uint64_t *y, uint64_t *out, int parts, int L,
                              int64_t count, const NttPlane *tab, cudaStream_t s);
cudaError_t launch_rescale(const uint64_t *in, uint64_t *out, int L, int64_t count,
                           const NttPlane *tab, const uint64_t *qlinv, const uint64_t *qlinv_s,
                           cudaStream_t s);
cudaError_t launch_transpose_u64(const uint64_t *in, uint64_t *out, int rows, int cols,
                                 int64_t ldi, int64_t ldo, int64_t si, int64_t so, int mats,
                                 cudaStream_t s);
// Last step of Alg. 8 fused with Rescale; see ring_kernels.cu.
struct CcFinishParams {
    const uint64_t *R;  // relinearised D0: [2][L][N][N]
    const uint64_t *Z;  // transposed (C00 | C10) batch: [2][L][2N][N]
    const uint64_t *Y;  // [C01; C11] per prime: [L][2N][N]
    uint64_t *out;      // [2][L-1][N][N]
    int L, N;
    const NttPlane *tab;
    const uint64_t *qlinv, *qlinv_s;
};
cudaError_t launch_cc_finish(const CcFinishParams &p, cudaStream_t s);

}  // namespace modpp
