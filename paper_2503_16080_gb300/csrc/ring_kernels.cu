// Ring kernels of the ciphertext-ciphertext product (Alg. 8): negacyclic NTT,
// automorphisms, RNS key switching, Tweak (Alg. 3) stages, the gathers of
// Transpose (Alg. 4), Rescale, and u64 matrix transposes.
//
// Ciphertext batches use the part-major layout [2][planes][n][N]: part 0 is
// the a-part, part 1 the b-part; polynomial (part, plane, c) holds the N
// coefficients of ciphertext c modulo prime `plane`.  All residues are
// canonical in [0, q).
//
// NTT: negacyclic transform of Z_q[X]/(X^N+1) by the Cooley-Tukey (forward)
// and Gentleman-Sande (inverse) butterflies with the powers of a primitive
// 2N-th root psi in bit-reversed order (Longa and Naehrig, "Speeding up the
// Number Theoretic Transform for Faster Ideal Lattice-Based Cryptography",
// CANS 2016).  Products are pointwise in the transformed domain.
//
// Key-switching keys are kept in the transformed domain and in Montgomery
// form (x * 2^64 mod q), so a product with a transformed digit is one
// Montgomery reduction (P. Montgomery, Math. Comp. 1985).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "modarith.cuh"
#include "ks_gadget.cuh"
#include "ring_internal.h"

namespace modpp {

// ------------------------------------------------------------ arithmetic

// ------------------------------------------------------------ NTT
// One CTA transforms one polynomial in shared memory, one barrier per stage
// (the transform for N < 1024; larger N use ntt_kernels.cu).  Polynomial p
// uses the tables of plane (p / inner) % nplanes.
__global__ void __launch_bounds__(512) ntt_kernel(uint64_t *polys, int N, int logN, int64_t inner,
                                                  int nplanes, const NttPlane *__restrict__ tab,
                                                  int inverse) {
    extern __shared__ uint64_t sa[];
    const int64_t p = blockIdx.x;
    const int plane = static_cast<int>((p / inner) % nplanes);
    const NttPlane tp = tab[plane];
    uint64_t *g = polys + p * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) sa[i] = g[i];
    __syncthreads();
    const uint64_t q = tp.q;
    const int half = N >> 1;
    if (!inverse) {
        int t = N;
        for (int m = 1; m < N; m <<= 1) {
            t >>= 1;
            for (int b = threadIdx.x; b < half; b += blockDim.x) {
                const int i = b / t, jj = b - (b / t) * t;
                const int j = 2 * i * t + jj;
                const uint64_t S = tp.fwd[m + i], Ss = tp.fwd_s[m + i];
                const uint64_t U = sa[j];
                const uint64_t V = shoup_mulmod(sa[j + t], S, Ss, q);
                sa[j] = add_mod(U, V, q);
                sa[j + t] = sub_mod(U, V, q);
            }
            __syncthreads();
        }
        for (int i = threadIdx.x; i < N; i += blockDim.x) g[i] = sa[i];
    } else {
        int t = 1;
        for (int m = N; m > 1; m >>= 1) {
            const int h = m >> 1;
            for (int b = threadIdx.x; b < half; b += blockDim.x) {
                const int i = b / t, jj = b - (b / t) * t;
                const int j = 2 * i * t + jj;
                const uint64_t S = tp.inv[h + i], Ss = tp.inv_s[h + i];
                const uint64_t U = sa[j], V = sa[j + t];
                sa[j] = add_mod(U, V, q);
                sa[j + t] = shoup_mulmod(sub_mod(U, V, q), S, Ss, q);
            }
            t <<= 1;
            __syncthreads();
        }
        for (int i = threadIdx.x; i < N; i += blockDim.x)
            g[i] = shoup_mulmod(sa[i], tp.ninv, tp.ninv_s, q);
    }
}

cudaError_t launch_ntt(uint64_t *polys, int64_t npolys, int N, int64_t inner, int nplanes,
                       const NttPlane *tab, bool inverse, cudaStream_t s) {
    if (npolys == 0) return cudaSuccess;
    if (ntt_fast_supported(N)) return launch_ntt_fast(polys, npolys, N, inner, nplanes, tab, inverse, s);
    int logN = 0;
    while ((1 << logN) < N) ++logN;
    const size_t smem = static_cast<size_t>(N) * 8;
    cudaError_t e = cudaFuncSetAttribute(ntt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int threads = N >= 1024 ? 512 : (N / 2 > 32 ? N / 2 : 32);
    ntt_kernel<<<static_cast<unsigned>(npolys), threads, smem, s>>>(polys, N, logN, inner, nplanes,
                                                                   tab, inverse ? 1 : 0);
    return cudaGetLastError();
}

// Keys to the evaluation domain in Montgomery form: x -> NTT(x) * 2^64 mod q.
__global__ void to_montgomery_kernel(uint64_t *polys, int64_t npolys, int N, int64_t inner,
                                     int nplanes, const NttPlane *__restrict__ tab) {
    const int64_t total = npolys * N;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t p = i / N;
        const NttPlane &tp = tab[(p / inner) % nplanes];
        polys[i] = shoup_mulmod(polys[i], tp.r64, tp.r64_s, tp.q);
    }
}

cudaError_t launch_to_montgomery(uint64_t *polys, int64_t npolys, int N, int64_t inner,
                                 int nplanes, const NttPlane *tab, cudaStream_t s) {
    if (npolys == 0) return cudaSuccess;
    to_montgomery_kernel<<<152 * 16, 256, 0, s>>>(polys, npolys, N, inner, nplanes, tab);
    return cudaGetLastError();
}

// ------------------------------------------------------------ key switching
// Digits of the a-parts of ciphertexts [c0, c0 + nb) (planes 0..L-1 of a
// batch [2][L][n][N]): D[c][d][k] = (digit d of the a-part of ciphertext c)
// mod q_k, k < L + K (ModUp: the digit's exact residue modulo Q_d).
__global__ void ks_garner_kernel(const uint64_t *__restrict__ ct, int64_t n, int logN, int64_t c0,
                                 int64_t nb, const NttPlane *__restrict__ tab, KsGadget g,
                                 uint64_t *__restrict__ V) {
    const int N = 1 << logN;
    const int64_t total = (nb * g.D) << logN;
    for (int64_t x = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; x < total;
         x += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int m = static_cast<int>(x) & (N - 1);
        const int64_t r = x >> logN;
        const int d = static_cast<int>(r % g.D);
        if (gadget_count(g, d) != 2) continue;
        const int64_t c = r / g.D;
        const uint64_t *a0 = ct + (static_cast<int64_t>(gadget_lo(g, d)) * n + c0 + c) * N + m;
        V[x] = garner_v1(g, tab, d, a0[0], a0[n * N]);
    }
}

__global__ void ks_decompose_kernel(const uint64_t *__restrict__ ct, int64_t n, int N, int64_t c0,
                                    int64_t nb, const NttPlane *__restrict__ tab, KsGadget g,
                                    const uint64_t *__restrict__ V, uint64_t *__restrict__ D) {
    const int Lp = g.L + g.K;
    const int64_t total = nb * g.D * Lp * static_cast<int64_t>(N);
    for (int64_t x = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; x < total;
         x += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int m = static_cast<int>(x % N);
        int64_t r = x / N;
        const int k = static_cast<int>(r % Lp);
        r /= Lp;
        const int d = static_cast<int>(r % g.D);
        const int64_t c = r / g.D;
        const uint64_t *a0 = ct + (static_cast<int64_t>(gadget_lo(g, d)) * n + c0 + c) * N;
        const DigitSrc s = make_digit_src(g, a0, V ? V + (c * g.D + d) * N : nullptr, d, k);
        D[x] = digit_at(s, m, tab[k].q, tab[k].mu, true);
    }
}

// U[c][part][k] = sum_d D[c][d][k] * key[kid(c)][d][part][k] in the
// evaluation domain (keys in Montgomery form, digits plain: the product is
// plain), k < L + K.  kid null: ciphertext c0 + c takes key c0 + c.
// d_shared: every ciphertext shares the digits D[0] (one a-part for the
// whole batch).  nb * (L + K) < 2^31 and N = 2^logN.
__global__ void ks_multacc_kernel(const uint64_t *__restrict__ D, const uint64_t *__restrict__ keys,
                                  const int *__restrict__ kid, int kper, int Dg, int Lp, int logN,
                                  int64_t c0, int64_t nb, const NttPlane *__restrict__ tab,
                                  uint64_t *__restrict__ U, int d_shared) {
    // Two neighbouring coefficients per thread (16-byte accesses).
    const int N = 1 << logN;
    const int64_t key_stride = static_cast<int64_t>(Dg) * 2 * Lp << logN;
    const int64_t total = (nb * Lp) << (logN - 1);
    for (int64_t x = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; x < total;
         x += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int m = (static_cast<int>(x) << 1) & (N - 1);
        const int r = static_cast<int>(x >> (logN - 1));
        const int k = r % Lp;
        const int c = r / Lp;
        const int kc = kid ? kid[(c0 + c) % kper] : static_cast<int>(c0 + c);
        if (kc < 0) continue;
        const uint64_t q = tab[k].q, qinv = tab[k].qinv_neg;
        const uint64_t *key = keys + kc * key_stride + (static_cast<int64_t>(k) << logN) + m;
        const uint64_t *d =
            D + ((static_cast<int64_t>(d_shared ? 0 : c) * Dg * Lp + k) << logN) + m;
        const int64_t dstep = static_cast<int64_t>(Lp) << logN;     // next digit
        const int64_t kstep = static_cast<int64_t>(2 * Lp) << logN; // next key digit
        const int64_t kpart = static_cast<int64_t>(Lp) << logN;     // part 1 of a key digit
        ulonglong2 u0 = make_ulonglong2(0, 0), u1 = make_ulonglong2(0, 0);
        for (int i = 0; i < Dg; ++i) {
            const ulonglong2 di = *reinterpret_cast<const ulonglong2 *>(d + i * dstep);
            const ulonglong2 k0 = *reinterpret_cast<const ulonglong2 *>(key + i * kstep);
            const ulonglong2 k1 = *reinterpret_cast<const ulonglong2 *>(key + i * kstep + kpart);
            u0.x = add_mod(u0.x, mont_mul(di.x, k0.x, q, qinv), q);
            u0.y = add_mod(u0.y, mont_mul(di.y, k0.y, q, qinv), q);
            u1.x = add_mod(u1.x, mont_mul(di.x, k1.x, q, qinv), q);
            u1.y = add_mod(u1.y, mont_mul(di.y, k1.y, q, qinv), q);
        }
        uint64_t *u = U + ((static_cast<int64_t>(c) * 2 * Lp + k) << logN) + m;
        *reinterpret_cast<ulonglong2 *>(u) = u0;
        *reinterpret_cast<ulonglong2 *>(u + kpart) = u1;
    }
}

// ModDown by P and accumulation: out_a = round(U_a / P), out_b = b + round(U_b / P),
// with round(x / P) = (x_k - r) * P^-1 mod q_k, r = [x]_P centred (the CRT
// lift of x's special residues, ks_gadget.cuh).  Ciphertexts with kid < 0 are
// copied unchanged.  With b_zero the input b-part is taken as 0 (Relin(D0, 0)
// in Alg. 8).  One thread takes two neighbouring coefficients of one
// (ciphertext, part) for every chain prime, so the special planes are read
// once.
__global__ void ks_moddown_kernel(const uint64_t *__restrict__ U, const uint64_t *__restrict__ ct,
                                  int64_t n, int logN, int64_t c0, int64_t nb,
                                  const int *__restrict__ kid, int kper, int b_zero,
                                  const NttPlane *__restrict__ tab, KsGadget g,
                                  const uint64_t *__restrict__ pinv,
                                  const uint64_t *__restrict__ pinv_s, uint64_t *__restrict__ out,
                                  int64_t n_out) {
    const int L = g.L, Lp = g.L + g.K;
    const int N = 1 << logN;
    const int part = blockIdx.y;
    const int64_t total = nb << (logN - 1);
    for (int64_t x = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; x < total;
         x += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int m = (static_cast<int>(x) << 1) & (N - 1);
        const int64_t c = x >> (logN - 1);
        const bool copy = kid != nullptr && kid[(c0 + c) % kper] < 0;
        const int64_t ub = ((c * 2 + part) * Lp) << logN;
        CentredP rx{}, ry{};
        if (!copy) {
            const ulonglong2 u0 =
                *reinterpret_cast<const ulonglong2 *>(U + ub + (static_cast<int64_t>(L) << logN) + m);
            ulonglong2 u1 = make_ulonglong2(0, 0);
            if (g.K == 2)
                u1 = *reinterpret_cast<const ulonglong2 *>(
                    U + ub + (static_cast<int64_t>(L + 1) << logN) + m);
            rx = centred_p_digits(g, tab, u0.x, u1.x);
            ry = centred_p_digits(g, tab, u0.y, u1.y);
        }
        for (int k = 0; k < L; ++k) {
            const int64_t io = ((static_cast<int64_t>(part) * L + k) * n + c0 + c) * N + m;
            const int64_t oo = ((static_cast<int64_t>(part) * L + k) * n_out + c0 + c) * N + m;
            ulonglong2 v;
            if (copy) {
                v = (part == 1 && b_zero) ? make_ulonglong2(0, 0)
                                          : *reinterpret_cast<const ulonglong2 *>(ct + io);
            } else {
                const uint64_t q = tab[k].q, pv = pinv[k], pvs = pinv_s[k];
                const ulonglong2 uk =
                    *reinterpret_cast<const ulonglong2 *>(U + ub + (static_cast<int64_t>(k) << logN) + m);
                v.x = shoup_mulmod(sub_mod(uk.x, centred_p_mod(g, tab, rx, k), q), pv, pvs, q);
                v.y = shoup_mulmod(sub_mod(uk.y, centred_p_mod(g, tab, ry, k), q), pv, pvs, q);
                if (part == 1 && !b_zero) {
                    const ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(ct + io);
                    v.x = add_mod(b.x, v.x, q);
                    v.y = add_mod(b.y, v.y, q);
                }
            }
            *reinterpret_cast<ulonglong2 *>(out + oo) = v;
        }
    }
}

cudaError_t launch_ks_garner(const uint64_t *ct, int64_t n, int N, int64_t c0, int64_t nb,
                             const NttPlane *tab, const KsGadget &g, uint64_t *V, cudaStream_t s) {
    if (nb == 0) return cudaSuccess;
    const int64_t bx = std::min<int64_t>((nb * g.D * N + 255) / 256, 152 * 16);
    ks_garner_kernel<<<static_cast<unsigned>(bx), 256, 0, s>>>(ct, n, 31 - __builtin_clz(N), c0,
                                                               nb, tab, g, V);
    return cudaGetLastError();
}
cudaError_t launch_ks_decompose(const uint64_t *ct, int64_t n, int N, int64_t c0, int64_t nb,
                                const NttPlane *tab, const KsGadget &g, const uint64_t *V,
                                uint64_t *D, cudaStream_t s) {
    if (nb == 0) return cudaSuccess;
    ks_decompose_kernel<<<152 * 16, 256, 0, s>>>(ct, n, N, c0, nb, tab, g, V, D);
    return cudaGetLastError();
}
cudaError_t launch_ks_multacc(const uint64_t *D, const uint64_t *keys, const int *kid, int kper,
                              const KsGadget &g, int N, int64_t c0, int64_t nb,
                              const NttPlane *tab, uint64_t *U, cudaStream_t s, int d_shared) {
    if (nb == 0) return cudaSuccess;
    const int logN = 31 - __builtin_clz(N);
    const int Lp = g.L + g.K;
    const int64_t total = nb * Lp * N / 2;
    const int64_t bx = std::min<int64_t>((total + 255) / 256, 152 * 16);
    ks_multacc_kernel<<<static_cast<unsigned>(bx), 256, 0, s>>>(D, keys, kid, kper, g.D, Lp, logN,
                                                                c0, nb, tab, U, d_shared);
    return cudaGetLastError();
}
cudaError_t launch_ks_moddown(const uint64_t *U, const uint64_t *ct, int64_t n, int N, int64_t c0,
                              int64_t nb, const int *kid, int kper, int b_zero,
                              const NttPlane *tab, const KsGadget &g, const uint64_t *pinv,
                              const uint64_t *pinv_s, uint64_t *out, int64_t n_out,
                              cudaStream_t s) {
    if (nb == 0) return cudaSuccess;
    const int logN = 31 - __builtin_clz(N);
    const int64_t bx = std::min<int64_t>((nb * N / 2 + 255) / 256, 152 * 8);
    ks_moddown_kernel<<<dim3(static_cast<unsigned>(bx), 2), 256, 0, s>>>(
        U, ct, n, logN, c0, nb, kid, kper, b_zero, tab, g, pinv, pinv_s, out, n_out);
    return cudaGetLastError();
}

// ------------------------------------------------------------ gathers, Tweak
// Batches have power-of-two N (and, for Tweak, n and the table period), so
// every index below is a shift or a mask; blockIdx.y selects the (part,
// prime) plane: 2L of them, or the L a-part planes only (parts = 1).

// out[c] = scale * sigma_ell(c)(in[src(c)]) for every part and plane (the
// N^-1, source permutation and Aut before the key switches of Alg. 4); the
// tables repeat with period t.per (ciphertext c reads entry c mod per, and
// src is relative to the block of `per` ciphertexts holding c).  sigma_ell
// maps X^i to X^(i*ell mod 2N) (X^N = -1).  One thread per output
// coefficient: it reads input coefficient i = pos * ell^-1 mod 2N.
__global__ void ct_gather_kernel(const uint64_t *__restrict__ in, uint64_t *__restrict__ out,
                                 int64_t n, int L, int logN, GatherTables t,
                                 const NttPlane *__restrict__ tab) {
    const int r = blockIdx.y;  // part * L + plane
    const int plane = r % L;
    const uint64_t q = tab[plane].q;
    const int N = 1 << logN;
    const int twoN_mask = 2 * N - 1;
    const int per_mask = t.per - 1;
    uint64_t sc_w = 0, sc_ws = 0;
    if (t.scale) {
        sc_w = t.scale[plane];
        sc_ws = t.scale_s[plane];
    }
    const uint64_t *inp = in + static_cast<int64_t>(r) * n * N;
    uint64_t *outp = out + static_cast<int64_t>(r) * n * N;
    const int64_t total = n << logN;
    for (int64_t x = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; x < total;
         x += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int pos = static_cast<int>(x) & (N - 1);
        const int64_t c = x >> logN;
        const int ci = static_cast<int>(c) & per_mask;
        const int si = t.src ? t.src[ci] : ci;
        int e = pos;
        if (t.ellinv) e = static_cast<int>((static_cast<int64_t>(e) * t.ellinv[ci]) & twoN_mask);
        const bool neg = e >= N;
        e &= N - 1;
        uint64_t v = inp[((c - ci + si) << logN) + e];
        if (t.scale) v = shoup_mulmod(v, sc_w, sc_ws, q);
        outp[x] = (neg && v != 0) ? q - v : v;
    }
}

cudaError_t launch_ct_gather(const uint64_t *in, uint64_t *out, int64_t n, int L, int N,
                             const GatherTables &t, const NttPlane *tab, cudaStream_t s,
                             int parts) {
    if (n == 0) return cudaSuccess;
    const int64_t per_plane = n * N;
    const int64_t bx = std::min<int64_t>((per_plane + 255) / 256, 152 * 8);
    ct_gather_kernel<<<dim3(static_cast<unsigned>(bx), parts * L), 256, 0, s>>>(in, out, n, L,
                                                                            31 - __builtin_clz(N), t, tab);
    return cudaGetLastError();
}

// ------------------------------------------------------------ Tweak passes
// Input and output maps of a Tweak pass (TweakMap, ring_internal.h) fold the
// gathers around the Tweaks of Alg. 4 into the first and last passes.
__device__ __forceinline__ uint64_t neg_mod(uint64_t v, uint64_t q) { return v == 0 ? 0 : q - v; }

// Coefficients m and m + 1 of X^t x, m and t even (t taken mod 2N): one
// 16-byte load, negated when the window lies in the upper half.
__device__ __forceinline__ ulonglong2 rot_load(const uint64_t *x, int m, int t, int N, uint64_t q) {
    // coefficient m (and m + 1) of X^t x, m and t even (t taken mod 2N)
    int e = (m - t) & (2 * N - 1);
    const bool neg = e >= N;
    e &= N - 1;
    ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(x + e);
    if (neg) {
        v.x = v.x == 0 ? 0 : q - v.x;
        v.y = v.y == 0 ? 0 : q - v.y;
    }
    return v;
}

// Coefficients m and m + 1 of X^t x for any t (odd t included: the two
// words are loaded separately and may sit on either side of the wrap).
__device__ __forceinline__ ulonglong2 rot_load_any(const uint64_t *x, int m, int t, int N,
                                                   uint64_t q) {
    const int e0 = (m - t) & (2 * N - 1), e1 = (m + 1 - t) & (2 * N - 1);
    ulonglong2 v;
    v.x = x[e0 & (N - 1)];
    v.y = x[e1 & (N - 1)];
    if (e0 >= N) v.x = neg_mod(v.x, q);
    if (e1 >= N) v.y = neg_mod(v.y, q);
    return v;
}

// Where input ciphertext i of a pass is read: itself, or (input map) the
// bit-reversed index si of its group of 2^in_bits, with an extra rotation
// X^si when in_shift.
template <bool MI>
__device__ __forceinline__ const uint64_t *tw_src(const uint64_t *inp, int64_t i, int logN,
                                                  const TweakMap &mp, int &rot) {
    if constexpr (!MI) {
        rot = 0;
        return inp + (i << logN);
    } else {
        const int64_t mask = (int64_t(1) << mp.in_bits) - 1;
        const int ci = static_cast<int>(i & mask);
        const int si = static_cast<int>(__brev(static_cast<unsigned>(ci)) >> (32 - mp.in_bits));
        rot = mp.in_shift ? si : 0;
        return inp + (((i - ci) + si) << logN);
    }
}

// Coefficients m, m + 1 of X^t times the source x (rotation rx of the map added).
template <bool MI>
__device__ __forceinline__ ulonglong2 tw_load(const uint64_t *x, int m, int t, int rx, int N,
                                              uint64_t q) {
    if constexpr (MI) return rot_load_any(x, m, t + rx, N, q);
    else return rot_load(x, m, t, N, q);
}
template <bool MI>
__device__ __forceinline__ ulonglong2 tw_load0(const uint64_t *x, int m, int rx, int N, uint64_t q) {
    if constexpr (MI) return rot_load_any(x, m, rx, N, q);
    else return *reinterpret_cast<const ulonglong2 *>(x + m);
}

// Stores coefficients m, m + 1 of output ciphertext o: in place, or (output
// map) into ciphertext j = (N - i) mod N of o's group of N (i = o mod N)
// times X^(N + i) for i > 0: ct'_j = X^(2N - j) ct''_(N - j), ct'_0 = ct''_0.
template <bool MO>
__device__ __forceinline__ void tw_store(uint64_t *outp, int64_t o, int m, ulonglong2 v, int logN,
                                         uint64_t q) {
    if constexpr (!MO) {
        *reinterpret_cast<ulonglong2 *>(outp + (o << logN) + m) = v;
    } else {
        const int N = 1 << logN;
        const int i = static_cast<int>(o & (N - 1));
        const int64_t dst = (o - i) + ((N - i) & (N - 1));
        const int rot = i == 0 ? 0 : N + i;
        const int p0 = (m + rot) & (2 * N - 1), p1 = (m + 1 + rot) & (2 * N - 1);
        uint64_t *d = outp + (dst << logN);
        d[p0 & (N - 1)] = p0 >= N ? neg_mod(v.x, q) : v.x;
        d[p1 & (N - 1)] = p1 >= N ? neg_mod(v.y, q) : v.y;
    }
}

// One radix-2 stage of Tweak (an n-point DFT over R_q with omega = X^(2N/n)):
// for pairs (lo, hi = lo + half) inside blocks of 2*half,
//   out_lo = x_lo + X^t x_hi,  out_hi = x_lo - X^t x_hi,  t = (lo mod half) * N / half.
// Input ciphertexts must be in bit-reversed order before the first stage
// (or the pass's input map bit-reverses them).
// Each thread takes two neighbouring coefficients with 16-byte accesses; t is
// even whenever half < N, so the rotated read stays 16-byte aligned.
template <bool MI, bool MO>
__global__ void tweak_stage_kernel(const uint64_t *__restrict__ in, uint64_t *__restrict__ out,
                                   int64_t n, int L, int logN, int lhalf,
                                   const NttPlane *__restrict__ tab, TweakMap mp) {
    const int r = blockIdx.y;  // part * L + plane
    const uint64_t q = tab[r % L].q;
    const int N = 1 << logN;
    const uint64_t *inp = in + static_cast<int64_t>(r) * n * N;
    uint64_t *outp = out + static_cast<int64_t>(r) * n * N;
    const int64_t total = (n >> 1) << (logN - 1);  // pairs x coefficient pairs
    const int64_t half_mask = (int64_t(1) << lhalf) - 1;
    for (int64_t w = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; w < total;
         w += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int m = (static_cast<int>(w) << 1) & (N - 1);
        const int64_t pr = w >> (logN - 1);
        const int64_t jj = pr & half_mask;
        const int64_t lo = ((pr >> lhalf) << (lhalf + 1)) + jj;
        const int64_t hi = lo + (int64_t(1) << lhalf);
        const int tt = static_cast<int>(jj << (logN - lhalf));
        int ra, rb;
        const uint64_t *xl = tw_src<MI>(inp, lo, logN, mp, ra);
        const uint64_t *xh = tw_src<MI>(inp, hi, logN, mp, rb);
        const ulonglong2 a = tw_load0<MI>(xl, m, ra, N, q);
        const ulonglong2 y = tw_load<MI>(xh, m, tt, rb, N, q);
        ulonglong2 o0, o1;
        o0.x = add_mod(a.x, y.x, q);
        o0.y = add_mod(a.y, y.y, q);
        o1.x = sub_mod(a.x, y.x, q);
        o1.y = sub_mod(a.y, y.y, q);
        tw_store<MO>(outp, lo, m, o0, logN, q);
        tw_store<MO>(outp, hi, m, o1, logN, q);
    }
}

// Two consecutive stages (half = h, then 2h) in one pass, for 4h <= N.  For
// the four ciphertexts i0 = 4h blk + jj, i1 = i0 + h, i2 = i0 + 2h,
// i3 = i0 + 3h, with R_t(x) = X^t x, tA = jj N / h and tB = jj N / (2h):
//   z0 = x0 + R_tA(x1) + R_tB(x2)       + R_{tA+tB}(x3)
//   z2 = x0 + R_tA(x1) - R_tB(x2)       - R_{tA+tB}(x3)
//   z1 = x0 - R_tA(x1) + R_{tB+N/2}(x2) - R_{tA+tB+N/2}(x3)
//   z3 = x0 - R_tA(x1) - R_{tB+N/2}(x2) + R_{tA+tB+N/2}(x3)
// (the second stage pairs (i1, i3) with twiddle X^(tB + N/2)).  Six rotated
// reads of contiguous windows give four outputs, instead of eight reads and
// eight writes for two radix-2 passes.  All rotations are even, so two
// neighbouring coefficients move together in 16-byte accesses (an input map
// adds rotations of any parity; those reads take two 8-byte loads).

template <bool MI, bool MO>
__global__ void tweak_radix4_kernel(const uint64_t *__restrict__ in, uint64_t *__restrict__ out,
                                    int64_t n, int L, int logN, int lh,
                                    const NttPlane *__restrict__ tab, TweakMap mp) {
    const int r = blockIdx.y;  // part * L + plane
    const uint64_t q = tab[r % L].q;
    const int N = 1 << logN;
    const uint64_t *inp = in + static_cast<int64_t>(r) * n * N;
    uint64_t *outp = out + static_cast<int64_t>(r) * n * N;
    const int64_t total = (n >> 2) << (logN - 1);  // groups of four x coefficient pairs
    const int64_t h_mask = (int64_t(1) << lh) - 1;
    for (int64_t w = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; w < total;
         w += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int m = (static_cast<int>(w) << 1) & (N - 1);
        const int64_t g = w >> (logN - 1);
        const int64_t jj = g & h_mask;
        const int64_t i0 = ((g >> lh) << (lh + 2)) + jj;
        const int64_t h = int64_t(1) << lh;
        const int tA = static_cast<int>(jj << (logN - lh));
        const int tB = static_cast<int>(jj << (logN - lh - 1));
        const int halfN = N >> 1;
        int rx[4];
        const uint64_t *x[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) x[k] = tw_src<MI>(inp, i0 + k * h, logN, mp, rx[k]);
        const ulonglong2 a = tw_load0<MI>(x[0], m, rx[0], N, q);
        const ulonglong2 b = tw_load<MI>(x[1], m, tA, rx[1], N, q);
        const ulonglong2 c0 = tw_load<MI>(x[2], m, tB, rx[2], N, q);
        const ulonglong2 c1 = tw_load<MI>(x[2], m, tB + halfN, rx[2], N, q);
        const ulonglong2 d0 = tw_load<MI>(x[3], m, tA + tB, rx[3], N, q);
        const ulonglong2 d1 = tw_load<MI>(x[3], m, tA + tB + halfN, rx[3], N, q);
        ulonglong2 z0, z1, z2, z3;
        {
            const uint64_t p = add_mod(a.x, b.x, q), mm = sub_mod(a.x, b.x, q);
            const uint64_t s0 = add_mod(c0.x, d0.x, q), s1 = sub_mod(c1.x, d1.x, q);
            z0.x = add_mod(p, s0, q);
            z2.x = sub_mod(p, s0, q);
            z1.x = add_mod(mm, s1, q);
            z3.x = sub_mod(mm, s1, q);
        }
        {
            const uint64_t p = add_mod(a.y, b.y, q), mm = sub_mod(a.y, b.y, q);
            const uint64_t s0 = add_mod(c0.y, d0.y, q), s1 = sub_mod(c1.y, d1.y, q);
            z0.y = add_mod(p, s0, q);
            z2.y = sub_mod(p, s0, q);
            z1.y = add_mod(mm, s1, q);
            z3.y = sub_mod(mm, s1, q);
        }
        tw_store<MO>(outp, i0, m, z0, logN, q);
        tw_store<MO>(outp, i0 + h, m, z1, logN, q);
        tw_store<MO>(outp, i0 + 2 * h, m, z2, logN, q);
        tw_store<MO>(outp, i0 + 3 * h, m, z3, logN, q);
    }
}

template <bool MI, bool MO>
static void tweak_radix4_go(dim3 g, cudaStream_t s, const uint64_t *in, uint64_t *out, int64_t n,
                            int L, int logN, int lh, const NttPlane *tab, const TweakMap &mp) {
    tweak_radix4_kernel<MI, MO><<<g, 256, 0, s>>>(in, out, n, L, logN, lh, tab, mp);
}

cudaError_t launch_tweak_radix4(const uint64_t *in, uint64_t *out, int64_t n, int L, int N,
                                int64_t half, const NttPlane *tab, cudaStream_t s, int parts,
                                const TweakMap &mp) {
    const int logN = 31 - __builtin_clz(N);
    const int lh = 63 - __builtin_clzll(static_cast<unsigned long long>(half));
    const int64_t per_plane = (n >> 2) * (N >> 1);
    const int64_t bx = std::min<int64_t>((per_plane + 255) / 256, 152 * 8);
    const dim3 g(static_cast<unsigned>(bx), parts * L);
    const bool mi = mp.in_bits > 0, mo = mp.out_t3 != 0;
    if (mi && mo) tweak_radix4_go<true, true>(g, s, in, out, n, L, logN, lh, tab, mp);
    else if (mi) tweak_radix4_go<true, false>(g, s, in, out, n, L, logN, lh, tab, mp);
    else if (mo) tweak_radix4_go<false, true>(g, s, in, out, n, L, logN, lh, tab, mp);
    else tweak_radix4_go<false, false>(g, s, in, out, n, L, logN, lh, tab, mp);
    return cudaGetLastError();
}

// Three consecutive stages (half = h, 2h, 4h) in one pass, for 8h <= N.  For
// the eight ciphertexts x_k = i0 + k h (k < 8), i0 = 8h blk + jj, with
// tA = jj N / h, tB = jj N / (2h), tC = jj N / (4h):
//   the first two stages are the radix-4 pass on x0..x3 (giving z0..z3) and
//   on x4..x7 (giving z4..z7); the third pairs (z_k, z_{k+4}) with twiddle
//   X^(c_k), c_k = tC + k N / 4 (element i0 + k h sits at index jj + k h of
//   its block of 8h).  R_{c_k}(z_{k+4}) is read directly as rotated windows
//   of x4..x7, with the signs and the N/2 shifts of z_{k+4}'s radix-4 row:
//     k = 0:  R_c x4 + R_{c+tA} x5 + R_{c+tB} x6       + R_{c+tA+tB} x7
//     k = 1:  R_c x4 - R_{c+tA} x5 + R_{c+tB+N/2} x6 - R_{c+tA+tB+N/2} x7
//     k = 2:  R_c x4 + R_{c+tA} x5 - R_{c+tB} x6       - R_{c+tA+tB} x7
//     k = 3:  R_c x4 - R_{c+tA} x5 - R_{c+tB+N/2} x6 + R_{c+tA+tB+N/2} x7
//   and the outputs are z_k + R_{c_k}(z_{k+4}) at i0 + k h and the difference
//   at i0 + (k + 4) h.
// 22 rotated 16-byte reads (the re-reads of a window hit in L2) and eight
// writes per thread replace three radix-2 passes' reads and writes of the
// batch.  All rotations stay even (8h <= N), so coefficient pairs move together.
// IDX: int when a (part, prime) plane of n * N words has fewer than 2^31 of
// them (64 registers: four CTAs of 256 threads per SM), else int64_t.
template <bool MI, bool MO, typename IDX>
__global__ void __launch_bounds__(256, sizeof(IDX) == 4 ? 4 : 3)
    tweak_radix8_kernel(const uint64_t *__restrict__ in, uint64_t *__restrict__ out, int64_t n,
                        int L, int logN, int lh, const NttPlane *__restrict__ tab, TweakMap mp) {
    const int r = blockIdx.y;  // part * L + plane
    const uint64_t q = tab[r % L].q;
    const int N = 1 << logN;
    const uint64_t *inp = in + static_cast<int64_t>(r) * n * N;
    uint64_t *outp = out + static_cast<int64_t>(r) * n * N;
    const IDX total = static_cast<IDX>((n >> 3) << (logN - 1));  // groups of eight x coefficient pairs
    const IDX h_mask = (IDX(1) << lh) - 1;
    const IDX h = IDX(1) << lh;
    const int halfN = N >> 1, quarterN = N >> 2;
    for (IDX w = static_cast<IDX>(blockIdx.x * blockDim.x + threadIdx.x); w < total;
         w += static_cast<IDX>(gridDim.x * blockDim.x)) {
        const int m = static_cast<int>(w << 1) & (N - 1);
        const IDX g = w >> (logN - 1);
        const IDX jj = g & h_mask;
        const IDX i0 = ((g >> lh) << (lh + 3)) + jj;
        const int tA = static_cast<int>(jj << (logN - lh));
        const int tB = static_cast<int>(jj << (logN - lh - 1));
        const int tC = static_cast<int>(jj << (logN - lh - 2));
        int rx[8];
        const uint64_t *xs[8];
        if constexpr (MI) {
#pragma unroll
            for (int k = 0; k < 8; ++k) xs[k] = tw_src<MI>(inp, i0 + k * h, logN, mp, rx[k]);
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) rx[k] = 0;
        }
        auto x = [&](int k) -> const uint64_t * {
            if constexpr (MI) return xs[k];
            else return inp + (static_cast<std::make_unsigned_t<IDX>>(i0 + k * h) << logN);
        };
        // z0..z3: the first two stages on x0..x3
        const ulonglong2 a = tw_load0<MI>(x(0), m, rx[0], N, q);
        const ulonglong2 b = tw_load<MI>(x(1), m, tA, rx[1], N, q);
        const ulonglong2 c0 = tw_load<MI>(x(2), m, tB, rx[2], N, q);
        const ulonglong2 c1 = tw_load<MI>(x(2), m, tB + halfN, rx[2], N, q);
        const ulonglong2 d0 = tw_load<MI>(x(3), m, tA + tB, rx[3], N, q);
        const ulonglong2 d1 = tw_load<MI>(x(3), m, tA + tB + halfN, rx[3], N, q);
        ulonglong2 z[4];
        {
            const uint64_t p = add_mod(a.x, b.x, q), mm = sub_mod(a.x, b.x, q);
            const uint64_t s0 = add_mod(c0.x, d0.x, q), s1 = sub_mod(c1.x, d1.x, q);
            z[0].x = add_mod(p, s0, q);
            z[2].x = sub_mod(p, s0, q);
            z[1].x = add_mod(mm, s1, q);
            z[3].x = sub_mod(mm, s1, q);
        }
        {
            const uint64_t p = add_mod(a.y, b.y, q), mm = sub_mod(a.y, b.y, q);
            const uint64_t s0 = add_mod(c0.y, d0.y, q), s1 = sub_mod(c1.y, d1.y, q);
            z[0].y = add_mod(p, s0, q);
            z[2].y = sub_mod(p, s0, q);
            z[1].y = add_mod(mm, s1, q);
            z[3].y = sub_mod(mm, s1, q);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c = tC + k * quarterN;
            const int tb = (k & 1) ? tB + halfN : tB;
            const ulonglong2 e4 = tw_load<MI>(x(4), m, c, rx[4], N, q);
            const ulonglong2 e5 = tw_load<MI>(x(5), m, c + tA, rx[5], N, q);
            const ulonglong2 e6 = tw_load<MI>(x(6), m, c + tb, rx[6], N, q);
            const ulonglong2 e7 = tw_load<MI>(x(7), m, c + tA + tb, rx[7], N, q);
            // u = e4 +- e5 +- e6 +- e7 with the signs of row k
            ulonglong2 u;
            {
                const uint64_t p = (k & 1) ? sub_mod(e4.x, e5.x, q) : add_mod(e4.x, e5.x, q);
                const uint64_t t = (k & 1) ? sub_mod(e6.x, e7.x, q) : add_mod(e6.x, e7.x, q);
                u.x = (k & 2) ? sub_mod(p, t, q) : add_mod(p, t, q);
            }
            {
                const uint64_t p = (k & 1) ? sub_mod(e4.y, e5.y, q) : add_mod(e4.y, e5.y, q);
                const uint64_t t = (k & 1) ? sub_mod(e6.y, e7.y, q) : add_mod(e6.y, e7.y, q);
                u.y = (k & 2) ? sub_mod(p, t, q) : add_mod(p, t, q);
            }
            ulonglong2 o0, o1;
            o0.x = add_mod(z[k].x, u.x, q);
            o0.y = add_mod(z[k].y, u.y, q);
            o1.x = sub_mod(z[k].x, u.x, q);
            o1.y = sub_mod(z[k].y, u.y, q);
            tw_store<MO>(outp, i0 + k * h, m, o0, logN, q);
            tw_store<MO>(outp, i0 + (k + 4) * h, m, o1, logN, q);
        }
    }
}

// MODPP_TWEAK_WIDE_INDEX=1 takes the 64-bit-index form at every size (tests).
template <bool MI, bool MO>
static void tweak_radix8_go(dim3 g, cudaStream_t s, const uint64_t *in, uint64_t *out, int64_t n,
                            int L, int logN, int lh, const NttPlane *tab, const TweakMap &mp) {
    const char *wide = std::getenv("MODPP_TWEAK_WIDE_INDEX");
    if ((n << logN) < (int64_t(1) << 31) && !(wide && wide[0] == '1'))
        tweak_radix8_kernel<MI, MO, int><<<g, 256, 0, s>>>(in, out, n, L, logN, lh, tab, mp);
    else
        tweak_radix8_kernel<MI, MO, int64_t><<<g, 256, 0, s>>>(in, out, n, L, logN, lh, tab, mp);
}

cudaError_t launch_tweak_radix8(const uint64_t *in, uint64_t *out, int64_t n, int L, int N,
                                int64_t half, const NttPlane *tab, cudaStream_t s, int parts,
                                const TweakMap &mp) {
    const int logN = 31 - __builtin_clz(N);
    const int lh = 63 - __builtin_clzll(static_cast<unsigned long long>(half));
    const int64_t per_plane = (n >> 3) * (N >> 1);
    const int64_t bx = std::min<int64_t>((per_plane + 255) / 256, 152 * 8);
    const dim3 g(static_cast<unsigned>(bx), parts * L);
    const bool mi = mp.in_bits > 0, mo = mp.out_t3 != 0;
    if (mi && mo) tweak_radix8_go<true, true>(g, s, in, out, n, L, logN, lh, tab, mp);
    else if (mi) tweak_radix8_go<true, false>(g, s, in, out, n, L, logN, lh, tab, mp);
    else if (mo) tweak_radix8_go<false, true>(g, s, in, out, n, L, logN, lh, tab, mp);
    else tweak_radix8_go<false, false>(g, s, in, out, n, L, logN, lh, tab, mp);
    return cudaGetLastError();
}

// The same stage for half = N (n = 2N), where t = jj is odd for odd jj: one
// coefficient per thread.
__global__ void tweak_stage_scalar_kernel(const uint64_t *__restrict__ in,
                                          uint64_t *__restrict__ out, int64_t n, int L, int logN,
                                          int lhalf, const NttPlane *__restrict__ tab) {
    const int r = blockIdx.y;
    const uint64_t q = tab[r % L].q;
    const int N = 1 << logN;
    const uint64_t *inp = in + static_cast<int64_t>(r) * n * N;
    uint64_t *outp = out + static_cast<int64_t>(r) * n * N;
    const int64_t total = (n >> 1) << logN;
    const int64_t half_mask = (int64_t(1) << lhalf) - 1;
    for (int64_t w = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; w < total;
         w += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int m = static_cast<int>(w) & (N - 1);
        const int64_t pr = w >> logN;
        const int64_t jj = pr & half_mask;
        const int64_t lo = ((pr >> lhalf) << (lhalf + 1)) + jj;
        const int64_t hi = lo + (int64_t(1) << lhalf);
        const int tt = static_cast<int>((jj << logN) >> lhalf);
        const uint64_t a = inp[(lo << logN) + m];
        const int src = m - tt;
        uint64_t y = inp[(hi << logN) + (src & (N - 1))];
        if (src < 0) y = y == 0 ? 0 : q - y;
        outp[(lo << logN) + m] = add_mod(a, y, q);
        outp[(hi << logN) + m] = sub_mod(a, y, q);
    }
}

template <bool MI, bool MO>
static void tweak_stage_go(dim3 g, cudaStream_t s, const uint64_t *in, uint64_t *out, int64_t n,
                           int L, int logN, int lh, const NttPlane *tab, const TweakMap &mp) {
    tweak_stage_kernel<MI, MO><<<g, 256, 0, s>>>(in, out, n, L, logN, lh, tab, mp);
}

cudaError_t launch_tweak_stage(const uint64_t *in, uint64_t *out, int64_t n, int L, int N,
                               int64_t half, const NttPlane *tab, cudaStream_t s, int parts,
                               const TweakMap &mp) {
    if (n < 2) return cudaSuccess;
    const int logN = 31 - __builtin_clz(N);
    const int lhalf = 63 - __builtin_clzll(static_cast<unsigned long long>(half));
    const int64_t per_plane = (n >> 1) * N;
    const bool mi = mp.in_bits > 0, mo = mp.out_t3 != 0;
    if (lhalf < logN && N >= 2) {
        const int64_t bx = std::min<int64_t>((per_plane / 2 + 255) / 256, 152 * 8);
        const dim3 g(static_cast<unsigned>(bx), parts * L);
        if (mi && mo) tweak_stage_go<true, true>(g, s, in, out, n, L, logN, lhalf, tab, mp);
        else if (mi) tweak_stage_go<true, false>(g, s, in, out, n, L, logN, lhalf, tab, mp);
        else if (mo) tweak_stage_go<false, true>(g, s, in, out, n, L, logN, lhalf, tab, mp);
        else tweak_stage_go<false, false>(g, s, in, out, n, L, logN, lhalf, tab, mp);
    } else {
        if (mi || mo) return cudaErrorInvalidValue;  // the half = N stage takes no map
        const int64_t bx = std::min<int64_t>((per_plane + 255) / 256, 152 * 8);
        tweak_stage_scalar_kernel<<<dim3(static_cast<unsigned>(bx), parts * L), 256, 0, s>>>(
            in, out, n, L, logN, lhalf, tab);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------ elementwise
// out = x + y (mod q of each plane); arrays [parts][L][count] with planes of
// `count` words.
__global__ void add_planes_kernel(const uint64_t *x, const uint64_t *y, uint64_t *out, int parts,
                                  int L, int64_t count, const NttPlane *__restrict__ tab) {
    const int64_t total = static_cast<int64_t>(parts) * L * count;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int plane = static_cast<int>((i / count) % L);
        out[i] = add_mod(x[i], y[i], tab[plane].q);
    }
}

cudaError_t launch_add_planes(const uint64_t *x, const uint64_t *y, uint64_t *out, int parts, int L,
                              int64_t count, const NttPlane *tab, cudaStream_t s) {
    add_planes_kernel<<<152 * 16, 256, 0, s>>>(x, y, out, parts, L, count, tab);
    return cudaGetLastError();
}

// Rescale by q_{L-1}: [2][L][count] -> [2][L-1][count],
// x -> (x_k - r) * q_{L-1}^-1 mod q_k with r = [x]_{q_{L-1}} centred.
__global__ void rescale_kernel(const uint64_t *__restrict__ in, uint64_t *__restrict__ out, int L,
                               int64_t count, const NttPlane *__restrict__ tab,
                               const uint64_t *__restrict__ qlinv,
                               const uint64_t *__restrict__ qlinv_s) {
    const uint64_t ql = tab[L - 1].q;
    const int64_t total = 2 * static_cast<int64_t>(L - 1) * count;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t e = i % count;
        const int64_t r = i / count;
        const int k = static_cast<int>(r % (L - 1));
        const int part = static_cast<int>(r / (L - 1));
        const uint64_t q = tab[k].q;
        const uint64_t xl = in[(static_cast<int64_t>(part) * L + (L - 1)) * count + e];
        const uint64_t xk = in[(static_cast<int64_t>(part) * L + k) * count + e];
        uint64_t rq;
        if (xl > ql / 2) {
            const uint64_t mag = barrett_u64(ql - xl, q, tab[k].mu);
            rq = mag == 0 ? 0 : q - mag;
        } else {
            rq = barrett_u64(xl, q, tab[k].mu);
        }
        out[i] = shoup_mulmod(sub_mod(xk, rq, q), qlinv[k], qlinv_s[k], q);
    }
}

cudaError_t launch_rescale(const uint64_t *in, uint64_t *out, int L, int64_t count,
                           const NttPlane *tab, const uint64_t *qlinv, const uint64_t *qlinv_s,
                           cudaStream_t s) {
    rescale_kernel<<<152 * 16, 256, 0, s>>>(in, out, L, count, tab, qlinv, qlinv_s);
    return cudaGetLastError();
}

// out[c][r] = in[r][c] for `mats` matrices of rows x cols (leading dimensions
// ldi, ldo; matrix strides si, so), through 32 x 32 shared-memory tiles.
__global__ void transpose_u64_kernel(const uint64_t *__restrict__ in, uint64_t *__restrict__ out,
                                     int rows, int cols, int64_t ldi, int64_t ldo, int64_t si,
                                     int64_t so) {
    __shared__ uint64_t tile[32][33];
    const int64_t mat = blockIdx.z;
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = r0 + y, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[y][threadIdx.x] = in[mat * si + r * ldi + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int c = c0 + y, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[mat * so + c * ldo + r] = tile[threadIdx.x][y];
    }
}

cudaError_t launch_transpose_u64(const uint64_t *in, uint64_t *out, int rows, int cols,
                                 int64_t ldi, int64_t ldo, int64_t si, int64_t so, int mats,
                                 cudaStream_t s) {
    if (rows == 0 || cols == 0 || mats == 0) return cudaSuccess;
    dim3 grid((cols + 31) / 32, (rows + 31) / 32, mats);
    transpose_u64_kernel<<<grid, dim3(32, 8), 0, s>>>(in, out, rows, cols, ldi, ldo, si, so);
    return cudaGetLastError();
}

// Step 5 of Alg. 8 fused with Rescale by q_{L-1}: for ciphertext j and
// coefficient m,
//   a = Relin(D0_j, 0)_a + D1_j + D2_j + C01[m][j],
//   b = Relin(D0_j, 0)_b + D3_j + C11[m][j],
// then x -> (x_k - r) * q_{L-1}^-1 mod q_k with r = [x]_{q_{L-1}} centred.
// C01 and C11 are read transposed through a 32 x 32 shared-memory tile.
__device__ __forceinline__ uint64_t lift_centred(uint64_t x, uint64_t ql, uint64_t q, uint64_t mu) {
    if (x > ql / 2) {
        const uint64_t mag = barrett_u64(ql - x, q, mu);
        return mag == 0 ? 0 : q - mag;
    }
    return barrett_u64(x, q, mu);
}

__global__ void __launch_bounds__(256) cc_finish_kernel(CcFinishParams p) {
    __shared__ uint64_t tile[32][33];
    const int N = p.N, L = p.L;
    const int part = blockIdx.z;
    const int m0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const int64_t NN = static_cast<int64_t>(N) * N;
    const int64_t Rpart = static_cast<int64_t>(part) * L * NN;
    const uint64_t ql = p.tab[L - 1].q;
    uint64_t rl[4];  // x_{L-1} of this thread's four elements
    for (int pass = 0; pass < L; ++pass) {
        const int k = pass == 0 ? L - 1 : pass - 1;
        const uint64_t q = p.tab[k].q;
        // transposed tile of C01 (part 0) or C11 (part 1): rows m, columns j
        const uint64_t *Yk = p.Y + static_cast<int64_t>(k) * 2 * NN + (part ? NN : 0);
        __syncthreads();
        for (int y = threadIdx.y; y < 32; y += 8) {
            const int m = m0 + y, j = j0 + threadIdx.x;
            if (m < N && j < N) tile[y][threadIdx.x] = Yk[static_cast<int64_t>(m) * N + j];
        }
        __syncthreads();
        for (int e = 0; e < 4; ++e) {
            const int jl = threadIdx.y + 8 * e;
            const int j = j0 + jl, m = m0 + threadIdx.x;
            if (j >= N || m >= N) continue;
            const int64_t o = static_cast<int64_t>(j) * N + m;
            const int64_t zk = static_cast<int64_t>(k) * 2 * NN;  // plane k of a 2N batch
            const int64_t zpart = static_cast<int64_t>(L) * 2 * NN;
            uint64_t v = p.R[Rpart + k * NN + o];
            if (part == 0) {
                v = add_mod(v, p.Z[zpart + zk + o], q);        // D1_j
                v = add_mod(v, p.Z[zk + NN + o], q);           // D2_j
            } else {
                v = add_mod(v, p.Z[zpart + zk + NN + o], q);   // D3_j
            }
            v = add_mod(v, tile[threadIdx.x][jl], q);          // C01 / C11, column j
            if (pass == 0) {
                rl[e] = v;
            } else {
                const uint64_t rq = lift_centred(rl[e], ql, q, p.tab[k].mu);
                p.out[(static_cast<int64_t>(part) * (L - 1) + k) * NN + o] =
                    shoup_mulmod(sub_mod(v, rq, q), p.qlinv[k], p.qlinv_s[k], q);
            }
        }
    }
}

cudaError_t launch_cc_finish(const CcFinishParams &p, cudaStream_t s) {
    if (p.N == 0) return cudaSuccess;
    dim3 grid((p.N + 31) / 32, (p.N + 31) / 32, 2);
    cc_finish_kernel<<<grid, dim3(32, 8), 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace modpp
