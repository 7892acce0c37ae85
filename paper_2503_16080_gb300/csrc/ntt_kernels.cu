// Negacyclic NTT of degree N >= 1024, E coefficients per thread in registers.
//
// Same transform as the per-stage kernel in ring_kernels.cu (Cooley-Tukey
// forward / Gentleman-Sande inverse with bit-reversed powers of psi, Longa and
// Naehrig, CANS 2016), organised for the GPU: each thread holds E = 8
// coefficients (16 or 32 selectable) in registers and runs up to log2(E)
// butterfly stages on them before the coefficients go back to shared memory;
// the log2(N) stages are spread as evenly as possible over
// ceil(log2(N) / log2(E)) shared-memory round trips.  The first pass reads
// global memory and the last writes it.  For the default shapes the degree
// is a template parameter, so the pass schedule is fixed at compile time.
// Butterflies keep values lazily reduced: in Harvey's form (D. Harvey,
// "Faster arithmetic for number-theoretic transforms", J. Symb. Comp. 2014)
// forward values live in [0, 4q) and inverse ones in [0, 2q), for q < 2^62;
// for the primes where 64-bit words have room the bounds grow instead (see
// ntt_grow_ok_fwd / ntt_grow_ok_inv).
//
// The forward transform can also read its input from the a-part of a
// ciphertext batch: the digit of key switching (ks_gadget.cuh) is formed on
// the fly in the first pass, so the decomposition is fused into the
// transform.
#include <cuda_runtime.h>

#include <cstdlib>

#include "ks_gadget.cuh"
#include "modarith.cuh"
#include "ring_internal.h"

namespace modpp {
namespace {

// Shared-memory index with one padding word per 32: strided groups of
// threads then fall into different banks.
__device__ __forceinline__ int pad_idx(int j) { return j + (j >> 5); }

struct NttFastArgs {
    uint64_t *polys;
    int N, logN;
    int64_t inner;
    int nplanes;
    const NttPlane *tab;
    // Key-switching source (forward only): polynomial p = (c * D + d) * (L + K) + k
    // reads digit d of the a-part of ciphertext c0 + c of a batch with plane
    // stride n, modulo prime k (the gadget g).  Null: transform polys in place.
    const uint64_t *ks_ct;
    int64_t ks_n, ks_c0;
    const uint64_t *ks_v;  // Garner digits of two-prime digits, [nb][D][N]
    KsGadget g;
};

// Constants of the polynomial's prime, held in registers.
struct PlaneRegs {
    uint64_t q, q2, q4, mu, ninv, ninv_s;
    const ulonglong2 *tw;  // (twiddle, Shoup quotient) pairs: fwd2 (forward) or inv2 (inverse)
};

// First coefficient of group g in a pass with group stride 2^lu and groups
// of 2^S: groups are blocks of u * 2^S coefficients split by residue r < u.
// For u >= 16 consecutive threads take consecutive r (contiguous
// addresses), otherwise consecutive blocks (distinct padded banks).
template <int S>
__device__ __forceinline__ int group_start(int g, int lu, int lnb) {
    int blk, r;
    if (lu >= 4) {
        r = g & ((1 << lu) - 1);
        blk = g >> lu;
    } else {
        blk = g & ((1 << lnb) - 1);
        r = g >> lnb;
    }
    return (blk << (lu + S)) + r;
}

// Sink of a forward transform's last pass in key switching: the transformed
// digit times the two key polynomials (evaluation domain, Montgomery form),
// accumulated into two shared-memory accumulators (padded index).
struct MacSink {
    uint64_t *acc0, *acc1;
    const uint64_t *k0, *k1;
    uint64_t qinv;  // -q^-1 mod 2^64
    bool assign;    // first digit: the accumulators take the products
};

// Value ranges.  GROW = false: Harvey's lazy butterflies with Shoup
// products in [0, 2q); every value stays in [0, 4q) (forward) or [0, 2q)
// (inverse) between stages, for q < 2^62.  GROW = true drops the per-stage
// conditional subtractions and lets the bound grow instead, for the primes
// where 64-bit words have room, with the three-product Shoup quotient
// (products in [0, 4q)):
//   forward: the sum and the difference (taken against 4q) each add less
//            than 4q per stage, so after m stages every value is below
//            B0 + 4mq, B0 the input bound: q, or the largest chain prime
//            when the key-switch digits are transformed without reduction;
//   inverse: before stage m (m stages done) values are below 2^(m+1) q
//            (q for m = 0): the sum doubles the bound, the product stays
//            below 4q, and the difference is taken against that bound.
// Shoup's products accept any 64-bit multiplicand, and the Montgomery
// product of the key sink any 64-bit a times b < q, so only the plain
// forward output needs a full reduction (Barrett).
__host__ __device__ constexpr bool ntt_grow_ok_fwd(uint64_t q, uint64_t in_max, int logN) {
    // B0 + 4 * logN * q < 2^57 + 64 * 2^57 < 2^64 for logN <= 16
    return logN <= 16 && q < (1ull << 57) && in_max < (1ull << 57);
}
__host__ __device__ constexpr bool ntt_grow_ok_inv(uint64_t q, int logN) {
    // the last stage's sum is below 2^(logN + 1) q
    return logN <= 62 && q <= (~0ull >> (logN + 1));
}
// Difference offset of inverse stage m under GROW: the bound of its inputs.
__device__ __forceinline__ uint64_t grow_inv_bound(uint64_t q, int m) {
    return m == 0 ? q : q << (m + 1);
}

// Shared-memory index of coefficient j0 + k * 2^lu of a group: groups start
// at (blk << (lu + S)) + r with r < 2^lu, so adding k * 2^lu never carries
// across a multiple of 32 except through k * 2^lu itself, and the padded
// index is pad_idx(j0) plus a constant of k and lu.
__device__ __forceinline__ int pad_off(int k, int lu) { return (k << lu) + ((k << lu) >> 5); }

// TWO: the first pass reads a two-prime key-switch digit through ds (its
// Garner digits present); otherwise ds, when given, is read at run time.
template <int E, int S, bool FWD, bool MAC = false, bool GROW = false, bool TWO = false>
__device__ __forceinline__ void ntt_pass(uint64_t *sa, const uint64_t *gin, uint64_t *gout,
                                         bool reduce_in, int N, int logN, int lu, bool first,
                                         bool last, const PlaneRegs &pr,
                                         const MacSink *mk = nullptr,
                                         const DigitSrc *ds = nullptr) {
    constexpr int G = E >> S;  // groups of 2^S coefficients per thread
    constexpr int W = 1 << S;
    const int T = N / E;
    const int lnb = logN - lu - S;  // log2 of the number of blocks
    uint64_t v[E];
#pragma unroll
    for (int gi = 0; gi < G; ++gi) {
        const int j0 = group_start<S>(threadIdx.x + T * gi, lu, lnb);
        const int p0 = pad_idx(j0);
#pragma unroll
        for (int k = 0; k < W; ++k) {
            uint64_t x;
            if (first) {
                if (TWO || ds) {
                    x = digit_at<TWO>(*ds, j0 + (k << lu), pr.q, pr.mu, reduce_in);
                } else {
                    x = gin[j0 + (k << lu)];
                    if (reduce_in) x = barrett_u64(x, pr.q, pr.mu);
                }
            } else {
                x = sa[p0 + pad_off(k, lu)];
            }
            v[gi * W + k] = x;
        }
    }
#pragma unroll
    for (int gi = 0; gi < G; ++gi) {
        const int blk = group_start<S>(threadIdx.x + T * gi, lu, lnb) >> (lu + S);
#pragma unroll
        for (int st = 0; st < S; ++st) {
            // Pairs (k, k + half) of the group, k with bit `half` clear; the
            // twiddle index depends on k's sub-block only.
            //   forward: distance d = u * 2^(S-1-st), stage m = N / (2d),
            //            i = blk * 2^st + (k >> (S - st))
            //   inverse: distance d = u * 2^st, h = N / (2d),
            //            i = blk * 2^(S-1-st) + (k >> (st + 1))
            const int half = FWD ? (W >> (st + 1)) : (1 << st);
            const int base = FWD ? (N >> (lu + S - st)) + (blk << st)
                                 : (N >> (lu + st + 1)) + (blk << (S - 1 - st));
            const int sh = FWD ? (S - st) : (st + 1);
#pragma unroll
            for (int k = 0; k < W; ++k) {
                if (k & half) continue;
                uint64_t &x = v[gi * W + k];
                uint64_t &y = v[gi * W + k + half];
                const int ti = base + (k >> sh);
                const ulonglong2 tw = pr.tw[ti];
                const uint64_t w = tw.x, ws = tw.y;
                if (FWD) {
                    if (GROW) {
                        const uint64_t t = shoup_lazy3(y, w, ws, pr.q);
                        y = x - t + pr.q4;
                        x = x + t;
                    } else {
                        const uint64_t xa = min(x, x - pr.q2);  // x - 2q when x >= 2q
                        const uint64_t t = shoup_lazy(y, w, ws, pr.q);
                        x = xa + t;
                        y = xa - t + pr.q2;
                    }
                } else {
                    if (GROW) {
                        const uint64_t d = x - y + grow_inv_bound(pr.q, lu + st);
                        x = x + y;
                        y = shoup_lazy3(d, w, ws, pr.q);
                    } else {
                        uint64_t sm = x + y;
                        sm = min(sm, sm - pr.q2);
                        const uint64_t d = x - y + pr.q2;
                        x = sm;
                        y = shoup_lazy(d, w, ws, pr.q);
                    }
                }
            }
        }
    }
    // Each thread writes back exactly the positions it read: no barrier
    // is needed between this pass's reads and writes.
#pragma unroll
    for (int gi = 0; gi < G; ++gi) {
        const int j0 = group_start<S>(threadIdx.x + T * gi, lu, lnb);
        const int p0 = pad_idx(j0);
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const int j = j0 + (k << lu);
            const int idx = p0 + pad_off(k, lu);
            uint64_t x = v[gi * W + k];
            if (last) {
                if constexpr (MAC) {
                    // any representative: the Montgomery product reduces it
                    const uint64_t m0 = mont_mul(x, mk->k0[j], pr.q, mk->qinv);
                    const uint64_t m1 = mont_mul(x, mk->k1[j], pr.q, mk->qinv);
                    mk->acc0[idx] = mk->assign ? m0 : add_mod(mk->acc0[idx], m0, pr.q);
                    mk->acc1[idx] = mk->assign ? m1 : add_mod(mk->acc1[idx], m1, pr.q);
                } else {
                    if (FWD) {
                        if (GROW) {
                            x = barrett_u64(x, pr.q, pr.mu);
                        } else {
                            x = x >= pr.q2 ? x - pr.q2 : x;
                            x = x >= pr.q ? x - pr.q : x;
                        }
                    } else {
                        x = shoup_mulmod(x, pr.ninv, pr.ninv_s, pr.q);
                    }
                    gout[j] = x;
                }
            } else {
                sa[idx] = x;
            }
        }
    }
    if (!last) __syncthreads();
}

// Stages of pass pi when logN stages run in `passes` passes: as even as
// possible, the longer passes first (13 stages in 4 passes: 4, 3, 3, 3).
__host__ __device__ constexpr int pass_stages(int logN, int passes, int pi) {
    return logN / passes + (pi < logN % passes ? 1 : 0);
}

// E coefficients per thread (N / E threads), passes of up to log2(E) stages.
template <int E>
struct NttShape {
    static constexpr int kLogE = E == 8 ? 3 : (E == 16 ? 4 : 5);
    static constexpr int kMaxThreads = E == 8 ? 1024 : 512;
};

// The passes of one transform with the degree fixed at compile time
// (N = 2^LOGN): each pass's stage count, distance and first/last role are
// constants, so the index arithmetic of ntt_pass folds away.  Same passes
// and arithmetic as ntt_run.
template <int E, bool FWD, bool MAC, bool GROW, int LOGN, bool TWO = false, int PI = 0,
          int DONE = 0>
__device__ __forceinline__ void ntt_run_c(uint64_t *sa, const uint64_t *gin, uint64_t *gout,
                                          bool reduce_in, const PlaneRegs &pr, bool from_smem,
                                          const MacSink *mk, const DigitSrc *ds = nullptr) {
    constexpr int SM = NttShape<E>::kLogE;
    constexpr int PASSES = (LOGN + SM - 1) / SM;
    constexpr int S = pass_stages(LOGN, PASSES, PI);
    constexpr bool LAST = DONE + S == LOGN;
    constexpr int LU = FWD ? LOGN - DONE - S : DONE;
    ntt_pass<E, S, FWD, MAC, GROW, TWO && PI == 0>(sa, gin, gout, reduce_in, 1 << LOGN, LOGN, LU,
                                                   PI == 0 && !from_smem, LAST, pr, mk, ds);
    if constexpr (!LAST)
        ntt_run_c<E, FWD, MAC, GROW, LOGN, TWO, PI + 1, DONE + S>(sa, gin, gout, reduce_in, pr,
                                                                  from_smem, mk, ds);
}

// LOGN > 0: the degree is 2^LOGN, known at compile time (ntt_run_c); 0: a.N
// at run time.
template <int E, bool FWD, int LOGN = 0>
__global__ void __launch_bounds__(NttShape<E>::kMaxThreads, 1) ntt_e_kernel(NttFastArgs a) {
    constexpr int SM = NttShape<E>::kLogE;
    extern __shared__ uint64_t sa[];
    const int64_t p = blockIdx.x;
    const int N = a.N;
    int plane;
    const uint64_t *gin;
    DigitSrc dsrc{};
    const DigitSrc *ds = nullptr;
    if (FWD && a.ks_ct) {
        const int Lp = a.g.L + a.g.K;
        plane = static_cast<int>(p % Lp);
        const int64_t r = p / Lp;
        const int d = static_cast<int>(r % a.g.D);
        const int64_t c = r / a.g.D;
        gin = a.ks_ct + (static_cast<int64_t>(gadget_lo(a.g, d)) * a.ks_n + a.ks_c0 + c) * N;
        dsrc = make_digit_src(a.g, gin, a.ks_v ? a.ks_v + (c * a.g.D + d) * N : nullptr, d,
                              plane);
        ds = &dsrc;
    } else {
        plane = static_cast<int>((p / a.inner) % a.nplanes);
        gin = a.polys + p * N;
    }
    const NttPlane &tp = a.tab[plane];
    PlaneRegs pr;
    pr.q = tp.q;
    pr.q2 = 2 * tp.q;
    pr.q4 = 4 * tp.q;
    pr.mu = tp.mu;
    pr.ninv = tp.ninv;
    pr.ninv_s = tp.ninv_s;
    pr.tw = FWD ? tp.fwd2 : tp.inv2;
    const bool reduce_in = FWD && a.ks_ct != nullptr;
    uint64_t *gout = a.polys + p * N;
    if constexpr (LOGN > 0) {
        // Uniform per CTA (one plane, one modulus).  Unreduced key-switch
        // digits stay below digit_bound.
        const uint64_t in_max = reduce_in ? digit_bound(a.g, pr.q) : 0;
        const bool grow = FWD ? ntt_grow_ok_fwd(pr.q, in_max, LOGN) : ntt_grow_ok_inv(pr.q, LOGN);
        // One-prime digits read gin itself (a0 of the digit source).
        if (ds && dsrc.v1) {
            if (grow)
                ntt_run_c<E, FWD, false, true, LOGN, true>(sa, gin, gout, false, pr, false,
                                                           nullptr, ds);
            else
                ntt_run_c<E, FWD, false, false, LOGN, true>(sa, gin, gout, reduce_in, pr, false,
                                                            nullptr, ds);
        } else {
            if (grow)
                ntt_run_c<E, FWD, false, true, LOGN>(sa, gin, gout, false, pr, false, nullptr);
            else
                ntt_run_c<E, FWD, false, false, LOGN>(sa, gin, gout, reduce_in, pr, false,
                                                      nullptr);
        }
        return;
    }
    const int logN = a.logN;
    const int passes = (logN + SM - 1) / SM;
    int done = 0;
    bool first = true;
    for (int pi = 0; done < logN; ++pi) {
        const int s = pass_stages(logN, passes, pi);
        const bool last = done + s == logN;
        // forward: distances fall from N/2; inverse: they rise from 1
        const int lu = FWD ? logN - done - s : done;
        if (s == SM) {
            ntt_pass<E, SM, FWD>(sa, gin, gout, reduce_in, N, logN, lu, first, last, pr, nullptr,
                                  ds);
        } else if (s == 4) {
            ntt_pass<E, (SM > 4 ? 4 : 1), FWD>(sa, gin, gout, reduce_in, N, logN, lu, first, last, pr, nullptr,
                                  ds);
        } else if (s == 3) {
            ntt_pass<E, (SM > 3 ? 3 : 1), FWD>(sa, gin, gout, reduce_in, N, logN, lu, first, last, pr, nullptr,
                                  ds);
        } else if (s == 2) {
            ntt_pass<E, 2, FWD>(sa, gin, gout, reduce_in, N, logN, lu, first, last, pr, nullptr,
                                  ds);
        } else {
            ntt_pass<E, 1, FWD>(sa, gin, gout, reduce_in, N, logN, lu, first, last, pr, nullptr,
                                  ds);
        }
        done += s;
        first = false;
    }
}

// All passes of one transform held in `sa`: the first reads gin (or `sa`
// itself when from_smem), the last writes gout (or the MAC sink).
template <int E, bool FWD, bool MAC, bool GROW = false>
__device__ __forceinline__ void ntt_run(uint64_t *sa, const uint64_t *gin, uint64_t *gout,
                                        bool reduce_in, int N, int logN, const PlaneRegs &pr,
                                        bool from_smem, const MacSink *mk,
                                        const DigitSrc *ds = nullptr) {
    constexpr int SM = NttShape<E>::kLogE;
    const int passes = (logN + SM - 1) / SM;
    int done = 0;
    bool first = !from_smem;
    for (int pi = 0; done < logN; ++pi) {
        const int s = pass_stages(logN, passes, pi);
        const bool last = done + s == logN;
        const int lu = FWD ? logN - done - s : done;
        if (s == SM) {
            ntt_pass<E, SM, FWD, MAC, GROW>(sa, gin, gout, reduce_in, N, logN, lu, first, last, pr, mk, ds);
        } else if (s == 4) {
            ntt_pass<E, (SM > 4 ? 4 : 1), FWD, MAC, GROW>(sa, gin, gout, reduce_in, N, logN, lu, first,
                                                    last, pr, mk, ds);
        } else if (s == 3) {
            ntt_pass<E, (SM > 3 ? 3 : 1), FWD, MAC, GROW>(sa, gin, gout, reduce_in, N, logN, lu, first,
                                                    last, pr, mk, ds);
        } else if (s == 2) {
            ntt_pass<E, 2, FWD, MAC, GROW>(sa, gin, gout, reduce_in, N, logN, lu, first, last, pr, mk, ds);
        } else {
            ntt_pass<E, 1, FWD, MAC, GROW>(sa, gin, gout, reduce_in, N, logN, lu, first, last, pr, mk, ds);
        }
        done += s;
        first = false;
    }
}

struct KsFusedArgs {
    const uint64_t *ct;  // batch [2][L][n][N]; digits come from the a-parts
    int64_t n, c0;
    int N, logN;
    const NttPlane *tab;
    KsGadget g;
    const uint64_t *V;     // Garner digits of two-prime digits, [nb][D][N]
    const uint64_t *keys;  // [count][D][2][L+K][N], prepared
    const int *kid;
    int kper;
    uint64_t *U;  // [nb][2][L+K][N]: sum_d digit_d * key_d[part] mod q_k, coefficients
};

// Key switching's digits, products and sums for one (ciphertext, target
// prime k) per CTA, in shared memory: for every gadget digit d the forward
// transform of (digit d mod q_k), multiplied in its last pass by key d (both
// parts) and summed into two accumulators; then both inverse transforms,
// written to U.  Shared memory: three padded polynomials (N <= 8192).
template <int E, int LOGN = 0>
__global__ void __launch_bounds__(NttShape<E>::kMaxThreads, 1) ks_fused_kernel(KsFusedArgs a) {
    extern __shared__ uint64_t smem[];
    const int N = a.N;
    const int Wd = N + N / 32;
    uint64_t *sa = smem, *acc0 = smem + Wd, *acc1 = smem + 2 * Wd;
    const int Lp = a.g.L + a.g.K;
    const int k = static_cast<int>(blockIdx.x % Lp);
    const int64_t c = blockIdx.x / Lp;
    const int kc = a.kid[(a.c0 + c) % a.kper];
    if (kc < 0) return;  // no key switch for this ciphertext (uniform per CTA)
    const NttPlane &tp = a.tab[k];
    PlaneRegs fw, iv;
    fw.q = iv.q = tp.q;
    fw.q2 = iv.q2 = 2 * tp.q;
    fw.q4 = iv.q4 = 4 * tp.q;
    fw.mu = iv.mu = tp.mu;
    fw.ninv = iv.ninv = tp.ninv;
    fw.ninv_s = iv.ninv_s = tp.ninv_s;
    fw.tw = tp.fwd2;
    iv.tw = tp.inv2;
    const int64_t key_stride = static_cast<int64_t>(a.g.D) * 2 * Lp * N;
    const uint64_t *key = a.keys + kc * key_stride;
    const bool grow_f = ntt_grow_ok_fwd(tp.q, digit_bound(a.g, tp.q), a.logN);
    for (int d = 0; d < a.g.D; ++d) {
        const uint64_t *gin =
            a.ct + (static_cast<int64_t>(gadget_lo(a.g, d)) * a.n + a.c0 + c) * N;
        const DigitSrc ds =
            make_digit_src(a.g, gin, a.V ? a.V + (c * a.g.D + d) * N : nullptr, d, k);
        MacSink mk{acc0, acc1, key + (static_cast<int64_t>(d * 2 + 0) * Lp + k) * N,
                   key + (static_cast<int64_t>(d * 2 + 1) * Lp + k) * N, tp.qinv_neg, d == 0};

        if constexpr (LOGN > 0) {
            if (ds.v1) {  // two-prime digit
                if (grow_f)  // unreduced digits
                    ntt_run_c<E, true, true, true, LOGN, true>(sa, gin, nullptr, false, fw, false,
                                                               &mk, &ds);
                else
                    ntt_run_c<E, true, true, false, LOGN, true>(sa, gin, nullptr, true, fw, false,
                                                                &mk, &ds);
            } else {
                if (grow_f)
                    ntt_run_c<E, true, true, true, LOGN>(sa, gin, nullptr, false, fw, false, &mk);
                else
                    ntt_run_c<E, true, true, false, LOGN>(sa, gin, nullptr, true, fw, false, &mk);
            }
        } else {
            ntt_run<E, true, true>(sa, gin, nullptr, true, N, a.logN, fw, false, &mk, &ds);
        }
        __syncthreads();  // sa is rewritten by the next digit; acc read by the inverse
    }
    uint64_t *u0 = a.U + ((c * 2 + 0) * Lp + k) * N;
    uint64_t *u1 = a.U + ((c * 2 + 1) * Lp + k) * N;
    if (LOGN > 0 && ntt_grow_ok_inv(tp.q, a.logN)) {
        ntt_run<E, false, false, true>(acc0, nullptr, u0, false, N, a.logN, iv, true, nullptr);
        ntt_run<E, false, false, true>(acc1, nullptr, u1, false, N, a.logN, iv, true, nullptr);
    } else {
        ntt_run<E, false, false>(acc0, nullptr, u0, false, N, a.logN, iv, true, nullptr);
        ntt_run<E, false, false>(acc1, nullptr, u1, false, N, a.logN, iv, true, nullptr);
    }
}

// Coefficients per thread for degree N: 8 up to N = 8192 (measured best of
// 8 / 16 / 32 on the CC-MM n=8192 key switches), 32 above
// (MODPP_NTT_E = 8, 16 or 32 overrides where the thread count allows).
int ntt_e_for(int N) {
    static const int forced = [] {
        const char *v = std::getenv("MODPP_NTT_E");
        return v ? std::atoi(v) : 0;
    }();
    int e = (forced == 8 || forced == 16 || forced == 32) ? forced : (N <= 8192 ? 8 : 32);
    if (e == 8 && N / 8 > NttShape<8>::kMaxThreads) e = 16;
    if (e == 16 && N / 16 > NttShape<16>::kMaxThreads) e = 32;
    return e;
}

template <int E, bool FWD, int LOGN>
cudaError_t launch_e_kernel(const NttFastArgs &a, int64_t npolys, cudaStream_t s) {
    const int threads = a.N / E;
    const size_t smem = static_cast<size_t>(a.N + a.N / 32) * sizeof(uint64_t);
    cudaError_t e = cudaFuncSetAttribute(ntt_e_kernel<E, FWD, LOGN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    ntt_e_kernel<E, FWD, LOGN><<<static_cast<unsigned>(npolys), threads, smem, s>>>(a);
    return cudaGetLastError();
}

// The degree as a compile-time constant for the default shapes (8
// coefficients per thread up to 2^13, 32 at 2^14); the run-time kernel
// otherwise.
template <int E, bool FWD>
cudaError_t launch_e(const NttFastArgs &a, int64_t npolys, cudaStream_t s) {
    if constexpr (E == 8) {
        switch (a.logN) {
            case 10: return launch_e_kernel<8, FWD, 10>(a, npolys, s);
            case 11: return launch_e_kernel<8, FWD, 11>(a, npolys, s);
            case 12: return launch_e_kernel<8, FWD, 12>(a, npolys, s);
            case 13: return launch_e_kernel<8, FWD, 13>(a, npolys, s);
            default: break;
        }
    }
    if constexpr (E == 32)
        if (a.logN == 14) return launch_e_kernel<32, FWD, 14>(a, npolys, s);
    return launch_e_kernel<E, FWD, 0>(a, npolys, s);
}

template <bool FWD>
cudaError_t launch_fast(const NttFastArgs &a, int64_t npolys, cudaStream_t s) {
    switch (ntt_e_for(a.N)) {
        case 8: return launch_e<8, FWD>(a, npolys, s);
        case 16: return launch_e<16, FWD>(a, npolys, s);
        default: return launch_e<32, FWD>(a, npolys, s);
    }
}

}  // namespace

// Coefficients per thread of the fused key switch (N / kKsE threads per CTA).
constexpr int kKsE = 8;

bool ks_fused_supported(int N) { return N >= 1024 && N <= 8192 && (N & (N - 1)) == 0; }

cudaError_t launch_ks_fused(const uint64_t *ct, int64_t n, int N, int64_t c0, int64_t nb,
                            const NttPlane *tab, const KsGadget &g, const uint64_t *V,
                            const uint64_t *keys, const int *kid, int kper, uint64_t *U,
                            cudaStream_t s) {
    if (nb == 0) return cudaSuccess;
    KsFusedArgs a{};
    a.V = V;
    a.ct = ct;
    a.n = n;
    a.c0 = c0;
    a.g = g;
    a.N = N;
    a.logN = 31 - __builtin_clz(N);
    a.tab = tab;
    a.keys = keys;
    a.kid = kid;
    a.kper = kper;
    a.U = U;
    const size_t smem = 3 * static_cast<size_t>(N + N / 32) * sizeof(uint64_t);
    const dim3 grid(static_cast<unsigned>(nb * (g.L + g.K)));
    auto go = [&](auto kernel) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        kernel<<<grid, N / kKsE, smem, s>>>(a);
        return cudaGetLastError();
    };
    switch (a.logN) {  // the degree as a compile-time constant (1024 <= N <= 8192)
        case 10: return go(ks_fused_kernel<kKsE, 10>);
        case 11: return go(ks_fused_kernel<kKsE, 11>);
        case 12: return go(ks_fused_kernel<kKsE, 12>);
        case 13: return go(ks_fused_kernel<kKsE, 13>);
        default: return go(ks_fused_kernel<kKsE, 0>);
    }
}

bool ntt_fast_supported(int N) { return N >= 1024 && N <= 16384 && (N & (N - 1)) == 0; }

cudaError_t launch_ntt_fast(uint64_t *polys, int64_t npolys, int N, int64_t inner, int nplanes,
                            const NttPlane *tab, bool inverse, cudaStream_t s) {
    if (npolys == 0) return cudaSuccess;
    NttFastArgs a{};
    a.polys = polys;
    a.N = N;
    a.logN = 0;
    while ((1 << a.logN) < N) ++a.logN;
    a.inner = inner;
    a.nplanes = nplanes;
    a.tab = tab;
    return inverse ? launch_fast<false>(a, npolys, s) : launch_fast<true>(a, npolys, s);
}

cudaError_t launch_ks_digits_ntt(const uint64_t *ct, int64_t n, int N, int64_t c0, int64_t nb,
                                 const NttPlane *tab, const KsGadget &g, const uint64_t *V,
                                 uint64_t *D, cudaStream_t s) {
    if (nb == 0) return cudaSuccess;
    NttFastArgs a{};
    a.polys = D;
    a.N = N;
    a.logN = 0;
    while ((1 << a.logN) < N) ++a.logN;
    a.inner = 1;
    a.nplanes = g.L + g.K;
    a.tab = tab;
    a.ks_ct = ct;
    a.ks_n = n;
    a.ks_c0 = c0;
    a.ks_v = V;
    a.g = g;
    return launch_fast<true>(a, nb * g.D * (g.L + g.K), s);
}

}  // namespace modpp
