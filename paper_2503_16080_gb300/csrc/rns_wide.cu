// Multi-modular (CRT) form of the wide Mod-PP-MM: C_j = U_j * A_j mod q_j
// when both operands are full residues (the products of Alg. 8, step 2).
//
// Both operands are lifted to balanced integers (|x| <= (q-1)/2), so the
// exact product X = U * A has |X| <= k ((q-1)/2)^2.  Instead of splitting
// both operands into digits (LU x LA digit products), X is computed modulo R
// small primes p_i whose product M exceeds 2 |X| with margin: one tensor-core
// product per p_i on the balanced residues of U and A modulo p_i, then the
// Chinese remainder theorem recovers X and reduces it modulo q_j.  This is
// the exact (lifting) variant of Strategy 3 of Sec. 6.1, with primes small
// enough for the f16 tensor cores.
//
// Exactness: residues satisfy |r| <= (p-1)/2 <= B with k B^2 < 2^24, so every
// FP32 sum of the product is an exact integer (no chunks), and the GEMM
// epilogue (mode 1 of gemm_f16_kernel) stores the balanced residue of X mod
// p_i as int8.  CRT (with y_i = r_i (M/p_i)^-1 mod p_i):
//   X = sum_i y_i (M/p_i) - alpha M,  alpha = round(sum_i y_i / p_i),
// valid because |X| / M < 0.36 leaves the rounding a margin far above the
// binary32 error of the 32-term sum; then
//   X mod q = sum_i y_i ((M/p_i) mod q) - alpha (M mod q)  (mod q).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "gemm_f16_kernel.cuh"
#include "modarith.cuh"
#include "modpp_internal.h"
#include "rns_wide.h"

namespace modpp {

namespace {

constexpr int kRnsNC = kRnsTileCols;  // output columns per tile (UMMA N = 256)
constexpr int kRnsT = 64;     // inner indices per split tile

// n mod p for n < 2^32 and p < 2^16, given mag = floor(2^32 / p): the
// quotient estimate __umulhi(n, mag) is low by at most one.
__device__ __forceinline__ uint32_t mod_small(uint32_t n, uint32_t p, uint32_t mag) {
    uint32_t r = n - __umulhi(n, mag) * p;
    return r >= p ? r - p : r;
}

// A balanced lift x (|x| < 2^62) as sign and three 21-bit limbs of |x|, so
// that |x| mod p = (m2 2^42 + m1 2^21 + m0) mod p needs one small reduction
// of m2 (2^42 mod p) + m1 (2^21 mod p) + m0 < 2^30 per prime.
struct Limbs {
    uint32_t m0, m1, m2;
    bool neg;
};
__device__ __forceinline__ Limbs to_limbs(int64_t x) {
    const uint64_t m = x < 0 ? static_cast<uint64_t>(-x) : static_cast<uint64_t>(x);
    return Limbs{static_cast<uint32_t>(m & 0x1fffffu), static_cast<uint32_t>((m >> 21) & 0x1fffffu),
                 static_cast<uint32_t>(m >> 42), x < 0};
}

// Balanced residue of |x| in [-(p-1)/2, (p-1)/2] (the caller applies x's sign).
__device__ __forceinline__ int bal_mod_abs(const Limbs &l, const RnsPrime &pp) {
    int v = static_cast<int>(mod_small(l.m2 * pp.t42 + l.m1 * pp.t21 + l.m0, pp.p, pp.mag));
    if (2 * v > static_cast<int>(pp.p)) v -= static_cast<int>(pp.p);
    return v;
}

// f16 bits of two small integers |v| < 512, as a half2 word: 1536 + v lies
// in [1024, 2048), where f16 values are the integers, so its bit pattern is
// 0x6600 + v, and subtracting 1536 in f16 is exact.  sign: 0x8000 in the
// half of each value to negate (a negated zero is -0, which multiplies and
// adds as 0).
__device__ __forceinline__ uint32_t small_half2(int v0, int v1, uint32_t sign) {
    const uint32_t biased = static_cast<uint32_t>(0x6600 + v0) |
                            (static_cast<uint32_t>(0x6600 + v1) << 16);
    __half2 h = *reinterpret_cast<const __half2 *>(&biased);
    h = __hsub2(h, __float2half2_rn(1536.0f));
    return *reinterpret_cast<const uint32_t *>(&h) ^ sign;
}

// U (d x k residues mod q, leading dimension ldu) -> R planes of balanced
// residues mod p_i as f16, plane i rows [i d, (i+1) d) of a (R d) x kp matrix
// (zero padded for t >= k).  One thread takes 8 consecutive entries of a row
// (kp is a multiple of 8) and writes one 16-byte word per prime.
__global__ void __launch_bounds__(256) rns_split_u_kernel(const uint64_t *__restrict__ U,
                                                          int64_t ldu, int d, int k, int kp,
                                                          uint64_t q, RnsPrimes pr,
                                                          __half *__restrict__ U16) {
    const int gpr = kp >> 3;  // groups of 8 per row
    const int64_t groups = static_cast<int64_t>(d) * gpr;
    const int64_t plane = static_cast<int64_t>(d) * kp;
    const uint64_t half_q = q >> 1;
    const bool vec = (reinterpret_cast<uintptr_t>(U) & 15u) == 0 && (ldu & 1) == 0;
    for (int64_t g = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; g < groups;
         g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = g / gpr;
        const int t = static_cast<int>(g - r * gpr) << 3;
        const uint64_t *row = U + r * ldu + t;
        uint64_t u[8];
        if (vec && t + 8 <= k) {
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
                const ulonglong2 w = *reinterpret_cast<const ulonglong2 *>(row + j);
                u[j] = w.x;
                u[j + 1] = w.y;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) u[j] = t + j < k ? row[j] : 0;
        }
        Limbs l[8];
        uint32_t sign[4] = {0, 0, 0, 0};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int64_t x = u[j] > half_q ? static_cast<int64_t>(u[j]) - static_cast<int64_t>(q)
                                            : static_cast<int64_t>(u[j]);
            l[j] = to_limbs(x);
            if (l[j].neg) sign[j >> 1] |= (j & 1) ? 0x80000000u : 0x8000u;
        }
        __half *out = U16 + r * kp + t;
        for (int i = 0; i < pr.R; ++i) {
            const RnsPrime pp = pr.p[i];
            uint4 w;
            w.x = small_half2(bal_mod_abs(l[0], pp), bal_mod_abs(l[1], pp), sign[0]);
            w.y = small_half2(bal_mod_abs(l[2], pp), bal_mod_abs(l[3], pp), sign[1]);
            w.z = small_half2(bal_mod_abs(l[4], pp), bal_mod_abs(l[5], pp), sign[2]);
            w.w = small_half2(bal_mod_abs(l[6], pp), bal_mod_abs(l[7], pp), sign[3]);
            *reinterpret_cast<uint4 *>(out + i * plane) = w;
        }
    }
}

// A (k x n residues mod q, leading dimension lda) -> R K-major planes: row
// (i * nblk + c / 256) * 256 + c % 256 holds column c of A's residues mod
// p_i over the inner index (kp halves per row).  One block per 64 x 64 tile:
// thread (column cl, quarter tq) reads 16 consecutive inner indices of its
// column (a warp reads 32 neighbouring columns of one row), packs their
// residues into two 16-byte words of the transposed shared tile, and 8
// threads per 128-byte row write the tile out along the inner index.
__global__ void __launch_bounds__(256) rns_split_a_kernel(const uint64_t *__restrict__ A,
                                                          int64_t lda, int k, int n, int kp,
                                                          int nblk, uint64_t q, RnsPrimes pr,
                                                          __half *__restrict__ D) {
    constexpr int kRow = kRnsT + 8;  // padded tile row (halves): 144 bytes
    __shared__ __align__(16) __half tile[64 * kRow];
    const int t0 = blockIdx.x * kRnsT;
    const int c0 = blockIdx.y * 64;
    const uint64_t half_q = q >> 1;
    const int cl = threadIdx.x & 63;
    const int tq = (threadIdx.x >> 6) * 16;
    Limbs x[16];
    uint32_t sign[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        const int t = t0 + tq + s, c = c0 + cl;
        int64_t v = 0;
        if (t < k && c < n) {
            const uint64_t a = A[static_cast<int64_t>(t) * lda + c];
            v = a > half_q ? static_cast<int64_t>(a) - static_cast<int64_t>(q)
                           : static_cast<int64_t>(a);
        }
        x[s] = to_limbs(v);
        if (x[s].neg) sign[s >> 1] |= (s & 1) ? 0x80000000u : 0x8000u;
    }
    const int sub = threadIdx.x & 7;   // 8 threads per 128-byte row, 8 halves each
    const int t = t0 + 8 * sub;
    uint4 *dst = reinterpret_cast<uint4 *>(&tile[cl * kRow + tq]);
    for (int i = 0; i < pr.R; ++i) {
        const RnsPrime pp = pr.p[i];
        uint32_t w[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            w[j] = small_half2(bal_mod_abs(x[2 * j], pp), bal_mod_abs(x[2 * j + 1], pp), sign[j]);
        dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
        dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
        __syncthreads();
        if (t < kp) {
            for (int row = threadIdx.x >> 3; row < 64; row += 32) {
                const int c = c0 + row;
                const int64_t drow =
                    (static_cast<int64_t>(i) * nblk + c / kRnsNC) * kRnsNC + (c % kRnsNC);
                const uint4 v = *reinterpret_cast<const uint4 *>(&tile[row * kRow + 8 * sub]);
                *reinterpret_cast<uint4 *>(D + drow * kp + t) = v;
            }
        }
        __syncthreads();
    }
}

// C[r][c] = X mod q from the R balanced residues res[i][r][c] (int8, plane
// stride d * n, row stride n).  Per small prime one shared-memory word,
// indexed by the residue r, holds y = r c_i mod p_i in its top 8 bits and
// y / p_i in 0.24 fixed point below (one table read per prime: the reads
// are at data-dependent addresses, so bank conflicts make them the cost).
// The sum S = sum_i y_i w_i (w_i = (M / p_i) mod q) is one 64-bit word when
// R (p_max - 1) (q - 1) < 2^64 (ONE: 50-bit chain primes), else two 64-bit
// halves, S = S_hi 2^32 + S_lo with w_i = w_hi 2^32 + w_lo (y_i w_lo < 2^40,
// y_i w_hi < 2^38: no overflow for R <= 32); either way it is reduced modulo
// q once.  alpha = round(sum_i
// y_i / p_i) from the fixed-point parts (rounding error below 2^-19 against
// the 0.14 margin of |X| / M < 0.36).  Four consecutive outputs per thread
// (n % 4 == 0) with 32-bit residue loads; one otherwise.
template <int V, bool ONE>
__global__ void __launch_bounds__(256) rns_crt_kernel(const int8_t *__restrict__ res, int d, int n,
                                                      RnsCrt cr, uint64_t *__restrict__ C,
                                                      int64_t ldc) {
    __shared__ uint32_t ytab[kMaxRnsPrimes][256];
    for (int e = threadIdx.x; e < cr.R * 256; e += blockDim.x) {
        const int i = e >> 8, r = (e & 255) - 128;  // residue r in [-128, 127]
        const int p = cr.p[i];
        int y = (r * cr.c[i]) % p;
        if (y < 0) y += p;
        const uint32_t frac = static_cast<uint32_t>(
            (static_cast<uint64_t>(y) << 24) / static_cast<uint64_t>(p) +
            ((((static_cast<uint64_t>(y) << 24) % static_cast<uint64_t>(p)) * 2 >=
              static_cast<uint64_t>(p))
                 ? 1u
                 : 0u));
        ytab[i][e & 255] = (static_cast<uint32_t>(y) << 24) | frac;
    }
    __syncthreads();
    const uint64_t q = cr.q;
    const int64_t total = static_cast<int64_t>(d) * n;
    const int64_t groups = total / V;
    for (int64_t g = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; g < groups;
         g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t e0 = g * V;
        uint64_t slo[V], shi[V];
        uint32_t F[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            slo[v] = 0;
            shi[v] = 0;
            F[v] = 0;
        }
        // Residue words in batches of 8 primes: eight loads in flight, then
        // their sums.
        for (int i0 = 0; i0 < cr.R; i0 += 8) {
            uint32_t words[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u;
                if (i >= cr.R) break;
                const int8_t *rp = res + static_cast<int64_t>(i) * total + e0;
                words[u] = V == 4 ? *reinterpret_cast<const uint32_t *>(rp)
                                  : static_cast<uint32_t>(static_cast<uint8_t>(rp[0]));
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u;
                if (i >= cr.R) break;
                const uint32_t wl = cr.wlo[i], wh = cr.whi[i];
                const uint64_t w = (static_cast<uint64_t>(wh) << 32) | wl;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const uint32_t idx = ((words[u] >> (8 * v)) & 0xffu) ^ 0x80u;  // r + 128
                    const uint32_t t = ytab[i][idx];
                    const uint32_t y = t >> 24;
                    if constexpr (ONE) {
                        slo[v] += y * w;
                    } else {
                        slo[v] += static_cast<uint64_t>(y) * wl;
                        shi[v] += static_cast<uint64_t>(y) * wh;
                    }
                    F[v] += t & 0xffffffu;
                }
            }
        }
        // The V outputs share one row (n % V == 0): one division per thread.
        const int64_t row = e0 / n;
        uint64_t *out = C + row * ldc + (e0 - row * n);
        uint64_t x[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            if constexpr (ONE) {
                x[v] = barrett_u64(slo[v], q, cr.mu);  // S itself fits 64 bits
            } else {
                // S mod q = (S_hi mod q) 2^32 + S_lo (mod q)
                x[v] = shoup_mulmod(barrett_u64(shi[v], q, cr.mu), cr.t32, cr.t32s, q);
                x[v] = add_mod(x[v], barrett_u64(slo[v], q, cr.mu), q);
            }
            const uint64_t alpha = (F[v] + (1u << 23)) >> 24;
            x[v] = sub_mod(x[v], shoup_mulmod(alpha, cr.mq, cr.mqs, q), q);
        }
        if (V == 4 && (reinterpret_cast<uintptr_t>(out) & 15u) == 0) {
            *reinterpret_cast<ulonglong2 *>(out) = make_ulonglong2(x[0], x[1 % V]);
            *reinterpret_cast<ulonglong2 *>(out + 2) = make_ulonglong2(x[2 % V], x[3 % V]);
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) out[v] = x[v];
        }
    }
}

uint64_t host_mulmod_u(uint64_t a, uint64_t b, uint64_t m) {
    return static_cast<uint64_t>((static_cast<unsigned __int128>(a) * b) % m);
}
uint64_t host_powmod_u(uint64_t b, uint64_t e, uint64_t m) {
    uint64_t r = 1 % m;
    b %= m;
    while (e) {
        if (e & 1) r = host_mulmod_u(r, b, m);
        b = host_mulmod_u(b, b, m);
        e >>= 1;
    }
    return r;
}
bool small_prime(int p) {
    if (p < 3 || (p & 1) == 0) return false;
    for (int f = 3; f * f <= p; f += 2)
        if (p % f == 0) return false;
    return true;
}

}  // namespace

namespace {
// Primes below 2B+1, largest first, until their product reaches 2^need.
bool pick_primes(int64_t B, long double need, RnsPrimes *r) {
    long double have = 0;
    r->R = 0;
    for (int p = static_cast<int>(2 * B + 1); p >= 3 && have < need; --p) {
        if (!small_prime(p)) continue;
        if (r->R == kMaxRnsPrimes) return false;
        RnsPrime &pp = r->p[r->R++];
        pp.p = static_cast<uint32_t>(p);
        pp.mag = static_cast<uint32_t>((uint64_t(1) << 32) / static_cast<uint64_t>(p));
        pp.t21 = static_cast<uint32_t>((uint64_t(1) << 21) % static_cast<uint64_t>(p));
        pp.t42 = static_cast<uint32_t>((uint64_t(1) << 42) % static_cast<uint64_t>(p));
        have += std::log2(static_cast<long double>(p));
    }
    return have >= need;
}
// Largest B with len B^2 < 2^24, capped.
int64_t residue_bound(int64_t len, int64_t cap) {
    int64_t B = static_cast<int64_t>(std::floor(std::sqrt(static_cast<double>((1 << 24) - 1) /
                                                          static_cast<double>(len))));
    while (B > 0 && len * B * B >= (int64_t(1) << 24)) --B;
    return B > cap ? cap : B;
}
}  // namespace

bool rns_choose(int64_t k, const uint64_t *qs, int P, RnsPrimes *out) {
    if (k <= 0 || P < 1) return false;
    uint64_t qmax = 0;
    for (int j = 0; j < P; ++j) qmax = qs[j] > qmax ? qs[j] : qmax;
    // Need M >= 2.8 k ((qmax - 1) / 2)^2 (then |X| / M < 0.36).
    const long double need = std::log2(2.8L) + std::log2(static_cast<long double>(k)) +
                             2.0L * std::log2(static_cast<long double>((qmax - 1) / 2 + 1));
    // One to kMaxRnsChunks pieces of the inner dimension (each piece's sums
    // exact: len B^2 < 2^24; every piece after the first adds into the
    // stored residues and reduces again, so |r| <= 125 holds for int8).
    // Cost model: products R, plus 5% per extra piece (the epilogue's
    // residue read-back and a shorter K loop per tile).
    bool found = false;
    double best = 0;
    for (int c = 1; c <= kMaxRnsChunks; ++c) {
        int64_t len = k;
        if (c > 1) {
            len = ((k + c - 1) / c + 63) / 64 * 64;
            if ((c - 1) * len >= k) continue;  // fewer real pieces than c
        }
        const int64_t B = residue_bound(len, 125);
        if (B < 1) continue;
        RnsPrimes r{};
        if (!pick_primes(B, need, &r)) continue;
        r.chunks = c;
        r.chunk_len = len;
        const double cost = r.R * (1.0 + 0.05 * (c - 1));
        if (!found || cost < best) {
            *out = r;
            best = cost;
            found = true;
        }
    }
    return found;
}

RnsCrt rns_crt_consts(const RnsPrimes &pr, uint64_t q) {
    RnsCrt c{};
    c.R = pr.R;
    c.chunks = 1;  // later chunks add into the first chunk's residues in the GEMM epilogue
    c.q = q;
    uint64_t mq = 1 % q;
    for (int i = 0; i < pr.R; ++i) mq = host_mulmod_u(mq, pr.p[i].p, q);
    c.mq = mq;
    c.mqs = host_shoup(mq, q);
    c.mu = host_barrett_mu(q);
    c.t32 = (uint64_t(1) << 32) % q;
    c.t32s = host_shoup(c.t32, q);
    for (int i = 0; i < pr.R; ++i) {
        const uint64_t p = pr.p[i].p;
        uint64_t wq = 1 % q, wp = 1;  // (M / p_i) mod q and mod p_i
        for (int l = 0; l < pr.R; ++l) {
            if (l == i) continue;
            wq = host_mulmod_u(wq, pr.p[l].p, q);
            wp = host_mulmod_u(wp, pr.p[l].p, p);
        }
        c.p[i] = static_cast<int>(p);
        c.c[i] = static_cast<int>(host_powmod_u(wp, p - 2, p));  // (M/p_i)^-1 mod p_i
        c.wlo[i] = static_cast<uint32_t>(wq & 0xffffffffu);
        c.whi[i] = static_cast<uint32_t>(wq >> 32);
    }
    return c;
}

RnsLayout rns_layout(int64_t d, int64_t k, int64_t n, const RnsPrimes &pr) {
    const int R = pr.R;
    RnsLayout l{};
    l.kp = (k + 7) / 8 * 8;
    l.nblk = (n + kRnsNC - 1) / kRnsNC;
    size_t off = 256;  // status word
    l.off_u16 = off;
    off += static_cast<size_t>(R) * d * l.kp * 2;
    off = (off + 255) & ~size_t(255);
    l.off_d = off;
    off += static_cast<size_t>(R) * l.nblk * kRnsNC * l.kp * 2;
    off = (off + 255) & ~size_t(255);
    l.off_res = off;
    off += static_cast<size_t>(R) * d * n;
    off = (off + 255) & ~size_t(255);
    l.total = off;
    return l;
}

int rns_split(int64_t d, int64_t k, int64_t n, const uint64_t *U, int64_t ldu, const uint64_t *A,
              int64_t lda, uint64_t q, const RnsPrimes &pr, const RnsLayout &lay, uint8_t *ws,
              bool split_u, cudaStream_t st) {
    __half *U16 = reinterpret_cast<__half *>(ws + lay.off_u16);
    __half *D = reinterpret_cast<__half *>(ws + lay.off_d);
    if (split_u) {
        const int64_t total = d * (lay.kp / 8);
        const int blocks = static_cast<int>(std::min<int64_t>((total + 255) / 256, 152 * 16));
        rns_split_u_kernel<<<blocks, 256, 0, st>>>(U, ldu, static_cast<int>(d), static_cast<int>(k),
                                                   static_cast<int>(lay.kp), q, pr, U16);
        if (cudaGetLastError() != cudaSuccess) return -5;
    }
    dim3 grid(static_cast<unsigned>((lay.kp + kRnsT - 1) / kRnsT),
              static_cast<unsigned>((n + 63) / 64));
    rns_split_a_kernel<<<grid, 256, 0, st>>>(A, lda, static_cast<int>(k), static_cast<int>(n),
                                             static_cast<int>(lay.kp), static_cast<int>(lay.nblk),
                                             q, pr, D);
    return cudaGetLastError() == cudaSuccess ? 0 : -5;
}

int rns_gemm(int64_t d, int64_t k, int64_t n, const RnsPrimes &pr, const RnsLayout &lay,
             uint8_t *ws, int *status, uint64_t timeout_ns, int num_sms, const CUtensorMap *tmU,
             const CUtensorMap *tmD, cudaStream_t st) {
    int8_t *res = reinterpret_cast<int8_t *>(ws + lay.off_res);
    for (int ch = 0; ch < pr.chunks; ++ch) {
        const int64_t k0 = ch * pr.chunk_len;
        const int64_t len = std::min(pr.chunk_len, k - k0);
        GemmParams gp{};
        gp.d = static_cast<int>(d);
        gp.n = static_cast<int>(n);
        gp.k = static_cast<int>(len);
        gp.m_blocks = static_cast<int>((d + kBM - 1) / kBM);
        gp.n_blocks = static_cast<int>(lay.nblk);
        gp.planes = pr.R;
        gp.kb_total = static_cast<int>((len + kBK - 1) / kBK);
        const int64_t tiles = static_cast<int64_t>(gp.m_blocks) * gp.n_blocks * pr.R;
        if (tiles >= (int64_t(1) << 31)) return -4;
        gp.num_tiles = static_cast<int>(tiles);
        gp.band_m = band_rows(gp.m_blocks, lay.kp);
        gp.u_per_plane = 1;
        gp.status = status;
        gp.timeout_ns = timeout_ns;
        for (int i = 0; i < pr.R; ++i) {
            PlaneConst &pc = gp.pc[i];
            pc.q = pr.p[i].p;
            const float pinv = 1.0f / static_cast<float>(pr.p[i].p);
            uint32_t bits;
            std::memcpy(&bits, &pinv, sizeof(bits));
            pc.mu = bits;  // mode 1: binary32 bits of 1/p
            // every chunk adds into the same residue plane
            pc.C = reinterpret_cast<uint64_t *>(res + static_cast<int64_t>(i) * d * n);
            pc.ldc = n;
            pc.accumulate = ch > 0 ? 1 : 0;
        }
        if (launch_gemm_kernel<1, 9, kRnsNC, false, 1>(tmU[ch], tmD[ch], gp, num_sms, st) !=
            cudaSuccess)
            return -5;
    }
    return 0;
}

int rns_crt(int64_t d, int64_t n, uint64_t *C, int64_t ldc, uint64_t q, const RnsPrimes &pr,
            const RnsLayout &lay, uint8_t *ws, cudaStream_t st) {
    const int8_t *res = reinterpret_cast<const int8_t *>(ws + lay.off_res);
    const RnsCrt cr = rns_crt_consts(pr, q);
    const int64_t total = d * n;
    const int V = n % 4 == 0 ? 4 : 1;
    const int blocks =
        static_cast<int>(std::min<int64_t>((total / V + 255) / 256, 152 * 8));
    // One 64-bit sum when R (p_max - 1) (q - 1) < 2^64.
    uint32_t pmax = 0;
    for (int i = 0; i < pr.R; ++i) pmax = std::max(pmax, pr.p[i].p);
    const unsigned __int128 bound =
        static_cast<unsigned __int128>(pr.R) * (pmax - 1) * (q - 1);
    const bool one = bound < (static_cast<unsigned __int128>(1) << 64);
    const int di = static_cast<int>(d), ni = static_cast<int>(n);
    if (V == 4 && one)
        rns_crt_kernel<4, true><<<blocks, 256, 0, st>>>(res, di, ni, cr, C, ldc);
    else if (V == 4)
        rns_crt_kernel<4, false><<<blocks, 256, 0, st>>>(res, di, ni, cr, C, ldc);
    else if (one)
        rns_crt_kernel<1, true><<<blocks, 256, 0, st>>>(res, di, ni, cr, C, ldc);
    else
        rns_crt_kernel<1, false><<<blocks, 256, 0, st>>>(res, di, ni, cr, C, ldc);
    return cudaGetLastError() == cudaSuccess ? 0 : -5;
}

}  // namespace modpp
