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
// Balanced residue in [-(p-1)/2, (p-1)/2].
__device__ __forceinline__ int bal_mod(const Limbs &l, const RnsPrime &pp) {
    const uint32_t r = mod_small(l.m2 * pp.t42 + l.m1 * pp.t21 + l.m0, pp.p, pp.mag);
    int v = static_cast<int>(r);
    if (l.neg && v != 0) v = static_cast<int>(pp.p) - v;
    if (2 * v > static_cast<int>(pp.p)) v -= static_cast<int>(pp.p);
    return v;
}

// U (d x k residues mod q, leading dimension ldu) -> R planes of balanced
// residues mod p_i as f16, plane i rows [i d, (i+1) d) of a (R d) x kp matrix
// (zero padded for t >= k).
__global__ void __launch_bounds__(256) rns_split_u_kernel(const uint64_t *__restrict__ U,
                                                          int64_t ldu, int d, int k, int kp,
                                                          uint64_t q, RnsPrimes pr,
                                                          __half *__restrict__ U16) {
    const int64_t total = static_cast<int64_t>(d) * kp;
    const int64_t plane = static_cast<int64_t>(d) * kp;
    const uint64_t half_q = q >> 1;
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = e / kp;
        const int t = static_cast<int>(e - r * kp);
        int64_t x = 0;
        if (t < k) {
            const uint64_t u = U[r * ldu + t];
            x = u > half_q ? static_cast<int64_t>(u) - static_cast<int64_t>(q)
                           : static_cast<int64_t>(u);
        }
        const Limbs l = to_limbs(x);
        for (int i = 0; i < pr.R; ++i) U16[i * plane + e] = __int2half_rn(bal_mod(l, pr.p[i]));
    }
}

// A (k x n residues mod q, leading dimension lda) -> R K-major planes: row
// (i * nblk + c / 256) * 256 + c % 256 holds column c of A's residues mod
// p_i over the inner index (kp halves per row).  One block per 64 x 64 tile.
__global__ void __launch_bounds__(256) rns_split_a_kernel(const uint64_t *__restrict__ A,
                                                          int64_t lda, int k, int n, int kp,
                                                          int nblk, uint64_t q, RnsPrimes pr,
                                                          __half *__restrict__ D) {
    __shared__ __align__(16) __half tile[64 * (kRnsT + 8)];
    const int t0 = blockIdx.x * kRnsT;
    const int c0 = blockIdx.y * 64;
    const uint64_t half_q = q >> 1;
    Limbs x[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        const int e = threadIdx.x + 256 * s;  // 64 x 64 elements, column fastest
        const int tl = e >> 6, cl = e & 63;
        const int t = t0 + tl, c = c0 + cl;
        int64_t v = 0;
        if (t < k && c < n) {
            const uint64_t a = A[static_cast<int64_t>(t) * lda + c];
            v = a > half_q ? static_cast<int64_t>(a) - static_cast<int64_t>(q)
                           : static_cast<int64_t>(a);
        }
        x[s] = to_limbs(v);
    }
    const int sub = threadIdx.x & 7;   // 8 threads per 128-byte row, 8 halves each
    const int t = t0 + 8 * sub;
    for (int i = 0; i < pr.R; ++i) {
#pragma unroll
        for (int s = 0; s < 16; ++s) {
            const int e = threadIdx.x + 256 * s;
            const int tl = e >> 6, cl = e & 63;
            tile[cl * (kRnsT + 8) + tl] = __int2half_rn(bal_mod(x[s], pr.p[i]));
        }
        __syncthreads();
        if (t < kp) {
            for (int row = threadIdx.x >> 3; row < 64; row += 32) {
                const int c = c0 + row;
                const int64_t drow =
                    (static_cast<int64_t>(i) * nblk + c / kRnsNC) * kRnsNC + (c % kRnsNC);
                const uint4 v = *reinterpret_cast<const uint4 *>(&tile[row * (kRnsT + 8) + 8 * sub]);
                *reinterpret_cast<uint4 *>(D + drow * kp + t) = v;
            }
        }
        __syncthreads();
    }
}

// C[r][c] = X mod q from the R balanced residues res[ch][i][r][c] (int8,
// plane stride d * n, row stride n; the chunks' residues of one prime add).
// Per small prime, y = r c_i mod p_i and
// y / p_i come from shared-memory tables indexed by r; the sum
// S = sum_i y_i w_i is kept as two 64-bit halves, S = S_hi 2^32 + S_lo with
// w_i = w_hi 2^32 + w_lo (y_i w_lo < 2^40, y_i w_hi < 2^38: no overflow for
// R <= 32), and reduced modulo q once.  Four consecutive outputs per thread
// (n % 4 == 0) with 32-bit residue loads; one otherwise.
template <int V>
__global__ void __launch_bounds__(256) rns_crt_kernel(const int8_t *__restrict__ res, int d, int n,
                                                      RnsCrt cr, uint64_t *__restrict__ C,
                                                      int64_t ldc) {
    __shared__ uint8_t ytab[kMaxRnsPrimes][256];
    __shared__ float ftab[kMaxRnsPrimes][256];
    for (int e = threadIdx.x; e < cr.R * 256; e += blockDim.x) {
        const int i = e >> 8, r = (e & 255) - 128;  // residue r in [-128, 127]
        const int p = cr.p[i];
        int y = (r * cr.c[i]) % p;
        if (y < 0) y += p;
        ytab[i][e & 255] = static_cast<uint8_t>(y);
        ftab[i][e & 255] = static_cast<float>(y) * cr.pinv[i];
    }
    __syncthreads();
    const uint64_t q = cr.q;
    const int64_t total = static_cast<int64_t>(d) * n;
    const int64_t groups = total / V;
    for (int64_t g = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; g < groups;
         g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t e0 = g * V;
        uint64_t slo[V], shi[V];
        float F[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            slo[v] = 0;
            shi[v] = 0;
            F[v] = 0.f;
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
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int idx = static_cast<int8_t>((words[u] >> (8 * v)) & 0xffu) + 128;
                    const uint32_t y = ytab[i][idx];
                    slo[v] += static_cast<uint64_t>(y) * wl;
                    shi[v] += static_cast<uint64_t>(y) * wh;
                    F[v] += ftab[i][idx];
                }
            }
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            // S mod q = (S_hi mod q) 2^32 + S_lo (mod q)
            uint64_t x = shoup_mulmod(barrett_u64(shi[v], q, cr.mu), cr.t32, cr.t32s, q);
            x = add_mod(x, barrett_u64(slo[v], q, cr.mu), q);
            const uint64_t alpha = static_cast<uint64_t>(__float2int_rn(F[v]));
            x = sub_mod(x, shoup_mulmod(alpha, cr.mq, cr.mqs, q), q);
            const int64_t e = e0 + v;
            const int64_t row = e / n;
            C[row * ldc + (e - row * n)] = x;
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
        c.pinv[i] = 1.0f / static_cast<float>(p);
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
        const int64_t total = d * lay.kp;
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
    if (V == 4)
        rns_crt_kernel<4><<<blocks, 256, 0, st>>>(res, static_cast<int>(d), static_cast<int>(n), cr,
                                                  C, ldc);
    else
        rns_crt_kernel<1><<<blocks, 256, 0, st>>>(res, static_cast<int>(d), static_cast<int>(n), cr,
                                                  C, ldc);
    return cudaGetLastError() == cudaSuccess ? 0 : -5;
}

}  // namespace modpp
