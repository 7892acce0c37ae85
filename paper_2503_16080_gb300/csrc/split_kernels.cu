// Operand preparation kernels (memory-bound passes around the GEMMs).
//
// f16 path (default):
//   u_to_f16        U (int8/int32, d x k) -> U16 (f16, d x kp, zero padded), K-major.
//   split_digits    A_j (u64 residues, k x n) -> balanced b-bit digits (b = 8..10):
//                   a = sum_l 2^(b l) * D_l with D_l in [-2^(b-1), 2^(b-1) - 1], written
//                   as f16 (exact) and transposed to K-major rows (plane, n_block, l, col).
//                   This is the limb split of the residue operand; the digit
//                   identity is Eq. decomp of Sec. 6.1 with base 2^b.
// FP64 path (Strategy 1, Lemma le:strategy1):
//   u_to_f64, fp64_split (signed base-K digits of the centred residue),
//   fp64_recombine (sum_i K^i * P_i mod q from the exact binary64 products).
#include <cuda_fp16.h>

#include "modarith.cuh"
#include "modpp_internal.h"
#include "split_tile.cuh"

namespace modpp {

// ---------------------------------------------------------------- U -> f16
// One thread converts 8 consecutive entries of a row (one 16-byte store).
// Rows are processed by blocks of threads along kp; entries at t >= k are 0.
__global__ void __launch_bounds__(256) u_to_f16_kernel(const void *__restrict__ U, int ukind,
                                                        int64_t ldu, int d, int k, int kp,
                                                        __half *__restrict__ U16) {
    const int groups = kp / 8;  // kp is a multiple of 8
    const int64_t total = static_cast<int64_t>(d) * groups;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = i / groups;
        const int t0 = static_cast<int>(i - r * groups) * 8;
        __align__(16) __half h[8];
        if (ukind == 0) {
            const int8_t *src = static_cast<const int8_t *>(U) + r * ldu + t0;
            const bool vec = t0 + 8 <= k && (reinterpret_cast<uintptr_t>(src) & 7u) == 0;
            if (vec) {
                const int2 w = *reinterpret_cast<const int2 *>(src);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int word = j < 4 ? w.x : w.y;
                    h[j] = __int2half_rn(static_cast<int8_t>((word >> (8 * (j & 3))) & 0xff));
                }
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    h[j] = __int2half_rn(t0 + j < k ? static_cast<int>(src[j]) : 0);
            }
        } else {
            const int32_t *src = static_cast<const int32_t *>(U) + r * ldu + t0;
#pragma unroll
            for (int j = 0; j < 8; ++j) h[j] = __int2half_rn(t0 + j < k ? src[j] : 0);
        }
        *reinterpret_cast<uint4 *>(U16 + r * kp + t0) = *reinterpret_cast<const uint4 *>(h);
    }
}

cudaError_t launch_u_to_f16(const void *U, int ukind, int64_t ldu, int d, int k, int kp,
                            __half *U16, cudaStream_t s) {
    const int64_t total = static_cast<int64_t>(d) * (kp / 8);
    if (total == 0) return cudaSuccess;
    int blocks = static_cast<int>((total + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    u_to_f16_kernel<<<blocks, 256, 0, s>>>(U, ukind, ldu, d, k, kp, U16);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- U residues -> int8 digits
// Balanced 8-bit digits of residues mod q for the left operand of a product
// of two residue matrices: u = sum_i 2^(8 i) U_i, U_i in [-128, 127].
__global__ void u64_to_i8_digits_kernel(const uint64_t *__restrict__ U, int64_t ldu, int d, int k,
                                        uint64_t q, uint64_t thresh, int digits,
                                        int8_t *__restrict__ out) {
    const int64_t total = static_cast<int64_t>(d) * k;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = i / k;
        const int64_t t = i - r * k;
        const uint64_t a = U[r * ldu + t];
        int64_t x = a > thresh ? static_cast<int64_t>(a - q) : static_cast<int64_t>(a);
        for (int l = 0; l < digits; ++l) {
            const int dgt = static_cast<int>(((x + 128) & 255) - 128);
            x = (x - dgt) >> 8;
            out[static_cast<int64_t>(l) * total + i] = static_cast<int8_t>(dgt);
        }
    }
}

cudaError_t launch_u64_to_i8_digits(const uint64_t *U, int64_t ldu, int d, int k, uint64_t q,
                                    uint64_t thresh, int digits, int8_t *out, cudaStream_t s) {
    const int64_t total = static_cast<int64_t>(d) * k;
    if (total == 0) return cudaSuccess;
    int blocks = static_cast<int>((total + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    u64_to_i8_digits_kernel<<<blocks, 256, 0, s>>>(U, ldu, d, k, q, thresh, digits, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- digits
// One block per (64 inner indices, one column block, one plane).
template <int L, int DB, int NC = tile_cols(L)>
__global__ void __launch_bounds__(256) split_digits_kernel(const __grid_constant__ SplitParams p) {
    __shared__ __align__(16) __half tile[L * NC * kSplitRow];
    const int plane = blockIdx.z;
    const int nb = blockIdx.y;
    const SplitPlane sp = p.sp[plane];
    __half *Dblock =
        p.D + (static_cast<int64_t>(plane) * p.n_blocks + nb) * L * NC * static_cast<int64_t>(p.kp);
    split_digit_tile<L, DB, NC>(tile, sp.A, sp.lda, sp.q, sp.thresh, p.k, p.n, p.kp, L,
                                blockIdx.x * kSplitT, nb * NC, Dblock, sp.shift);
}

template <int DB>
static bool launch_split_db(const SplitParams &p, dim3 grid, cudaStream_t s) {
    if (p.nc == 32 && p.digits == 5) {
        split_digits_kernel<5, DB, 32><<<grid, 256, 0, s>>>(p);
        return true;
    }
    if (p.nc == 32 && p.digits == 6) {
        split_digits_kernel<6, DB, 32><<<grid, 256, 0, s>>>(p);
        return true;
    }
    if (p.nc != 0 && p.nc != tile_cols(p.digits)) return false;
    switch (p.digits) {
        case 1: split_digits_kernel<1, DB><<<grid, 256, 0, s>>>(p); return true;
        case 2: split_digits_kernel<2, DB><<<grid, 256, 0, s>>>(p); return true;
        case 3: split_digits_kernel<3, DB><<<grid, 256, 0, s>>>(p); return true;
        case 4: split_digits_kernel<4, DB><<<grid, 256, 0, s>>>(p); return true;
        case 5: split_digits_kernel<5, DB><<<grid, 256, 0, s>>>(p); return true;
        case 6: split_digits_kernel<6, DB><<<grid, 256, 0, s>>>(p); return true;
        case 7: split_digits_kernel<7, DB><<<grid, 256, 0, s>>>(p); return true;
        case 8: split_digits_kernel<8, DB><<<grid, 256, 0, s>>>(p); return true;
        default: return false;
    }
}

cudaError_t launch_split_digits(const SplitParams &p, cudaStream_t s) {
    if (p.kp == 0 || p.n_blocks == 0 || p.planes == 0) return cudaSuccess;
    dim3 grid((p.kp + kSplitT - 1) / kSplitT, p.n_blocks, p.planes);
    bool ok = false;
    switch (p.digit_bits) {
        case 8: ok = launch_split_db<8>(p, grid, s); break;
        case 9: ok = launch_split_db<9>(p, grid, s); break;
        case 10: ok = launch_split_db<10>(p, grid, s); break;
        default: break;
    }
    if (!ok) return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// ---------------------------------------------------------------- FP64 path
__global__ void u_to_f64_kernel(const void *__restrict__ U, int ukind, int64_t ldu, int d, int k,
                                double *__restrict__ Ud) {
    const int64_t total = static_cast<int64_t>(d) * k;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = i / k;
        const int64_t t = i - r * k;
        const int v = ukind == 0 ? static_cast<int>(static_cast<const int8_t *>(U)[r * ldu + t])
                                 : static_cast<const int32_t *>(U)[r * ldu + t];
        Ud[i] = static_cast<double>(v);
    }
}

cudaError_t launch_u_to_f64(const void *U, int ukind, int64_t ldu, int d, int k, double *Ud,
                            cudaStream_t s) {
    const int64_t total = static_cast<int64_t>(d) * k;
    if (total == 0) return cudaSuccess;
    int blocks = static_cast<int>((total + 255) / 256);
    if (blocks > 152 * 32) blocks = 152 * 32;
    u_to_f64_kernel<<<blocks, 256, 0, s>>>(U, ukind, ldu, d, k, Ud);
    return cudaGetLastError();
}

// Signed base-K digits (Eq. decomp): the centred residue r = sum_i r_i K^i
// with every r_i of the sign of r and |r_i| < K.
__global__ void fp64_split_kernel(const Fp64SplitParams p) {
    const int64_t total = static_cast<int64_t>(p.k) * p.n;
    const int64_t ldo = static_cast<int64_t>(p.digits) * p.n;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t t = i / p.n;
        const int64_t c = i - t * p.n;
        const uint64_t a = p.A[t * p.lda + c];
        const bool neg = a > p.q / 2;  // centred representative in (-q/2, q/2]
        uint64_t mag = neg ? p.q - a : a;
        double *o = p.out + t * ldo + c;
        for (int dgt = 0; dgt < p.digits; ++dgt) {
            const uint64_t qd = mag / p.base;
            const uint64_t r = mag - qd * p.base;
            mag = qd;
            o[static_cast<int64_t>(dgt) * p.n] = neg ? -static_cast<double>(r) : static_cast<double>(r);
        }
    }
}

cudaError_t launch_fp64_split(const Fp64SplitParams &p, cudaStream_t s) {
    const int64_t total = static_cast<int64_t>(p.k) * p.n;
    if (total == 0) return cudaSuccess;
    int blocks = static_cast<int>((total + 255) / 256);
    if (blocks > 152 * 32) blocks = 152 * 32;
    fp64_split_kernel<<<blocks, 256, 0, s>>>(p);
    return cudaGetLastError();
}

// C = sum_i K^i * P_i mod q.  Each P_i entry is an exact integer below 2^53
// in magnitude, so the conversion to int64 is exact.
__global__ void fp64_recombine_kernel(const __grid_constant__ Fp64RecombineParams p) {
    const int64_t total = static_cast<int64_t>(p.d) * p.n;
    const int64_t ldp = static_cast<int64_t>(p.digits) * p.n;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = i / p.n;
        const int64_t c = i - r * p.n;
        const double *row = p.P + r * ldp + c;
        uint64_t acc = 0;
        for (int dgt = 0; dgt < p.digits; ++dgt) {
            const int64_t v = __double2ll_rn(row[static_cast<int64_t>(dgt) * p.n]);
            const uint64_t red = smod_i64(v, p.q, p.mu);
            acc = add_mod(acc, shoup_mulmod(red, p.powK[dgt], p.powKs[dgt], p.q), p.q);
        }
        p.C[r * p.ldc + c] = acc;
    }
}

// Exact residue modulo q of integer-valued binary64 products (Strategy 2 of
// Sec. 6.1): v = m * 2^e with an integer mantissa |m| < 2^53; for e > 0 the
// residue is (m mod q) * (2^e mod q).
__global__ void fp64_residue_kernel(const __grid_constant__ Fp64ResidueParams p) {
    const int64_t total = static_cast<int64_t>(p.d) * p.n;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = i / p.n;
        const int64_t c = i - r * p.n;
        const double v = p.P[r * p.n + c];
        int e = 0;
        const double f = frexp(v, &e);  // v = f * 2^e, 0.5 <= |f| < 1
        uint64_t res;
        if (e <= 53) {
            res = smod_i64(__double2ll_rn(v), p.q, p.mu);  // |v| < 2^53: exact
        } else {
            const int64_t m = __double2ll_rn(ldexp(f, 53));  // exact integer mantissa
            const int sh = e - 53;
            res = shoup_mulmod(smod_i64(m, p.q, p.mu), p.pow2[sh], p.pow2s[sh], p.q);
        }
        p.C[r * p.ldc + c] = res;
    }
}

cudaError_t launch_fp64_residue(const Fp64ResidueParams &p, cudaStream_t s) {
    const int64_t total = static_cast<int64_t>(p.d) * p.n;
    if (total == 0) return cudaSuccess;
    int blocks = static_cast<int>((total + 255) / 256);
    if (blocks > 152 * 32) blocks = 152 * 32;
    fp64_residue_kernel<<<blocks, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_fp64_recombine(const Fp64RecombineParams &p, cudaStream_t s) {
    const int64_t total = static_cast<int64_t>(p.d) * p.n;
    if (total == 0) return cudaSuccess;
    int blocks = static_cast<int>((total + 255) / 256);
    if (blocks > 152 * 32) blocks = 152 * 32;
    fp64_recombine_kernel<<<blocks, 256, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace modpp
