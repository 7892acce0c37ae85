// One 64 x NC tile of the residue -> balanced-digit split, shared by the
// single-problem and the grouped split kernels (split_kernels.cu, grouped.cu).
//
// Phase 1 reads A coalesced along the columns, computes the Lp <= LMAX
// digits of each residue and stores them in shared memory as [l][c][t].
// Phase 2 writes each (l, c) row of 64 digits (128 bytes) contiguously along
// the inner index t, so the digit matrix is K-major for the tensor cores.
// The digit identity is Eq. decomp of Sec. 6.1 with base 2^b:
//   a = sum_l 2^(b l) D_l,  D_l in [-2^(b-1), 2^(b-1) - 1].
#pragma once
#include <cuda_fp16.h>

#include <cstdint>

namespace modpp {

constexpr int kSplitT = 64;
constexpr int kSplitRow = kSplitT + 4;  // padded row (halves): 136-byte rows

// f16 bits of two integers |v| < 512 as a half2 word: 1536 + v lies in
// [1024, 2048), where the f16 values are the integers, so its bit pattern is
// 0x6600 + v, and one half2 subtraction of 1536 is exact.
__device__ __forceinline__ uint32_t digit_half2(int v0, int v1) {
    const uint32_t biased = static_cast<uint32_t>(0x6600 + v0) |
                            (static_cast<uint32_t>(0x6600 + v1) << 16);
    __half2 h = *reinterpret_cast<const __half2 *>(&biased);
    h = __hsub2(h, __float2half2_rn(1536.0f));
    return *reinterpret_cast<const uint32_t *>(&h);
}

// Lifts residue a (in [0, q)) into the balanced window of Lp digits (values
// above `thresh` become a - q), then peels digits from the bottom:
// d = ((x + 2^(b-1)) mod 2^b) - 2^(b-1), x <- (x - d) / 2^b (exact).
// With shift s > 0 the lifted value is first rounded to its high-order
// bits, x <- floor((x + 2^(s-1)) / 2^s) (the truncation of Strategy 2,
// Sec. 6.1; the caller multiplies the product by 2^s).
// Phase 1: a thread takes four consecutive inner indices of one column
// (loads coalesced along the columns) and writes each digit's four values as
// one 8-byte word of the tile's row (row stride 136 bytes: a half-warp's
// 8-byte stores fall in distinct banks).
template <int LMAX, int DB, int NC>
__device__ __forceinline__ void split_digit_tile(__half *tile, const uint64_t *A, int64_t lda,
                                                 uint64_t q, uint64_t thresh, int k, int n, int kp,
                                                 int Lp, int t0, int c0, __half *Dblock,
                                                 int shift = 0) {
    static_assert(DB <= 10, "digits must satisfy |d| < 512 for the f16 packing");
    constexpr int64_t kHalf = int64_t(1) << (DB - 1);
    constexpr int64_t kMask = (int64_t(1) << DB) - 1;
#pragma unroll 2
    for (int e = threadIdx.x; e < (kSplitT / 4) * NC; e += 256) {
        const int tq = e / NC, cl = e - (e / NC) * NC;
        const int c = c0 + cl;
        int64_t x[4];
#pragma unroll
        for (int s4 = 0; s4 < 4; ++s4) {
            const int t = t0 + 4 * tq + s4;
            uint64_t a = 0;
            if (t < k && c < n) a = A[static_cast<int64_t>(t) * lda + c];
            x[s4] = a > thresh ? static_cast<int64_t>(a - q) : static_cast<int64_t>(a);
            if (shift > 0) x[s4] = (x[s4] + (int64_t(1) << (shift - 1))) >> shift;
        }
#pragma unroll
        for (int l = 0; l < LMAX; ++l) {
            if (l >= Lp) break;
            int dg[4];
#pragma unroll
            for (int s4 = 0; s4 < 4; ++s4) {
                dg[s4] = static_cast<int>(((x[s4] + kHalf) & kMask) - kHalf);
                x[s4] = (x[s4] - dg[s4]) >> DB;
            }
            *reinterpret_cast<uint2 *>(&tile[(l * NC + cl) * kSplitRow + 4 * tq]) =
                make_uint2(digit_half2(dg[0], dg[1]), digit_half2(dg[2], dg[3]));
        }
    }
    __syncthreads();
    // 16 threads per 128-byte row, 4 halves (8 bytes) each.
    const int sub = threadIdx.x & 15;
    const int t = t0 + 4 * sub;
    if (t < kp) {
        for (int row = threadIdx.x >> 4; row < Lp * NC; row += 16) {
            const uint2 v = *reinterpret_cast<const uint2 *>(&tile[row * kSplitRow + 4 * sub]);
            *reinterpret_cast<uint2 *>(Dblock + static_cast<int64_t>(row) * kp + t) = v;
        }
    }
}

}  // namespace modpp
