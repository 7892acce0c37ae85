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

// Lifts residue a (in [0, q)) into the balanced window of Lp digits (values
// above `thresh` become a - q), then peels digits from the bottom:
// d = ((x + 2^(b-1)) mod 2^b) - 2^(b-1), x <- (x - d) / 2^b (exact).
template <int LMAX, int DB, int NC>
__device__ __forceinline__ void split_digit_tile(__half *tile, const uint64_t *A, int64_t lda,
                                                 uint64_t q, uint64_t thresh, int k, int n, int kp,
                                                 int Lp, int t0, int c0, __half *Dblock) {
    constexpr int64_t kHalf = int64_t(1) << (DB - 1);
    constexpr int64_t kMask = (int64_t(1) << DB) - 1;
#pragma unroll 4
    for (int e = threadIdx.x; e < kSplitT * NC; e += 256) {
        const int tl = e / NC, cl = e - (e / NC) * NC;
        const int t = t0 + tl, c = c0 + cl;
        uint64_t a = 0;
        if (t < k && c < n) a = A[static_cast<int64_t>(t) * lda + c];
        int64_t x = a > thresh ? static_cast<int64_t>(a - q) : static_cast<int64_t>(a);
#pragma unroll
        for (int l = 0; l < LMAX; ++l) {
            if (l >= Lp) break;
            const int dgt = static_cast<int>(((x + kHalf) & kMask) - kHalf);
            x = (x - dgt) >> DB;
            tile[(l * NC + cl) * kSplitRow + tl] = __int2half_rn(dgt);
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
