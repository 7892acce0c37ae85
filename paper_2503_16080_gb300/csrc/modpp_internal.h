// Internal declarations shared by the library's translation units:
// parameter blocks passed by value to kernels, the per-plane modular
// constants, and the launchers each .cu file provides.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cstddef>
#include <cstdint>

namespace modpp {

constexpr int kMaxPlanes = 32;       // (prime, part) output planes per launch
constexpr int kBM = 128;             // output rows per tile (UMMA M)
constexpr int kNC = 32;              // output columns per tile
constexpr int kBK = 64;              // f16 elements per K block (one 128-byte row)
constexpr int kDigitBits = 10;       // balanced digits in [-512, 511]
constexpr int kChunkK = 256;         // FP32-exact inner chunk: 256 * 128 * 512 = 2^24
constexpr int kChunkKB = kChunkK / kBK;
constexpr int kMaxDigits = 7;        // q < 2^62 needs at most 7 ten-bit digits

// Constants of one output plane (one prime, one part).
struct PlaneConst {
    uint64_t q;
    uint64_t mu;    // floor(2^64 / q), Barrett
    uint64_t w30;   // 2^30 mod q
    uint64_t w30s;  // floor(w30 * 2^64 / q), Shoup
    uint64_t w60;   // 2^60 mod q
    uint64_t w60s;
    uint64_t *C;    // output plane, d x n, leading dimension ldc
    int64_t ldc;
};

struct GemmParams {
    int d, n, k;      // output rows, output columns, inner dimension
    int m_blocks;     // ceil(d / kBM)
    int n_blocks;     // ceil(n / kNC)
    int planes;
    int kb_total;     // ceil(k / kBK)
    int num_tiles;    // planes * n_blocks * m_blocks
    int *status;      // device status word (workspace)
    uint64_t timeout_ns;
    PlaneConst pc[kMaxPlanes];
};

// Source of one plane for the digit split.
struct SplitPlane {
    const uint64_t *A;  // k x n residues, leading dimension lda
    int64_t lda;
    uint64_t q;
    uint64_t thresh;    // residues above thresh are lifted to a - q (balanced window)
};

struct SplitParams {
    int k, n, kp, n_blocks, planes, digits;
    __half *D;          // digit matrix: rows (plane, n_block, digit, col), kp columns
    SplitPlane sp[kMaxPlanes];
};

// ------------------------------------------------------------ host helpers
inline uint64_t host_mulmod(uint64_t a, uint64_t b, uint64_t q) {
    return static_cast<uint64_t>((static_cast<unsigned __int128>(a) * b) % q);
}
inline uint64_t host_pow2_mod(int e, uint64_t q) {
    uint64_t r = 1 % q, b = 2 % q;
    while (e) {
        if (e & 1) r = host_mulmod(r, b, q);
        b = host_mulmod(b, b, q);
        e >>= 1;
    }
    return r;
}
inline uint64_t host_shoup(uint64_t w, uint64_t q) {
    return static_cast<uint64_t>((static_cast<unsigned __int128>(w) << 64) / q);
}
inline uint64_t host_barrett_mu(uint64_t q) {
    return static_cast<uint64_t>((static_cast<unsigned __int128>(1) << 64) / q);
}
inline int bit_length(uint64_t q) {
    int b = 0;
    while (q) {
        ++b;
        q >>= 1;
    }
    return b;
}
// Number of balanced 10-bit digits covering residues mod q: the window of L
// such digits holds 2^(10L) consecutive integers, so q <= 2^(10L).
inline int f16_digit_count(uint64_t q) { return (bit_length(q - 1) + kDigitBits - 1) / kDigitBits; }

// Largest value kept positive when lifting a residue into the balanced
// window [-512*S, 511*S], S = sum_{i<L} 2^(10 i); saturated to 2^63 - 1.
inline uint64_t f16_lift_threshold(int L) {
    unsigned __int128 S = 0;
    for (int i = 0; i < L; ++i) S += static_cast<unsigned __int128>(1) << (kDigitBits * i);
    unsigned __int128 T = S * 511u;
    const unsigned __int128 cap = (static_cast<unsigned __int128>(1) << 63) - 1;
    return static_cast<uint64_t>(T > cap ? cap : T);
}

inline PlaneConst make_plane_const(uint64_t q, uint64_t *C, int64_t ldc) {
    PlaneConst p{};
    p.q = q;
    p.mu = host_barrett_mu(q);
    p.w30 = host_pow2_mod(30, q);
    p.w30s = host_shoup(p.w30, q);
    p.w60 = host_pow2_mod(60, q);
    p.w60s = host_shoup(p.w60, q);
    p.C = C;
    p.ldc = ldc;
    return p;
}

// ------------------------------------------------------------ launchers
// Each returns a cudaError_t from the launch (cudaSuccess when enqueued).
cudaError_t launch_u_to_f16(const void *U, int ukind, int64_t ldu, int d, int k, int kp,
                            __half *U16, cudaStream_t s);
cudaError_t launch_split_digits(const SplitParams &p, cudaStream_t s);
cudaError_t launch_gemm_f16(const CUtensorMap &tmU, const CUtensorMap &tmD, const GemmParams &p,
                            int digits, int num_sms, cudaStream_t s);

// FP64-limb (Strategy 1) helpers.
struct Fp64SplitParams {
    const uint64_t *A;
    int64_t lda;
    int k, n, digits;
    uint64_t q, base;
    double *out;  // k x (digits * n): digit i of column c at column i*n + c
};
cudaError_t launch_u_to_f64(const void *U, int ukind, int64_t ldu, int d, int k, double *Ud,
                            cudaStream_t s);
cudaError_t launch_fp64_split(const Fp64SplitParams &p, cudaStream_t s);
struct Fp64RecombineParams {
    const double *P;  // d x (digits * n) products
    int d, n, digits;
    uint64_t q, mu;
    uint64_t powK[8];   // K^i mod q
    uint64_t powKs[8];  // Shoup quotients
    uint64_t *C;
    int64_t ldc;
};
cudaError_t launch_fp64_recombine(const Fp64RecombineParams &p, cudaStream_t s);

}  // namespace modpp
