// Internal declarations shared by the library's translation units:
// parameter blocks passed by value to kernels, the per-plane modular
// constants, and the launchers each .cu file provides.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <atomic>
#include <cstddef>
#include <cstdint>

namespace modpp {

constexpr int kMaxPlanes = 32;       // (prime, part) output planes per launch
constexpr int kBM = 128;             // output rows per tile (UMMA M)
// Output columns per tile for L digits: the UMMA N = L * cols is a multiple
// of 16 up to 256 (192..256 for L >= 3), each of the two epilogue column halves
// is a whole number of 4-column TMEM loads, and the epilogue's int64 group
// accumulators (one per 3 digits and column) fit the register budget.
__host__ __device__ constexpr int tile_cols(int L) {
    return L <= 3 ? 64 : (L <= 5 ? 48 : (L == 6 ? 40 : 32));
}
// Tile columns for L digits and n output columns: thin outputs (n <= 64)
// with L = 5 or 6 take 32-column tiles when that pads less than the default
// width (PC-Mv's 32 columns: no padding instead of 8 wasted columns of 40).
__host__ __device__ constexpr int tile_cols_for(int L, long long n) {
    return ((L == 5 || L == 6) && n <= 64 &&
            (n + 31) / 32 * 32 < (n + tile_cols(L) - 1) / tile_cols(L) * tile_cols(L))
               ? 32
               : tile_cols(L);
}
// Grouped launches share one column width for all problems, whose digit
// counts Lp <= L vary: every Lp * cols must be a multiple of 16.
__host__ __device__ constexpr int grouped_tile_cols(int L) {
    return L <= 3 ? 64 : (L <= 5 ? 48 : 32);
}
// Tile columns of the CTA-pair GEMM (gemm_f16_kernel with CTAS = 2): the
// pair's UMMA N = L * cols must be a multiple of 32 (each CTA holds N / 2
// rows of B in whole swizzle atoms) and at most 256.
__host__ __device__ constexpr int pair_tile_cols(int L) {
    return L <= 3 ? 64 : (L == 4 ? 48 : 32);
}
constexpr int kMaxTileCols = 64;
constexpr int kBK = 64;              // f16 elements per K block: one 128-byte row
constexpr int kRowBytes = kBK * 2;   // swizzle span of the operand tiles (64 or 128)
static_assert(kRowBytes == 64 || kRowBytes == 128, "K block must be a 64- or 128-byte row");
constexpr int kMinDigitBits = 8;     // balanced b-bit digits in [-2^(b-1), 2^(b-1) - 1]
constexpr int kMaxDigitBits = 10;
constexpr int kMaxDigits = 8;        // q < 2^62 needs at most 8 eight-bit digits

// Inner-dimension chunk whose FP32 partial sums stay exact for b-bit digits:
// chunk * 128 * 2^(b-1) = 2^24 (|U| <= 128), i.e. chunk = 2^(18 - b).
__host__ __device__ constexpr int chunk_k(int digit_bits) { return 1 << (18 - digit_bits); }

// Constants of one output plane (one prime, one part).
struct PlaneConst {
    uint64_t q;
    uint64_t mu;    // floor(2^64 / q), Barrett
    uint64_t wg1;   // 2^(3b) mod q: weight of digit group 1 (digits 3..5)
    uint64_t wg1s;  // floor(wg1 * 2^64 / q), Shoup
    uint64_t wg2;   // 2^(6b) mod q: weight of digit group 2 (digits 6..8)
    uint64_t wg2s;
    uint64_t *C;    // output plane, d x n, leading dimension ldc
    int64_t ldc;
    uint64_t qoff;  // a multiple of q >= 2^57: g + qoff lies in [0, 2^64) for |g| < 2^57
    uint64_t wout;  // accumulate mode: C <- C + wout * (U*A) mod q
    uint64_t wouts; // Shoup quotient of wout
    int accumulate; // 0: C <- U*A mod q;  1: C <- C + wout * (U*A);  2: C <- wout * (U*A)
};

// One (problem, prime) plane of a grouped launch.  Planes are stored in tile
// order: plane i owns tiles [tile_begin, tile_begin + m_blocks * n_blocks).
struct GroupPlane {
    PlaneConst pc;
    const CUtensorMap *tmU;  // the problem's U16 map (global memory)
    const CUtensorMap *tmD;  // the problem's digit-matrix map (global memory)
    int d, n, kb_total;
    int m_blocks, n_blocks;
    int Lp;                  // digits of this problem
    int dplane;              // index of this plane within the problem's digit matrix
    int tile_begin;
    int band_m;              // row blocks per band of the tile order (see band_rows)
};

struct GemmParams {
    int d, n, k;      // output rows, output columns, inner dimension
    int m_blocks;     // ceil(d / kBM)
    int n_blocks;     // ceil(n / tile_cols(L))
    int planes;
    int kb_total;     // ceil(k / kBK)
    int num_tiles;    // planes * n_blocks * m_blocks
    int plane_fastest;  // tile order: 0 = row block fastest (in bands), 1 = plane fastest
    int band_m;         // row blocks per band of the row-fastest order (see band_rows)
    int *status;      // device status word (workspace)
    uint64_t timeout_ns;
    const GroupPlane *gplanes;  // grouped launches only
    int num_gplanes;
    const int *tile_plane;      // grouped: plane of every tile (index into gplanes)
    int u_per_plane;            // 1: plane i reads U rows [i*d, (i+1)*d) of the U map
    PlaneConst pc[kMaxPlanes];
};

// Source of one plane for the digit split.
struct SplitPlane {
    const uint64_t *A;  // k x n residues, leading dimension lda
    int64_t lda;
    uint64_t q;
    uint64_t thresh;    // residues above thresh are lifted to a - q (balanced window)
    int shift = 0;      // > 0: lifted value rounded to floor((x + 2^(s-1)) / 2^s) first
};

struct SplitParams {
    int k, n, kp, n_blocks, planes, digits, digit_bits;
    int nc;             // tile columns (tile_cols_for(digits, n))
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
// Number of balanced b-bit digits covering residues mod q: the window of L
// such digits holds 2^(bL) consecutive integers, so q <= 2^(bL).
inline int f16_digit_count(uint64_t q, int b) { return (bit_length(q - 1) + b - 1) / b; }

// Largest value kept positive when lifting a residue into the balanced
// window [-2^(b-1) S, (2^(b-1) - 1) S], S = sum_{i<L} 2^(b i); saturated to
// 2^63 - 1 (then no residue needs lifting).
inline uint64_t f16_lift_threshold(int L, int b) {
    unsigned __int128 S = 0;
    for (int i = 0; i < L; ++i) S += static_cast<unsigned __int128>(1) << (b * i);
    unsigned __int128 T = S * ((1u << (b - 1)) - 1u);
    const unsigned __int128 cap = (static_cast<unsigned __int128>(1) << 63) - 1;
    return static_cast<uint64_t>(T > cap ? cap : T);
}

inline PlaneConst make_plane_const(uint64_t q, int b, uint64_t *C, int64_t ldc) {
    PlaneConst p{};
    p.q = q;
    p.mu = host_barrett_mu(q);
    p.wg1 = host_pow2_mod(3 * b, q);
    p.wg1s = host_shoup(p.wg1, q);
    p.wg2 = host_pow2_mod(6 * b, q);
    p.wg2s = host_shoup(p.wg2, q);
    p.qoff = static_cast<uint64_t>(((static_cast<unsigned __int128>(1) << 57) + q - 1) / q * q);
    p.C = C;
    p.ldc = ldc;
    p.wout = 1 % q;
    p.wouts = host_shoup(p.wout, q);
    p.accumulate = 0;
    return p;
}

// True while modpp_profile_enable(1) is in effect.
bool profile_active();
// Kernel timing hooks for other translation units (no-ops when profiling is
// off or the stream is being captured): prof_begin returns a handle for
// prof_end, or null.
void *prof_begin(int kernel, cudaStream_t st);
void prof_end(void *handle, cudaStream_t st);

// Row blocks per band of the tile order.  Tiles run band by band: inside a
// band the row block varies fastest, then the column block.  The concurrently
// running tiles then share the band's rows of U and a few column blocks of
// digits; the band's U rows (kBM * kp f16 each block) stay in L2 while all
// column blocks pass, so U is read from HBM about once and the digit matrix
// once per band.  U that fits the budget whole forms a single band.
constexpr int64_t kBandBytes = int64_t(32) << 20;
inline int band_rows(int m_blocks, int64_t kp) {
    const int64_t per_block = static_cast<int64_t>(kBM) * kp * 2;
    int64_t b = kBandBytes / (per_block > 0 ? per_block : 1);
    if (b < 1) b = 1;
    return b >= m_blocks ? m_blocks : static_cast<int>(b);
}

// Raises a kernel's dynamic shared-memory limit to `bytes` once per device
// (the setting stays with the kernel on that device), so repeated launches
// skip the driver call.  `done` holds one bit per device (devices >= 64 set
// it every time).
inline cudaError_t set_smem_limit_once(const void *kernel, int bytes,
                                       std::atomic<unsigned long long> &done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev >= 0 && dev < 64 ? (1ull << dev) : 0ull;
    if (bit != 0 && (done.load(std::memory_order_acquire) & bit) != 0) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit != 0) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

// ------------------------------------------------------------ launchers
// Each returns a cudaError_t from the launch (cudaSuccess when enqueued).
cudaError_t launch_u_to_f16(const void *U, int ukind, int64_t ldu, int d, int k, int kp,
                            __half *U16, cudaStream_t s);
// Residues U (d x k, leading dimension ldu, mod q) -> `digits` balanced 8-bit
// digit planes, int8, plane i at out + i * d * k (leading dimension k).
cudaError_t launch_u64_to_i8_digits(const uint64_t *U, int64_t ldu, int d, int k, uint64_t q,
                                    uint64_t thresh, int digits, int8_t *out, cudaStream_t s);
cudaError_t launch_split_digits(const SplitParams &p, cudaStream_t s);
cudaError_t launch_gemm_f16(const CUtensorMap &tmU, const CUtensorMap &tmD, const GemmParams &p,
                            int digits, int digit_bits, int num_sms, cudaStream_t s,
                            int nc = 0);  // 0: tile_cols(digits)
// The CTA-pair GEMM (tiles of 256 rows x pair_tile_cols(digits) columns;
// p.m_blocks counts 256-row blocks), launched as clusters of two CTAs, as
// many clusters as can be resident at once.
cudaError_t launch_gemm_f16_pair(const CUtensorMap &tmU, const CUtensorMap &tmD,
                                 const GemmParams &p, int digits, int digit_bits, cudaStream_t s);


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
// Exact residues of integer-valued double products (Strategy 2).
constexpr int kMaxPow2Shift = 72;
struct Fp64ResidueParams {
    const double *P;  // d x n, leading dimension n
    int d, n;
    uint64_t q, mu;
    uint64_t pow2[kMaxPow2Shift];   // 2^e mod q
    uint64_t pow2s[kMaxPow2Shift];  // Shoup quotients
    uint64_t *C;
    int64_t ldc;
};
cudaError_t launch_fp64_residue(const Fp64ResidueParams &p, cudaStream_t s);

// Value-range checks of the inputs (debug mode, range_checks.cu).
constexpr int kMaxRangeQ = 40;
struct RangeCheckU64 {
    const uint64_t *base;
    int64_t planes, rows, cols, ld, plane_stride;
    int nq;                // plane p is bounded by q[p % nq]
    uint64_t q[kMaxRangeQ];
    int *status;           // MODPP_ERR_RANGE is written here on a violation
};
bool debug_checks_on();
cudaError_t launch_range_u64(const RangeCheckU64 &a, cudaStream_t s);
cudaError_t launch_range_i32(const int32_t *U, int64_t rows, int64_t cols, int64_t ld, int *status,
                             cudaStream_t s);
// Planes p < planes of rows x cols (leading dimension ld, plane stride
// plane_stride) bounded by q[p % nq].
cudaError_t range_planes(const uint64_t *base, int64_t planes, int64_t rows, int64_t cols,
                         int64_t ld, int64_t plane_stride, const uint64_t *q, int nq, int *status,
                         cudaStream_t s);

// Host-side argument checks of modpp_mm other than the path and the
// workspace: sizes, primes, U kind, null pointers, leading dimensions and
// plane strides.  Returns MODPP_OK or the negative status modpp_mm returns.
int mm_check_args(int64_t d, int64_t k, int64_t n, const void *U, int ukind, int64_t ldu,
                  const uint64_t *A, int64_t lda, int64_t strideA, const uint64_t *C, int64_t ldc,
                  int64_t strideC, const uint64_t *primes_host, int P);

}  // namespace modpp
