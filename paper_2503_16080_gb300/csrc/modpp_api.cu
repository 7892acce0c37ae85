// Host side of the C ABI declared in include/modpp.h: argument checks,
// workspace layout, TMA descriptors, and the kernel / cuBLAS sequence of each
// path.  Nothing here allocates device memory except the cuBLAS handle that
// the FP64 path creates once per device on first use.
#include <cublas_v2.h>
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "modpp.h"
#include "modpp_internal.h"
#include "ptx_sm103.cuh"
#include "rns_wide.h"

using namespace modpp;

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kHeaderBytes = 256;        // status word + reserve
constexpr size_t kCublasWsBytes = 32u << 20;  // cuBLAS scratch inside the workspace
constexpr int64_t kMaxK = int64_t(1) << 20;
constexpr int kMaxDevices = 64;
// Internal U kind: U is a prepared f16 plaintext (modpp_u_to_f16).
constexpr int kUPrepared = 16;

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

bool prime_ok(uint64_t q) { return q >= 3 && (q & 1u) && q < (uint64_t(1) << 62); }

int check_primes(const uint64_t *primes, int P, int max_planes) {
    if (P < 1 || P > max_planes || primes == nullptr) return MODPP_ERR_ARG;
    for (int j = 0; j < P; ++j)
        if (!prime_ok(primes[j])) return MODPP_ERR_PRIME;
    return MODPP_OK;
}

int check_sizes(int64_t d, int64_t k, int64_t n) {
    if (d < 0 || k < 0 || n < 0) return MODPP_ERR_ARG;
    if (d >= (int64_t(1) << 31) || n >= (int64_t(1) << 31) || k > kMaxK) return MODPP_ERR_ARG;
    return MODPP_OK;
}

// Digit width of the f16 path: 0 selects the default.  Narrower digits allow
// deeper exact FP32 chunks (fewer TMEM drains) at the cost of more digits.
constexpr int kDefaultDigitBits = 9;
std::atomic<int> g_digit_bits{0};
int current_digit_bits() {
    const int b = g_digit_bits.load();
    return b == 0 ? kDefaultDigitBits : b;
}
// The width a product with n output columns per plane takes.  At the default,
// thin products (n <= 32, e.g. PC-Mv) are bound by the accumulator drains,
// not by the tensor pipe: 8-bit digits (exact FP32 chunks of 1024) halve the
// drains for one more digit product (measured 6% faster on 16384^2 x 32).
int digit_bits_for(int64_t n) {
    const int b = g_digit_bits.load();
    if (b != 0) return b;
    return n <= 32 ? 8 : kDefaultDigitBits;
}

bool path_ok(int path) {
    return path == MODPP_PATH_F16 || path == MODPP_PATH_FP64 || path == MODPP_PATH_FP64_TIGHT;
}

struct PlaneIn {
    const uint64_t *A;
    int64_t lda;
    uint64_t q;
    uint64_t *C;
    int64_t ldc;
};

// ------------------------------------------------------------ f16 layout
struct F16Layout {
    int b = 0;
    int L = 0;
    bool pair = false;  // CTA-pair GEMM
    int nc = 0;  // tile columns
    int64_t kp = 0, n_blocks = 0, rows = 0;
    size_t off_u16 = 0, off_d = 0, total = 0;
};

// CTA-pair GEMM (tiles of 256 rows, cta_group::2) for single-problem
// products: chosen process-wide (modpp_set_gemm_pair, MODPP_GEMM_PAIR), for
// outputs of at least 256 rows and more than 64 columns (thin outputs keep
// the one-CTA kernel's plane-fastest order).
std::atomic<int> g_gemm_pair{[] {
    const char *v = std::getenv("MODPP_GEMM_PAIR");
    return (v != nullptr && v[0] != '\0') ? (v[0] != '0' ? 1 : 0) : 0;
}()};
bool use_pair(int64_t d, int64_t n) { return g_gemm_pair.load() != 0 && d >= 2 * kBM && n > 64; }

F16Layout f16_layout(int64_t d, int64_t k, int64_t n, const uint64_t *qs, int planes,
                     bool pair_ok = false) {
    F16Layout lay;
    lay.b = digit_bits_for(n);
    for (int i = 0; i < planes; ++i) {
        const int l = f16_digit_count(qs[i], lay.b);
        if (l > lay.L) lay.L = l;
    }
    lay.pair = pair_ok && use_pair(d, n);
    const int nc = lay.pair ? pair_tile_cols(lay.L) : tile_cols_for(lay.L, n);
    lay.nc = nc;
    lay.kp = (k + 7) / 8 * 8;
    lay.n_blocks = (n + nc - 1) / nc;
    lay.rows = static_cast<int64_t>(planes) * lay.n_blocks * lay.L * nc;
    lay.off_u16 = kHeaderBytes;
    lay.off_d = lay.off_u16 + align_up(static_cast<size_t>(d) * lay.kp * 2);
    lay.total = lay.off_d + align_up(static_cast<size_t>(lay.rows) * lay.kp * 2);
    return lay;
}

// ------------------------------------------------------------ fp64 layout
struct Fp64Layout {
    uint64_t base = 0;
    int k1max = 0;
    size_t off_u = 0, off_a = 0, off_p = 0, off_cublas = 0, total = 0;
};

uint64_t isqrt_u64(uint64_t x) {
    uint64_t r = 0;
    for (int b = 31; b >= 0; --b) {
        const uint64_t c = r | (uint64_t(1) << b);
        if (static_cast<unsigned __int128>(c) * c <= x) r = c;
    }
    return r;
}

// Lemma le:strategy1: K = floor(sqrt(2^53 / d2)).  The tight variant takes
// the largest base with d2 * 128 * (K - 1) < 2^53 for the residue operand,
// since |U| <= 128 needs a single digit.
uint64_t fp64_base(int64_t k, bool tight) {
    const uint64_t two53 = uint64_t(1) << 53;
    if (tight) return two53 / (static_cast<uint64_t>(k) * 128u);
    return isqrt_u64(two53 / static_cast<uint64_t>(k));
}

// Smallest count c with K^c > theta (the decomposition needs |r| < K^c).
int fp64_digit_count(uint64_t theta, uint64_t K) {
    int c = 1;
    unsigned __int128 p = K;
    while (p <= theta) {
        p *= K;
        ++c;
    }
    return c;
}

Fp64Layout fp64_layout(int64_t d, int64_t k, int64_t n, const uint64_t *qs, int planes,
                       bool tight) {
    Fp64Layout lay;
    lay.base = fp64_base(k > 0 ? k : 1, tight);
    for (int i = 0; i < planes; ++i) {
        const int c = fp64_digit_count((qs[i] - 1) / 2, lay.base);
        if (c > lay.k1max) lay.k1max = c;
    }
    lay.off_u = kHeaderBytes;
    lay.off_a = lay.off_u + align_up(static_cast<size_t>(d) * k * 8);
    lay.off_p = lay.off_a + align_up(static_cast<size_t>(k) * lay.k1max * n * 8);
    lay.off_cublas = lay.off_p + align_up(static_cast<size_t>(d) * lay.k1max * n * 8);
    lay.total = lay.off_cublas + kCublasWsBytes;
    return lay;
}

// ------------------------------------------------------------ device state
int device_sms() {
    static int cache[kMaxDevices] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
    if (cache[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        cache[dev] = v;
    }
    return cache[dev];
}

uint64_t wait_limit_ns() {
    static uint64_t v = [] {
        const char *e = std::getenv("MODPP_WAIT_LIMIT_MS");
        long ms = e ? std::atol(e) : 2000;
        if (ms <= 0) ms = 2000;
        return static_cast<uint64_t>(ms) * 1000000ull;
    }();
    return v;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult r{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &r) != cudaSuccess ||
            r != cudaDriverEntryPointSuccess)
            return static_cast<EncodeTiledFn>(nullptr);
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// 2-D f16 tensor [outer][inner] (rows of row_elems elements in memory) with
// swizzled boxes of box_inner x box_outer (box_inner * 2 = kRowBytes, the
// swizzle span).  Elements outside the tensor read as zero.
bool make_map_f16_strided(CUtensorMap *m, const void *base, uint64_t inner, uint64_t outer,
                          uint64_t row_elems, uint32_t box_inner, uint32_t box_outer) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {row_elems * 2};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(base), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              kRowBytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

bool make_map_f16(CUtensorMap *m, const void *base, uint64_t inner, uint64_t outer,
                  uint32_t box_inner, uint32_t box_outer) {
    return make_map_f16_strided(m, base, inner, outer, inner, box_inner, box_outer);
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? MODPP_OK : MODPP_ERR_CUDA; }

// ------------------------------------------------------------ kernel timing
struct EventPair {
    cudaEvent_t start = nullptr, stop = nullptr;
};
struct KernelTimer {
    std::vector<EventPair> pool;
    size_t used = 0;
};
constexpr int kTimedKernels = 3;
std::mutex g_prof_mu;
bool g_prof_on = false;
KernelTimer g_timers[kTimedKernels];

// Records the start event of a timed launch; returns the pair to close, or null.
EventPair *timer_begin(int kernel, cudaStream_t st) {
    if (!g_prof_on) return nullptr;
    std::lock_guard<std::mutex> lock(g_prof_mu);
    KernelTimer &t = g_timers[kernel];
    if (t.used == t.pool.size()) {
        EventPair e;
        if (cudaEventCreate(&e.start) != cudaSuccess || cudaEventCreate(&e.stop) != cudaSuccess)
            return nullptr;
        t.pool.push_back(e);
    }
    EventPair *e = &t.pool[t.used++];
    if (cudaEventRecord(e->start, st) != cudaSuccess) return nullptr;
    return e;
}
void timer_end(EventPair *e, cudaStream_t st) {
    if (e) cudaEventRecord(e->stop, st);
}

int zero_outputs(int64_t d, int64_t n, const PlaneIn *pl, int planes, cudaStream_t st) {
    for (int i = 0; i < planes; ++i) {
        if (d == 0 || n == 0) continue;
        cudaError_t e = cudaMemset2DAsync(pl[i].C, static_cast<size_t>(pl[i].ldc) * 8, 0,
                                          static_cast<size_t>(n) * 8, static_cast<size_t>(d), st);
        if (e != cudaSuccess) return MODPP_ERR_CUDA;
    }
    return MODPP_OK;
}

// ------------------------------------------------------------ f16 path
int run_f16(int64_t d, int64_t k, int64_t n, const void *U, int ukind, int64_t ldu,
            const PlaneIn *pl, int planes, void *ws, size_t ws_bytes, cudaStream_t st) {
    uint64_t qs[kMaxPlanes];
    for (int i = 0; i < planes; ++i) qs[i] = pl[i].q;
    const F16Layout lay = f16_layout(d, k, n, qs, planes, /*pair_ok=*/true);
    if (ws_bytes < lay.total) return MODPP_ERR_WORKSPACE;
    if (lay.rows >= (int64_t(1) << 31)) return MODPP_ERR_UNSUPPORTED;
    uint8_t *w = static_cast<uint8_t *>(ws);
    int *status = reinterpret_cast<int *>(w);
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return MODPP_ERR_CUDA;
    if (d == 0 || n == 0) return MODPP_OK;
    if (k == 0) return zero_outputs(d, n, pl, planes, st);

    // A prepared plaintext (kUPrepared: U is already the f16 layout, d rows
    // of kp halves) is read in place; otherwise U is converted into the
    // workspace.
    __half *U16 = ukind == kUPrepared ? static_cast<__half *>(const_cast<void *>(U))
                                      : reinterpret_cast<__half *>(w + lay.off_u16);
    __half *D = reinterpret_cast<__half *>(w + lay.off_d);
    EventPair *ev = nullptr;
    int rc = MODPP_OK;
    if (ukind != kUPrepared) {
        ev = timer_begin(MODPP_KERNEL_U16, st);
        rc = cuda_status(launch_u_to_f16(U, ukind, ldu, static_cast<int>(d), static_cast<int>(k),
                                         static_cast<int>(lay.kp), U16, st));
        timer_end(ev, st);
        if (rc) return rc;
    }

    SplitParams sp{};
    sp.k = static_cast<int>(k);
    sp.n = static_cast<int>(n);
    sp.kp = static_cast<int>(lay.kp);
    sp.n_blocks = static_cast<int>(lay.n_blocks);
    sp.planes = planes;
    sp.digits = lay.L;
    sp.digit_bits = lay.b;
    sp.nc = lay.nc;
    sp.D = D;
    const uint64_t thresh = f16_lift_threshold(lay.L, lay.b);
    for (int i = 0; i < planes; ++i) sp.sp[i] = SplitPlane{pl[i].A, pl[i].lda, pl[i].q, thresh};
    ev = timer_begin(MODPP_KERNEL_SPLIT, st);
    rc = cuda_status(launch_split_digits(sp, st));
    timer_end(ev, st);
    if (rc) return rc;

    CUtensorMap tmU, tmD;
    if (!make_map_f16(&tmU, U16, static_cast<uint64_t>(lay.kp), static_cast<uint64_t>(d), kBK, kBM))
        return MODPP_ERR_CUDA;
    // One box is one CTA's share of a tile's digit rows: all L * nc of them,
    // or half of them for a CTA pair (each CTA stages N / 2 rows of B).
    if (!make_map_f16(&tmD, D, static_cast<uint64_t>(lay.kp), static_cast<uint64_t>(lay.rows), kBK,
                      static_cast<uint32_t>(lay.pair ? lay.L * lay.nc / 2 : lay.L * lay.nc)))
        return MODPP_ERR_CUDA;

    GemmParams gp{};
    gp.d = static_cast<int>(d);
    gp.n = static_cast<int>(n);
    gp.k = static_cast<int>(k);
    const int rows_per_tile = lay.pair ? 2 * kBM : kBM;
    gp.m_blocks = static_cast<int>((d + rows_per_tile - 1) / rows_per_tile);
    gp.n_blocks = static_cast<int>(lay.n_blocks);
    gp.planes = planes;
    gp.kb_total = static_cast<int>((k + kBK - 1) / kBK);
    const int64_t tiles = static_cast<int64_t>(gp.m_blocks) * gp.n_blocks * planes;
    if (tiles >= (int64_t(1) << 31)) return MODPP_ERR_UNSUPPORTED;
    gp.num_tiles = static_cast<int>(tiles);
    // U larger than a slice of L2 and few column blocks: run the planes of a
    // row block together so each U block is read from HBM once.
    gp.plane_fastest = (!lay.pair && static_cast<int64_t>(d) * lay.kp * 2 > (int64_t(48) << 20) &&
                        lay.n_blocks <= 2 && planes > 1)
                           ? 1
                           : 0;
    // Bands of row blocks whose U rows fit the L2 budget (a pair block is
    // twice as tall).
    gp.band_m = band_rows(gp.m_blocks, lay.pair ? 2 * lay.kp : lay.kp);
    gp.status = status;
    gp.timeout_ns = wait_limit_ns();
    for (int i = 0; i < planes; ++i)
        gp.pc[i] = make_plane_const(pl[i].q, lay.b, pl[i].C, pl[i].ldc);
    const int sms = device_sms();
    if (sms <= 0) return MODPP_ERR_CUDA;
    ev = timer_begin(MODPP_KERNEL_GEMM, st);
    rc = cuda_status(lay.pair ? launch_gemm_f16_pair(tmU, tmD, gp, lay.L, lay.b, st)
                              : launch_gemm_f16(tmU, tmD, gp, lay.L, lay.b, sms, st, lay.nc));
    timer_end(ev, st);
    return rc;
}

// ------------------------------------------------------------ fp64 path
std::mutex g_cublas_mu;
cublasHandle_t g_cublas[kMaxDevices] = {nullptr};

int run_fp64(int64_t d, int64_t k, int64_t n, const void *U, int ukind, int64_t ldu,
             const PlaneIn *pl, int planes, void *ws, size_t ws_bytes, cudaStream_t st,
             bool tight) {
    uint64_t qs[kMaxPlanes];
    for (int i = 0; i < planes; ++i) qs[i] = pl[i].q;
    const Fp64Layout lay = fp64_layout(d, k, n, qs, planes, tight);
    if (ws_bytes < lay.total) return MODPP_ERR_WORKSPACE;
    if (lay.k1max > 8) return MODPP_ERR_UNSUPPORTED;
    uint8_t *w = static_cast<uint8_t *>(ws);
    int *status = reinterpret_cast<int *>(w);
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return MODPP_ERR_CUDA;
    if (d == 0 || n == 0) return MODPP_OK;
    if (k == 0) return zero_outputs(d, n, pl, planes, st);

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev >= kMaxDevices) return MODPP_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_cublas_mu);
    if (!g_cublas[dev] && cublasCreate(&g_cublas[dev]) != CUBLAS_STATUS_SUCCESS)
        return MODPP_ERR_CUDA;
    cublasHandle_t h = g_cublas[dev];
    if (cublasSetStream(h, st) != CUBLAS_STATUS_SUCCESS ||
        cublasSetWorkspace(h, w + lay.off_cublas, kCublasWsBytes) != CUBLAS_STATUS_SUCCESS ||
        cublasSetMathMode(h, CUBLAS_DEFAULT_MATH) != CUBLAS_STATUS_SUCCESS)
        return MODPP_ERR_CUDA;

    double *Ud = reinterpret_cast<double *>(w + lay.off_u);
    double *Ad = reinterpret_cast<double *>(w + lay.off_a);
    double *Pd = reinterpret_cast<double *>(w + lay.off_p);
    int rc = cuda_status(
        launch_u_to_f64(U, ukind, ldu, static_cast<int>(d), static_cast<int>(k), Ud, st));
    if (rc) return rc;
    for (int i = 0; i < planes; ++i) {
        const uint64_t q = pl[i].q;
        const int digits = fp64_digit_count((q - 1) / 2, lay.base);
        Fp64SplitParams sp{pl[i].A, pl[i].lda, static_cast<int>(k), static_cast<int>(n), digits, q,
                           lay.base, Ad};
        rc = cuda_status(launch_fp64_split(sp, st));
        if (rc) return rc;
        // Row-major P (d x digits*n) = U (d x k) * Adig (k x digits*n), issued
        // column-major as P^T = Adig^T * U^T.
        const double one = 1.0, zero = 0.0;
        const int m = digits * static_cast<int>(n);
        if (cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, m, static_cast<int>(d), static_cast<int>(k),
                        &one, Ad, m, Ud, static_cast<int>(k), &zero, Pd, m) != CUBLAS_STATUS_SUCCESS)
            return MODPP_ERR_CUDA;
        Fp64RecombineParams rp{};
        rp.P = Pd;
        rp.d = static_cast<int>(d);
        rp.n = static_cast<int>(n);
        rp.digits = digits;
        rp.q = q;
        rp.mu = host_barrett_mu(q);
        uint64_t pk = 1 % q;
        const uint64_t Kq = lay.base % q;
        for (int t = 0; t < digits; ++t) {
            rp.powK[t] = pk;
            rp.powKs[t] = host_shoup(pk, q);
            pk = host_mulmod(pk, Kq, q);
        }
        rp.C = pl[i].C;
        rp.ldc = pl[i].ldc;
        rc = cuda_status(launch_fp64_recombine(rp, st));
        if (rc) return rc;
    }
    return MODPP_OK;
}

// ------------------------------------------------------------ wide products
// C_j = U_j * A_j mod q_j with both operands residues (the products of two
// ciphertext matrices, Alg. 8 step 2).  U_j is split into balanced 8-bit
// digits U_j = sum_i 2^(8 i) U_ji (each an int8 matrix the f16 path takes as
// its plaintext operand); A_j is split once into f16 digits; then, for each
// i, the tensor-core GEMM adds 2^(8 i) * (U_ji * A_j) into C_j mod q_j.
// Wide products run either as digit products (LU x LA per prime) or in the
// multi-modular form of rns_wide.cu (R small-prime products per prime),
// whichever needs fewer tensor-core products (modpp_set_wide_path forces
// one).
std::atomic<int> g_wide_path{0};  // 0 automatic, 1 digits, 2 CRT

struct WideLayout {
    int LU = 0;                 // 8-bit digits of the left operand
    F16Layout f16;              // one plane
    size_t off_udig = 0, off_f16 = 0, total = 0;
    bool rns = false;           // multi-modular form
    RnsPrimes rp{};
    RnsLayout rl{};
};

WideLayout wide_layout(int64_t d, int64_t k, int64_t n, const uint64_t *qs, int P) {
    WideLayout w;
    const int mode = g_wide_path.load();
    if (mode != 1 && k > 0 && rns_choose(k, qs, P, &w.rp)) {
        int digit_products = 0;
        for (int j = 0; j < P; ++j)
            digit_products = std::max(digit_products, f16_digit_count(qs[j], 8) *
                                                          f16_digit_count(qs[j], current_digit_bits()));
        // The CRT form adds two residue passes and a recombination pass
        // (memory-bound): take it when it saves more than 10% of the products.
        if (mode == 2 || w.rp.R * 11 < digit_products * 10) {
            w.rns = true;
            w.rl = rns_layout(d, k, n, w.rp);
            w.total = w.rl.total;
            return w;
        }
    }
    for (int j = 0; j < P; ++j) w.LU = std::max(w.LU, f16_digit_count(qs[j], 8));
    // One plane at a time: the largest per-prime layout (tile widths differ
    // between digit counts, so the largest L need not have the most rows).
    for (int j = 0; j < P; ++j) {
        const F16Layout l = f16_layout(d, k, n, &qs[j], 1);
        if (l.total > w.f16.total) w.f16 = l;
    }
    w.off_udig = kHeaderBytes;
    w.off_f16 = w.off_udig + align_up(static_cast<size_t>(w.LU) * d * k);
    w.total = w.off_f16 + w.f16.total;
    return w;
}

// CRT form of the wide products for one or two right operands sharing U
// (A2 / C2 null for one): per chain prime, U's residue planes are formed once.
int run_rns_wide(int64_t d, int64_t k, int64_t n, const uint64_t *U, int64_t ldu, int64_t strideU,
                 const uint64_t *A1, const uint64_t *A2, int64_t lda, int64_t strideA,
                 uint64_t *C1, uint64_t *C2, int64_t ldc, int64_t strideC, const uint64_t *primes,
                 int P, const WideLayout &wl, uint8_t *w, cudaStream_t st) {
    const RnsLayout &rl = wl.rl;
    const int sms = device_sms();
    if (sms <= 0) return MODPP_ERR_CUDA;
    // One pair of maps per chunk of the inner dimension: base at the chunk's
    // first index, inner extent the chunk (reads past it are zero), row
    // stride kp.
    CUtensorMap tmU[kMaxRnsChunks], tmD[kMaxRnsChunks];
    for (int ch = 0; ch < wl.rp.chunks; ++ch) {
        const int64_t k0 = ch * wl.rp.chunk_len;
        const int64_t len = std::min<int64_t>(wl.rp.chunk_len, rl.kp - k0);
        if (!make_map_f16_strided(&tmU[ch], w + rl.off_u16 + k0 * 2, static_cast<uint64_t>(len),
                                  static_cast<uint64_t>(wl.rp.R) * d,
                                  static_cast<uint64_t>(rl.kp), kBK, kBM) ||
            !make_map_f16_strided(&tmD[ch], w + rl.off_d + k0 * 2, static_cast<uint64_t>(len),
                                  static_cast<uint64_t>(wl.rp.R) * rl.nblk * kRnsTileCols,
                                  static_cast<uint64_t>(rl.kp), kBK, kRnsTileCols))
            return MODPP_ERR_CUDA;
    }
    for (int j = 0; j < P; ++j) {
        for (int op = 0; op < (A2 ? 2 : 1); ++op) {
            const uint64_t *A = (op == 0 ? A1 : A2) + static_cast<int64_t>(j) * strideA;
            uint64_t *C = (op == 0 ? C1 : C2) + static_cast<int64_t>(j) * strideC;
            EventPair *ev = timer_begin(MODPP_KERNEL_SPLIT, st);
            int rc = rns_split(d, k, n, U + static_cast<int64_t>(j) * strideU, ldu, A, lda,
                               primes[j], wl.rp, rl, w, op == 0, st);
            timer_end(ev, st);
            if (rc) return rc;
            ev = timer_begin(MODPP_KERNEL_GEMM, st);
            rc = rns_gemm(d, k, n, wl.rp, rl, w, reinterpret_cast<int *>(w), wait_limit_ns(), sms,
                          tmU, tmD, st);
            timer_end(ev, st);
            if (rc) return rc;
            ev = timer_begin(MODPP_KERNEL_U16, st);
            rc = rns_crt(d, n, C, ldc, primes[j], wl.rp, rl, w, st);
            timer_end(ev, st);
            if (rc) return rc;
        }
    }
    return MODPP_OK;
}

int run_f16_wide(int64_t d, int64_t k, int64_t n, const uint64_t *U, int64_t ldu, int64_t strideU,
                 const uint64_t *A, int64_t lda, int64_t strideA, uint64_t *C, int64_t ldc,
                 int64_t strideC, const uint64_t *primes, int P, void *ws, size_t ws_bytes,
                 cudaStream_t st) {
    const WideLayout wl = wide_layout(d, k, n, primes, P);
    if (ws_bytes < wl.total) return MODPP_ERR_WORKSPACE;
    uint8_t *w = static_cast<uint8_t *>(ws);
    if (cudaMemsetAsync(w, 0, sizeof(int), st) != cudaSuccess) return MODPP_ERR_CUDA;
    if (d == 0 || n == 0) return MODPP_OK;
    if (wl.rns)
        return run_rns_wide(d, k, n, U, ldu, strideU, A, nullptr, lda, strideA, C, nullptr, ldc,
                            strideC, primes, P, wl, w, st);
    int8_t *Udig = reinterpret_cast<int8_t *>(w + wl.off_udig);
    uint8_t *wf = w + wl.off_f16;  // the f16 path's workspace (one plane)
    const F16Layout &lay = wl.f16;
    __half *U16 = reinterpret_cast<__half *>(wf + lay.off_u16);
    __half *D = reinterpret_cast<__half *>(wf + lay.off_d);
    const int sms = device_sms();
    if (sms <= 0) return MODPP_ERR_CUDA;
    for (int j = 0; j < P; ++j) {
        const uint64_t q = primes[j];
        uint64_t *Cj = C + static_cast<int64_t>(j) * strideC;
        if (k == 0) {
            PlaneIn pz{nullptr, n, q, Cj, ldc};
            const int rc = zero_outputs(d, n, &pz, 1, st);
            if (rc) return rc;
            continue;
        }
        const int LU = f16_digit_count(q, 8);
        int rc = cuda_status(launch_u64_to_i8_digits(U + static_cast<int64_t>(j) * strideU, ldu,
                                                     static_cast<int>(d), static_cast<int>(k), q,
                                                     f16_lift_threshold(LU, 8), LU, Udig, st));
        if (rc) return rc;
        // f16 digits of A_j (the plane's own digit count; the layout holds the largest).
        const int L = f16_digit_count(q, lay.b);
        const int nc = tile_cols_for(L, n);  // as f16_layout for this prime
        const int64_t nblk = (n + nc - 1) / nc;
        const int64_t rows = nblk * L * nc;
        SplitParams sp{};
        sp.nc = nc;
        sp.k = static_cast<int>(k);
        sp.n = static_cast<int>(n);
        sp.kp = static_cast<int>(lay.kp);
        sp.n_blocks = static_cast<int>(nblk);
        sp.planes = 1;
        sp.digits = L;
        sp.digit_bits = lay.b;
        sp.D = D;
        sp.sp[0] = SplitPlane{A + static_cast<int64_t>(j) * strideA, lda, q,
                              f16_lift_threshold(L, lay.b)};
        rc = cuda_status(launch_split_digits(sp, st));
        if (rc) return rc;
        CUtensorMap tmU, tmD;
        if (!make_map_f16(&tmU, U16, static_cast<uint64_t>(lay.kp), static_cast<uint64_t>(d), kBK,
                          kBM) ||
            !make_map_f16(&tmD, D, static_cast<uint64_t>(lay.kp), static_cast<uint64_t>(rows), kBK,
                          static_cast<uint32_t>(L * nc)))
            return MODPP_ERR_CUDA;
        GemmParams gp{};
        gp.d = static_cast<int>(d);
        gp.n = static_cast<int>(n);
        gp.k = static_cast<int>(k);
        gp.m_blocks = static_cast<int>((d + kBM - 1) / kBM);
        gp.n_blocks = static_cast<int>(nblk);
        gp.planes = 1;
        gp.kb_total = static_cast<int>((k + kBK - 1) / kBK);
        const int64_t tiles = static_cast<int64_t>(gp.m_blocks) * gp.n_blocks;
        if (tiles >= (int64_t(1) << 31)) return MODPP_ERR_UNSUPPORTED;
        gp.num_tiles = static_cast<int>(tiles);
        gp.band_m = band_rows(gp.m_blocks, lay.kp);
        gp.status = reinterpret_cast<int *>(w);
        gp.timeout_ns = wait_limit_ns();
        uint64_t w8 = 1 % q;
        for (int i = 0; i < LU; ++i) {
            rc = cuda_status(launch_u_to_f16(Udig + static_cast<int64_t>(i) * d * k, MODPP_U_I8, k,
                                             static_cast<int>(d), static_cast<int>(k),
                                             static_cast<int>(lay.kp), U16, st));
            if (rc) return rc;
            gp.pc[0] = make_plane_const(q, lay.b, Cj, ldc);
            gp.pc[0].wout = w8;
            gp.pc[0].wouts = host_shoup(w8, q);
            gp.pc[0].accumulate = i > 0 ? 1 : 0;
            EventPair *ev = timer_begin(MODPP_KERNEL_GEMM, st);
            rc = cuda_status(launch_gemm_f16(tmU, tmD, gp, L, lay.b, sms, st, nc));
            timer_end(ev, st);
            if (rc) return rc;
            w8 = host_mulmod(w8, 256 % q, q);
        }
    }
    return MODPP_OK;
}

// Debug-mode value checks of a product's inputs, after its launches (the
// inputs are read-only and the call's status word was cleared at its start):
// the residue planes of A bounded by their primes and, for int32 U, the
// plaintext range [-128, 127].  Off unless debug_checks_on().
int debug_check_inputs(int64_t d, int64_t k, int64_t n, const void *U, int ukind, int64_t ldu,
                       const uint64_t *A, int64_t lda, int64_t strideA, const uint64_t *primes,
                       int P, void *ws, cudaStream_t st) {
    if (!debug_checks_on() || d == 0 || n == 0 || k == 0) return MODPP_OK;
    int *status = static_cast<int *>(ws);
    cudaError_t e = range_planes(A, P, k, n, lda, strideA, primes, P, status, st);
    if (e == cudaSuccess && ukind == MODPP_U_I32)
        e = launch_range_i32(static_cast<const int32_t *>(U), d, k, ldu, status, st);
    return cuda_status(e);
}

// The same for wide products: U_j and A_j (and A2_j) residues mod q_j.
int debug_check_wide(int64_t d, int64_t k, int64_t n, const uint64_t *U, int64_t ldu,
                     int64_t strideU, const uint64_t *A1, const uint64_t *A2, int64_t lda,
                     int64_t strideA, const uint64_t *primes, int P, void *ws, cudaStream_t st) {
    if (!debug_checks_on() || d == 0 || n == 0 || k == 0) return MODPP_OK;
    int *status = static_cast<int *>(ws);
    cudaError_t e = cudaSuccess;
    if (U) e = range_planes(U, P, d, k, ldu, strideU, primes, P, status, st);
    if (e == cudaSuccess && A1) e = range_planes(A1, P, k, n, lda, strideA, primes, P, status, st);
    if (e == cudaSuccess && A2) e = range_planes(A2, P, k, n, lda, strideA, primes, P, status, st);
    return cuda_status(e);
}

// ------------------------------------------------------------ Strategy 2
// Approximate Mod-PP-MM of one modulus from the high-order bits of the
// residue operand (Sec. 6.1, "Strategy 2: truncation").
//
// F16 form: each centred residue x of B is rounded to the nearest multiple
// of 2^s, y = floor((x + 2^(s-1)) / 2^s); C = 2^s * (U * y) mod q exactly
// (the digit GEMM on y's balanced digits, whose epilogue multiplies by 2^s).
// Balanced b-bit digits of y: the fewest L whose window
// [-2^(b-1) S_L, (2^(b-1) - 1) S_L], S_L = sum_{i<L} 2^(b i), holds every y.
struct TruncF16Layout {
    F16Layout f16;
    int64_t ymin = 0, ymax = 0;
};
TruncF16Layout trunc_f16_layout(int64_t d, int64_t k, int64_t n, uint64_t q, int s) {
    TruncF16Layout t;
    const int64_t half = static_cast<int64_t>((q - 1) / 2);
    const int64_t rnd = s > 0 ? (int64_t(1) << (s - 1)) : 0;
    t.ymax = (half + rnd) >> s;
    t.ymin = (-half + rnd) >> s;  // arithmetic shift: floor
    F16Layout &lay = t.f16;
    lay.b = current_digit_bits();
    lay.L = 0;
    for (int L = 1; L <= kMaxDigits; ++L) {
        unsigned __int128 S = 0;
        for (int i = 0; i < L; ++i) S += static_cast<unsigned __int128>(1) << (lay.b * i);
        const unsigned __int128 lo = S << (lay.b - 1);
        const unsigned __int128 hi = S * ((1u << (lay.b - 1)) - 1u);
        if (static_cast<unsigned __int128>(-t.ymin) <= lo &&
            static_cast<unsigned __int128>(t.ymax) <= hi) {
            lay.L = L;
            break;
        }
    }
    if (lay.L == 0) return t;
    const int nc = tile_cols_for(lay.L, n);
    lay.nc = nc;
    lay.kp = (k + 7) / 8 * 8;
    lay.n_blocks = (n + nc - 1) / nc;
    lay.rows = lay.n_blocks * lay.L * nc;
    lay.off_u16 = kHeaderBytes;
    lay.off_d = lay.off_u16 + align_up(static_cast<size_t>(d) * lay.kp * 2);
    lay.total = lay.off_d + align_up(static_cast<size_t>(lay.rows) * lay.kp * 2);
    return t;
}

int run_f16_trunc(int64_t d, int64_t k, int64_t n, const void *U, int ukind, int64_t ldu,
                  const uint64_t *B, int64_t ldb, uint64_t *C, int64_t ldc, uint64_t q, int s,
                  void *ws, size_t ws_bytes, cudaStream_t st) {
    const TruncF16Layout tl = trunc_f16_layout(d, k, n, q, s);
    const F16Layout &lay = tl.f16;
    if (lay.L == 0) return MODPP_ERR_UNSUPPORTED;
    if (ws_bytes < lay.total) return MODPP_ERR_WORKSPACE;
    if (lay.rows >= (int64_t(1) << 31)) return MODPP_ERR_UNSUPPORTED;
    uint8_t *w = static_cast<uint8_t *>(ws);
    int *status = reinterpret_cast<int *>(w);
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return MODPP_ERR_CUDA;
    PlaneIn pl{B, ldb, q, C, ldc};
    if (d == 0 || n == 0) return MODPP_OK;
    if (k == 0) return zero_outputs(d, n, &pl, 1, st);

    __half *U16 = reinterpret_cast<__half *>(w + lay.off_u16);
    __half *D = reinterpret_cast<__half *>(w + lay.off_d);
    int rc = cuda_status(launch_u_to_f16(U, ukind, ldu, static_cast<int>(d), static_cast<int>(k),
                                         static_cast<int>(lay.kp), U16, st));
    if (rc) return rc;
    SplitParams sp{};
    sp.k = static_cast<int>(k);
    sp.n = static_cast<int>(n);
    sp.kp = static_cast<int>(lay.kp);
    sp.n_blocks = static_cast<int>(lay.n_blocks);
    sp.planes = 1;
    sp.digits = lay.L;
    sp.digit_bits = lay.b;
    sp.nc = lay.nc;
    sp.D = D;
    // Centred lift (values above (q-1)/2 become x - q), then the rounding shift.
    sp.sp[0] = SplitPlane{B, ldb, q, (q - 1) / 2, s};
    rc = cuda_status(launch_split_digits(sp, st));
    if (rc) return rc;

    CUtensorMap tmU, tmD;
    if (!make_map_f16(&tmU, U16, static_cast<uint64_t>(lay.kp), static_cast<uint64_t>(d), kBK, kBM) ||
        !make_map_f16(&tmD, D, static_cast<uint64_t>(lay.kp), static_cast<uint64_t>(lay.rows), kBK,
                      static_cast<uint32_t>(lay.L * lay.nc)))
        return MODPP_ERR_CUDA;
    GemmParams gp{};
    gp.d = static_cast<int>(d);
    gp.n = static_cast<int>(n);
    gp.k = static_cast<int>(k);
    gp.m_blocks = static_cast<int>((d + kBM - 1) / kBM);
    gp.n_blocks = static_cast<int>(lay.n_blocks);
    gp.planes = 1;
    gp.kb_total = static_cast<int>((k + kBK - 1) / kBK);
    const int64_t tiles = static_cast<int64_t>(gp.m_blocks) * gp.n_blocks;
    if (tiles >= (int64_t(1) << 31)) return MODPP_ERR_UNSUPPORTED;
    gp.num_tiles = static_cast<int>(tiles);
    gp.band_m = band_rows(gp.m_blocks, lay.kp);
    gp.status = status;
    gp.timeout_ns = wait_limit_ns();
    gp.pc[0] = make_plane_const(q, lay.b, C, ldc);
    if (s > 0) {  // C <- 2^s * (U * y) mod q
        gp.pc[0].accumulate = 2;
        gp.pc[0].wout = host_pow2_mod(s, q);
        gp.pc[0].wouts = host_shoup(gp.pc[0].wout, q);
    }
    const int sms = device_sms();
    if (sms <= 0) return MODPP_ERR_CUDA;
    EventPair *ev = timer_begin(MODPP_KERNEL_GEMM, st);
    rc = cuda_status(launch_gemm_f16(tmU, tmD, gp, lay.L, lay.b, sms, st, lay.nc));
    timer_end(ev, st);
    return rc;
}

// FP64 form, as printed: the centred entries of B rounded to the nearest
// double (53 bits), one cuBLAS DGEMM with U, and the exact residue of every
// integer-valued double product.
struct TruncFp64Layout {
    size_t off_u = 0, off_b = 0, off_p = 0, off_cublas = 0, total = 0;
};
TruncFp64Layout trunc_fp64_layout(int64_t d, int64_t k, int64_t n) {
    TruncFp64Layout lay;
    lay.off_u = kHeaderBytes;
    lay.off_b = lay.off_u + align_up(static_cast<size_t>(d) * k * 8);
    lay.off_p = lay.off_b + align_up(static_cast<size_t>(k) * n * 8);
    lay.off_cublas = lay.off_p + align_up(static_cast<size_t>(d) * n * 8);
    lay.total = lay.off_cublas + kCublasWsBytes;
    return lay;
}

int run_fp64_trunc(int64_t d, int64_t k, int64_t n, const void *U, int ukind, int64_t ldu,
                   const uint64_t *B, int64_t ldb, uint64_t *C, int64_t ldc, uint64_t q, void *ws,
                   size_t ws_bytes, cudaStream_t st) {
    const TruncFp64Layout lay = trunc_fp64_layout(d, k, n);
    if (ws_bytes < lay.total) return MODPP_ERR_WORKSPACE;
    uint8_t *w = static_cast<uint8_t *>(ws);
    int *status = reinterpret_cast<int *>(w);
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return MODPP_ERR_CUDA;
    PlaneIn pl{B, ldb, q, C, ldc};
    if (d == 0 || n == 0) return MODPP_OK;
    if (k == 0) return zero_outputs(d, n, &pl, 1, st);
    if (d >= (int64_t(1) << 31) || n >= (int64_t(1) << 31)) return MODPP_ERR_UNSUPPORTED;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev >= kMaxDevices) return MODPP_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_cublas_mu);
    if (!g_cublas[dev] && cublasCreate(&g_cublas[dev]) != CUBLAS_STATUS_SUCCESS)
        return MODPP_ERR_CUDA;
    cublasHandle_t h = g_cublas[dev];
    if (cublasSetStream(h, st) != CUBLAS_STATUS_SUCCESS ||
        cublasSetWorkspace(h, w + lay.off_cublas, kCublasWsBytes) != CUBLAS_STATUS_SUCCESS ||
        cublasSetMathMode(h, CUBLAS_DEFAULT_MATH) != CUBLAS_STATUS_SUCCESS)
        return MODPP_ERR_CUDA;
    double *Ud = reinterpret_cast<double *>(w + lay.off_u);
    double *Bd = reinterpret_cast<double *>(w + lay.off_b);
    double *Pd = reinterpret_cast<double *>(w + lay.off_p);
    int rc = cuda_status(
        launch_u_to_f64(U, ukind, ldu, static_cast<int>(d), static_cast<int>(k), Ud, st));
    if (rc) return rc;
    // One signed "digit" of base 2^63: the centred residue itself, converted
    // to the nearest double.
    Fp64SplitParams sp{B, ldb, static_cast<int>(k), static_cast<int>(n), 1, q,
                       uint64_t(1) << 63, Bd};
    rc = cuda_status(launch_fp64_split(sp, st));
    if (rc) return rc;
    const double one = 1.0, zero = 0.0;
    if (cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, static_cast<int>(n), static_cast<int>(d),
                    static_cast<int>(k), &one, Bd, static_cast<int>(n), Ud, static_cast<int>(k),
                    &zero, Pd, static_cast<int>(n)) != CUBLAS_STATUS_SUCCESS)
        return MODPP_ERR_CUDA;
    Fp64ResidueParams rp{};
    rp.P = Pd;
    rp.d = static_cast<int>(d);
    rp.n = static_cast<int>(n);
    rp.q = q;
    rp.mu = host_barrett_mu(q);
    for (int e = 0; e < kMaxPow2Shift; ++e) {
        rp.pow2[e] = host_pow2_mod(e, q);
        rp.pow2s[e] = host_shoup(rp.pow2[e], q);
    }
    rp.C = C;
    rp.ldc = ldc;
    return cuda_status(launch_fp64_residue(rp, st));
}

size_t layout_bytes(int64_t d, int64_t k, int64_t n, const uint64_t *qs, int planes, int path) {
    if (path == MODPP_PATH_F16) return f16_layout(d, k, n, qs, planes, /*pair_ok=*/true).total;
    return fp64_layout(d, k, n, qs, planes, path == MODPP_PATH_FP64_TIGHT).total;
}

int dispatch(int64_t d, int64_t k, int64_t n, const void *U, int ukind, int64_t ldu,
             const PlaneIn *pl, int planes, int path, void *ws, size_t ws_bytes, void *stream) {
    if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)) != 0)
        return MODPP_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (path == MODPP_PATH_F16) return run_f16(d, k, n, U, ukind, ldu, pl, planes, ws, ws_bytes, st);
    return run_fp64(d, k, n, U, ukind, ldu, pl, planes, ws, ws_bytes, st,
                    path == MODPP_PATH_FP64_TIGHT);
}

int pc_common(int64_t d, int64_t kct, int64_t N, const void *U, const uint64_t *A,
              const uint64_t *B, uint64_t *Aout, uint64_t *Bout, const uint64_t *primes, int P,
              int path, void *ws, size_t ws_bytes, void *stream, int ukind = MODPP_U_I8) {
    int rc = check_sizes(d, kct, N);
    if (rc) return rc;
    rc = check_primes(primes, P, kMaxPlanes / 2);
    if (rc) return rc;
    if (!path_ok(path)) return MODPP_ERR_ARG;
    const bool work = d > 0 && N > 0;
    if (work && (Aout == nullptr || Bout == nullptr)) return MODPP_ERR_ARG;
    if (work && kct > 0 && (U == nullptr || A == nullptr || B == nullptr)) return MODPP_ERR_ARG;
    PlaneIn pl[kMaxPlanes];
    for (int j = 0; j < P; ++j) {
        pl[j] = PlaneIn{A + static_cast<int64_t>(j) * kct * N, N, primes[j],
                        Aout + static_cast<int64_t>(j) * d * N, N};
        pl[P + j] = PlaneIn{B + static_cast<int64_t>(j) * kct * N, N, primes[j],
                            Bout + static_cast<int64_t>(j) * d * N, N};
    }
    rc = dispatch(d, kct, N, U, ukind, kct, pl, 2 * P, path, ws, ws_bytes, stream);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rc = debug_check_inputs(d, kct, N, U, MODPP_U_I8, kct, A, N, kct * N, primes, P, ws, st);
    if (rc) return rc;
    return debug_check_inputs(d, kct, N, U, MODPP_U_I8, kct, B, N, kct * N, primes, P, ws, st);
}

}  // namespace

// ====================================================================== ABI
namespace modpp {
// Self-test of the bounded device waits: one thread waits on an mbarrier
// that nothing ever arrives at; the wait must give up after limit_ns and the
// kernel must return, recording MODPP_ERR_TIMEOUT in the status word.
__global__ void bounded_wait_selftest_kernel(int *status, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0, &abort_flag, limit_ns))
        atomicExch(status, MODPP_ERR_TIMEOUT);
}

int mm_check_args(int64_t d, int64_t k, int64_t n, const void *U, int ukind, int64_t ldu,
                  const uint64_t *A, int64_t lda, int64_t strideA, const uint64_t *C, int64_t ldc,
                  int64_t strideC, const uint64_t *primes_host, int P) {
    int rc = check_sizes(d, k, n);
    if (rc) return rc;
    rc = check_primes(primes_host, P, kMaxPlanes);
    if (rc) return rc;
    if (ukind != MODPP_U_I8 && ukind != MODPP_U_I32) return MODPP_ERR_ARG;
    const bool work = d > 0 && n > 0;
    if (work && C == nullptr) return MODPP_ERR_ARG;
    if (work && k > 0 && (U == nullptr || A == nullptr)) return MODPP_ERR_ARG;
    if (ldu < k || lda < n || ldc < n) return MODPP_ERR_ARG;
    if (P > 1 && (strideA < k * lda || strideC < d * ldc)) return MODPP_ERR_ARG;
    return MODPP_OK;
}
}  // namespace modpp

extern "C" {

const char *modpp_status_string(int status) {
    switch (status) {
        case MODPP_OK: return "MODPP_OK";
        case MODPP_ERR_ARG: return "MODPP_ERR_ARG: invalid size, pointer or leading dimension";
        case MODPP_ERR_PRIME: return "MODPP_ERR_PRIME: prime must be odd, >= 3 and < 2^62";
        case MODPP_ERR_WORKSPACE: return "MODPP_ERR_WORKSPACE: workspace null, misaligned or too small";
        case MODPP_ERR_UNSUPPORTED: return "MODPP_ERR_UNSUPPORTED: request outside this build's limits";
        case MODPP_ERR_CUDA: return "MODPP_ERR_CUDA: a CUDA, driver or cuBLAS call failed";
        case MODPP_ERR_RANGE: return "MODPP_ERR_RANGE: input value outside its documented range";
        case MODPP_ERR_TIMEOUT: return "MODPP_ERR_TIMEOUT: a bounded device wait gave up";
        default: return "unknown modpp status";
    }
}

int modpp_abi_version(void) { return (1 << 16) | 1; }

int modpp_set_digit_bits(int bits) {
    if (bits != 0 && (bits < kMinDigitBits || bits > kMaxDigitBits)) return MODPP_ERR_ARG;
    g_digit_bits.store(bits);
    return MODPP_OK;
}

int modpp_get_digit_bits(void) { return current_digit_bits(); }

int modpp_set_gemm_pair(int on) {
    if (on != 0 && on != 1) return MODPP_ERR_ARG;
    g_gemm_pair.store(on);
    return MODPP_OK;
}

int modpp_get_gemm_pair(void) { return g_gemm_pair.load(); }

int modpp_set_wide_path(int mode) {
    if (mode < 0 || mode > 2) return MODPP_ERR_ARG;
    g_wide_path.store(mode);
    return MODPP_OK;
}

int modpp_get_wide_path(void) { return g_wide_path.load(); }

int modpp_wide_plan_info(int64_t k, const uint64_t *primes_host, int P, int *crt_primes) {
    if (crt_primes == nullptr || P < 1 || primes_host == nullptr) return MODPP_ERR_ARG;
    int rc = check_primes(primes_host, P, kMaxPlanes);
    if (rc) return rc;
    const WideLayout w = wide_layout(1, k, 1, primes_host, P);
    *crt_primes = w.rns ? w.rp.R : 0;
    return MODPP_OK;
}

int modpp_plan_info(int64_t k, uint64_t q, int path, int *digits, int *digit_bits,
                    int64_t *k_chunk) {
    if (k < 1 || k > kMaxK || !prime_ok(q) || !path_ok(path)) return MODPP_ERR_ARG;
    int dg, bits;
    int64_t chunk;
    if (path == MODPP_PATH_F16) {
        bits = current_digit_bits();
        dg = f16_digit_count(q, bits);
        chunk = chunk_k(bits);
    } else {
        const uint64_t K = fp64_base(k, path == MODPP_PATH_FP64_TIGHT);
        dg = fp64_digit_count((q - 1) / 2, K);
        bits = bit_length(K) - 1;
        chunk = k;
    }
    if (digits) *digits = dg;
    if (digit_bits) *digit_bits = bits;
    if (k_chunk) *k_chunk = chunk;
    return MODPP_OK;
}

size_t modpp_mm_workspace(int64_t d, int64_t k, int64_t n, const uint64_t *primes_host, int P,
                          int path) {
    if (check_sizes(d, k, n) || check_primes(primes_host, P, kMaxPlanes) || !path_ok(path))
        return 0;
    return layout_bytes(d, k, n, primes_host, P, path);
}

int modpp_mm(int64_t d, int64_t k, int64_t n, const void *U, int ukind, int64_t ldu,
             const uint64_t *A, int64_t lda, int64_t strideA, uint64_t *C, int64_t ldc,
             int64_t strideC, const uint64_t *primes_host, int P, int path, void *ws,
             size_t ws_bytes, void *stream) {
    if (!path_ok(path)) return MODPP_ERR_ARG;
    const int rc = modpp::mm_check_args(d, k, n, U, ukind, ldu, A, lda, strideA, C, ldc, strideC,
                                        primes_host, P);
    if (rc) return rc;
    PlaneIn pl[kMaxPlanes];
    for (int j = 0; j < P; ++j)
        pl[j] = PlaneIn{A + static_cast<int64_t>(j) * strideA, lda, primes_host[j],
                        C + static_cast<int64_t>(j) * strideC, ldc};
    const int rc2 = dispatch(d, k, n, U, ukind, ldu, pl, P, path, ws, ws_bytes, stream);
    if (rc2) return rc2;
    return debug_check_inputs(d, k, n, U, ukind, ldu, A, lda, strideA, primes_host, P, ws,
                              static_cast<cudaStream_t>(stream));
}

size_t pc_mm_workspace(int64_t d, int64_t kct, int64_t N, const uint64_t *primes_host, int P,
                       int path) {
    if (check_sizes(d, kct, N) || check_primes(primes_host, P, kMaxPlanes / 2) || !path_ok(path))
        return 0;
    uint64_t qs[kMaxPlanes];
    for (int j = 0; j < P; ++j) qs[j] = qs[P + j] = primes_host[j];
    return layout_bytes(d, kct, N, qs, 2 * P, path);
}

int pc_mm(int64_t d, int64_t kct, int64_t N, const int8_t *U, const uint64_t *A,
          const uint64_t *B, uint64_t *Aout, uint64_t *Bout, const uint64_t *primes_host, int P,
          int path, void *ws, size_t ws_bytes, void *stream) {
    return pc_common(d, kct, N, U, A, B, Aout, Bout, primes_host, P, path, ws, ws_bytes, stream);
}

size_t modpp_u16_bytes(int64_t d, int64_t k) {
    if (d < 0 || k < 0 || d >= (int64_t(1) << 31) || k > kMaxK) return 0;
    return align_up(static_cast<size_t>(d) * static_cast<size_t>((k + 7) / 8 * 8) * 2);
}

int modpp_u_to_f16(int64_t d, int64_t k, const void *U, int ukind, int64_t ldu, void *U16,
                   void *stream) {
    if (d < 0 || k < 0 || d >= (int64_t(1) << 31) || k > kMaxK || ldu < k) return MODPP_ERR_ARG;
    if (ukind != MODPP_U_I8 && ukind != MODPP_U_I32) return MODPP_ERR_ARG;
    if (d == 0 || k == 0) return MODPP_OK;
    if (U == nullptr || U16 == nullptr || (reinterpret_cast<uintptr_t>(U16) & 15u) != 0)
        return MODPP_ERR_ARG;
    return cuda_status(launch_u_to_f16(U, ukind, ldu, static_cast<int>(d), static_cast<int>(k),
                                       static_cast<int>((k + 7) / 8 * 8),
                                       static_cast<__half *>(U16),
                                       static_cast<cudaStream_t>(stream)));
}

int pc_mm_u16(int64_t d, int64_t kct, int64_t N, const void *U16, const uint64_t *A,
              const uint64_t *B, uint64_t *Aout, uint64_t *Bout, const uint64_t *primes_host, int P,
              void *ws, size_t ws_bytes, void *stream) {
    if (d > 0 && kct > 0 && N > 0 &&
        (U16 == nullptr || (reinterpret_cast<uintptr_t>(U16) & 15u) != 0))
        return MODPP_ERR_ARG;
    return pc_common(d, kct, N, U16, A, B, Aout, Bout, primes_host, P, MODPP_PATH_F16, ws,
                     ws_bytes, stream, kUPrepared);
}

int pc_mv(int64_t d, int64_t kct, int64_t nvec, const int8_t *U, const uint64_t *A,
          const uint64_t *B, uint64_t *Aout, uint64_t *Bout, const uint64_t *primes_host, int P,
          int path, void *ws, size_t ws_bytes, void *stream) {
    return pc_common(d, kct, nvec, U, A, B, Aout, Bout, primes_host, P, path, ws, ws_bytes,
                     stream);
}

int modpp_profile_enable(int on) {
    std::lock_guard<std::mutex> lock(g_prof_mu);
    g_prof_on = on != 0;
    for (auto &t : g_timers) t.used = 0;
    return MODPP_OK;
}

int modpp_profile_read(int kernel, double *total_ms, int64_t *launches) {
    if (kernel < 0 || kernel >= kTimedKernels) return MODPP_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_prof_mu);
    KernelTimer &t = g_timers[kernel];
    double sum = 0.0;
    for (size_t i = 0; i < t.used; ++i) {
        float ms = 0.f;
        if (cudaEventSynchronize(t.pool[i].stop) != cudaSuccess ||
            cudaEventElapsedTime(&ms, t.pool[i].start, t.pool[i].stop) != cudaSuccess)
            return MODPP_ERR_CUDA;
        sum += ms;
    }
    if (total_ms) *total_ms = sum;
    if (launches) *launches = static_cast<int64_t>(t.used);
    t.used = 0;
    return MODPP_OK;
}

size_t modpp_mm_wide_workspace(int64_t d, int64_t k, int64_t n, const uint64_t *primes_host,
                               int P) {
    if (check_sizes(d, k, n) || check_primes(primes_host, P, kMaxPlanes)) return 0;
    return wide_layout(d, k, n, primes_host, P).total;
}

int modpp_mm_wide(int64_t d, int64_t k, int64_t n, const uint64_t *U, int64_t ldu, int64_t strideU,
                  const uint64_t *A, int64_t lda, int64_t strideA, uint64_t *C, int64_t ldc,
                  int64_t strideC, const uint64_t *primes_host, int P, void *ws, size_t ws_bytes,
                  void *stream) {
    int rc = check_sizes(d, k, n);
    if (rc) return rc;
    rc = check_primes(primes_host, P, kMaxPlanes);
    if (rc) return rc;
    const bool work = d > 0 && n > 0;
    if (work && C == nullptr) return MODPP_ERR_ARG;
    if (work && k > 0 && (U == nullptr || A == nullptr)) return MODPP_ERR_ARG;
    if (ldu < k || lda < n || ldc < n) return MODPP_ERR_ARG;
    if (P > 1 && (strideU < d * ldu || strideA < k * lda || strideC < d * ldc)) return MODPP_ERR_ARG;
    if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)) != 0)
        return MODPP_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rc = run_f16_wide(d, k, n, U, ldu, strideU, A, lda, strideA, C, ldc, strideC, primes_host, P,
                      ws, ws_bytes, st);
    if (rc) return rc;
    return debug_check_wide(d, k, n, U, ldu, strideU, A, nullptr, lda, strideA, primes_host, P,
                            ws, st);
}

int modpp_mm_wide_pair(int64_t d, int64_t k, int64_t n, const uint64_t *U, int64_t ldu,
                       int64_t strideU, const uint64_t *A1, const uint64_t *A2, int64_t lda,
                       int64_t strideA, uint64_t *C1, uint64_t *C2, int64_t ldc, int64_t strideC,
                       const uint64_t *primes_host, int P, void *ws, size_t ws_bytes,
                       void *stream) {
    int rc = check_sizes(d, k, n);
    if (rc) return rc;
    rc = check_primes(primes_host, P, kMaxPlanes);
    if (rc) return rc;
    const WideLayout wl = wide_layout(d, k, n, primes_host, P);
    if (!wl.rns || d == 0 || n == 0 || k == 0) {
        rc = modpp_mm_wide(d, k, n, U, ldu, strideU, A1, lda, strideA, C1, ldc, strideC,
                           primes_host, P, ws, ws_bytes, stream);
        if (rc) return rc;
        rc = modpp_mm_wide(d, k, n, U, ldu, strideU, A2, lda, strideA, C2, ldc, strideC,
                           primes_host, P, ws, ws_bytes, stream);
        if (rc) return rc;
        // The second call cleared the status word: check the first operand again.
        return debug_check_wide(d, k, n, nullptr, ldu, strideU, A1, nullptr, lda, strideA,
                                primes_host, P, ws, static_cast<cudaStream_t>(stream));
    }
    if (!U || !A1 || !A2 || !C1 || !C2) return MODPP_ERR_ARG;
    if (ldu < k || lda < n || ldc < n) return MODPP_ERR_ARG;
    if (P > 1 && (strideU < d * ldu || strideA < k * lda || strideC < d * ldc)) return MODPP_ERR_ARG;
    if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)) != 0 ||
        ws_bytes < wl.total)
        return MODPP_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint8_t *w = static_cast<uint8_t *>(ws);
    if (cudaMemsetAsync(w, 0, sizeof(int), st) != cudaSuccess) return MODPP_ERR_CUDA;
    rc = run_rns_wide(d, k, n, U, ldu, strideU, A1, A2, lda, strideA, C1, C2, ldc, strideC,
                      primes_host, P, wl, w, st);
    if (rc) return rc;
    return debug_check_wide(d, k, n, U, ldu, strideU, A1, A2, lda, strideA, primes_host, P, ws,
                            st);
}

size_t modpp_mm_trunc_workspace(int64_t d, int64_t k, int64_t n, uint64_t q, int path,
                                int drop_bits) {
    if (check_sizes(d, k, n) || !prime_ok(q)) return 0;
    if (path == MODPP_PATH_F16) {
        if (drop_bits < 0 || drop_bits > bit_length(q)) return 0;
        const TruncF16Layout t = trunc_f16_layout(d, k, n, q, drop_bits);
        return t.f16.L == 0 ? 0 : t.f16.total;
    }
    if (path == MODPP_PATH_FP64 && drop_bits == 0) return trunc_fp64_layout(d, k, n).total;
    return 0;
}

int modpp_mm_trunc(int64_t d, int64_t k, int64_t n, const void *U, int ukind, int64_t ldu,
                   const uint64_t *B, int64_t ldb, uint64_t *C, int64_t ldc, uint64_t q, int path,
                   int drop_bits, void *ws, size_t ws_bytes, void *stream) {
    if (path != MODPP_PATH_F16 && path != MODPP_PATH_FP64) return MODPP_ERR_ARG;
    if (path == MODPP_PATH_F16 ? (drop_bits < 0 || (q >= 3 && drop_bits > bit_length(q)))
                               : drop_bits != 0)
        return MODPP_ERR_ARG;
    const int rc = modpp::mm_check_args(d, k, n, U, ukind, ldu, B, ldb, 0, C, ldc, 0, &q, 1);
    if (rc) return rc;
    if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)) != 0)
        return MODPP_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int rc2 = path == MODPP_PATH_F16
                        ? run_f16_trunc(d, k, n, U, ukind, ldu, B, ldb, C, ldc, q, drop_bits, ws,
                                        ws_bytes, st)
                        : run_fp64_trunc(d, k, n, U, ukind, ldu, B, ldb, C, ldc, q, ws, ws_bytes,
                                         st);
    if (rc2) return rc2;
    // Debug mode: B canonical; int32 U in [-128, 127] on the f16 path only
    // (the binary64 form takes any int32 plaintext).
    return debug_check_inputs(d, k, n, U, path == MODPP_PATH_F16 ? ukind : MODPP_U_I8, ldu, B,
                              ldb, 0, &q, 1, ws, st);
}

int modpp_selftest_bounded_wait(void *ws, uint64_t limit_ns, void *stream) {
    if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || limit_ns == 0 ||
        limit_ns > uint64_t(10) * 1000000000ull)
        return MODPP_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int *status = static_cast<int *>(ws);
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return MODPP_ERR_CUDA;
    bounded_wait_selftest_kernel<<<1, 32, 0, st>>>(status, limit_ns);
    return cuda_status(cudaGetLastError());
}

int modpp_status_read(void *ws, void *stream) {
    if (ws == nullptr) return MODPP_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return MODPP_ERR_CUDA;
    int v = 0;
    if (cudaMemcpy(&v, ws, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return MODPP_ERR_CUDA;
    if (v != 0 && cudaMemset(ws, 0, sizeof(int)) != cudaSuccess) return MODPP_ERR_CUDA;
    return v;
}

}  // extern "C"

namespace modpp {
void *prof_begin(int kernel, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return nullptr;
    return timer_begin(kernel, st);
}
void prof_end(void *handle, cudaStream_t st) { timer_end(static_cast<EventPair *>(handle), st); }
bool profile_active() {
    std::lock_guard<std::mutex> lock(g_prof_mu);
    return g_prof_on;
}
}  // namespace modpp
