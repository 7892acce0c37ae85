// Grouped Mod-PP-MM: many products of uneven d x k x n with their own prime
// lists run in a few launches (one U -> f16 pass, then a digit split and a
// persistent tensor-core GEMM per digit-count class) that walk one table of
// problems.
//
// - A plan (modpp_group_plan_create) lays out the caller's workspace, writes
//   the device tables (one GroupPlane per (problem, prime), the per-problem
//   TMA tensor maps, the pre-pass job lists).  Problems are partitioned by
//   their digit count L (the widest prime decides); each class runs one
//   split launch and one persistent GEMM launch with the tile width chosen
//   for that L, and its planes are ordered longest-K first, so the persistent
//   CTAs take the long tiles before the short ones.
// - The digit width is chosen per plan by an autotuner: it times every
//   candidate width on the plan's own problems and keeps the fastest.  The
//   choice is cached in process, keyed by the problem shapes, prime sizes and
//   GPU name, and optionally in a text file named by MODPP_TUNE_CACHE.
// - modpp_group_run_graph captures the launches in a CUDA graph once and
//   replays it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "gemm_f16_kernel.cuh"
#include "modpp.h"
#include "modpp_internal.h"
#include "split_tile.cuh"

namespace modpp {

// ------------------------------------------------------------ device tables
struct GroupUJob {
    const int8_t *U;
    int64_t ldu;
    int d, k, kp;
    __half *U16;
    int64_t block_begin;  // first block of this job in the flattened grid
};

struct GroupSplitJob {
    const uint64_t *A;
    int64_t lda;
    uint64_t q, thresh;
    int k, n, kp, n_blocks, t_blocks, Lp;
    __half *D;            // first row of this plane's digit block (nb = 0)
    int64_t block_begin;
};

// U elements per block of the U -> f16 pass: 8 per thread and step, 4 steps.
constexpr int kUElemsPerBlock = 8 * 256 * 4;

// Each block of the two pre-passes finds its job in a table with one entry
// per block (written by the plan), not by a search over the job list.
__global__ void __launch_bounds__(256) group_u_to_f16_kernel(const GroupUJob *jobs,
                                                             const int *block_job) {
    const GroupUJob j = jobs[block_job[blockIdx.x]];
    const int groups = j.kp / 8;  // kp is a multiple of 8
    const int64_t total = static_cast<int64_t>(j.d) * groups;
    const int64_t g0 = (blockIdx.x - j.block_begin) * static_cast<int64_t>(kUElemsPerBlock / 8);
    for (int64_t i = g0 + threadIdx.x; i < g0 + kUElemsPerBlock / 8 && i < total; i += 256) {
        const int64_t r = i / groups;
        const int t0 = static_cast<int>(i - r * groups) * 8;
        const int8_t *src = j.U + r * j.ldu + t0;
        __align__(16) __half h[8];
        if (t0 + 8 <= j.k && (reinterpret_cast<uintptr_t>(src) & 7u) == 0) {
            const int2 w = *reinterpret_cast<const int2 *>(src);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int word = q < 4 ? w.x : w.y;
                h[q] = __int2half_rn(static_cast<int8_t>((word >> (8 * (q & 3))) & 0xff));
            }
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q)
                h[q] = __int2half_rn(t0 + q < j.k ? static_cast<int>(src[q]) : 0);
        }
        *reinterpret_cast<uint4 *>(j.U16 + r * j.kp + t0) = *reinterpret_cast<const uint4 *>(h);
    }
}

// Every plane of a class has exactly L = LMAX digits.
template <int LMAX, int DB, int NC>
__global__ void __launch_bounds__(256) group_split_kernel(const GroupSplitJob *jobs,
                                                          const int *block_job) {
    __shared__ __align__(16) __half tile[LMAX * NC * kSplitRow];
    const GroupSplitJob j = jobs[block_job[blockIdx.x]];
    const int64_t lb = blockIdx.x - j.block_begin;
    const int tb = static_cast<int>(lb % j.t_blocks);
    const int nb = static_cast<int>(lb / j.t_blocks);
    __half *Dblock = j.D + static_cast<int64_t>(nb) * LMAX * NC * static_cast<int64_t>(j.kp);
    split_digit_tile<LMAX, DB, NC>(tile, j.A, j.lda, j.q, j.thresh, j.k, j.n, j.kp, LMAX,
                                   tb * kSplitT, nb * NC, Dblock);
}

template <int LMAX, int DB>
static cudaError_t launch_group_kernels(const GroupSplitJob *sjobs, const int *sblock_job,
                                        int64_t s_blocks, const GemmParams &gp, int num_sms,
                                        cudaStream_t st) {
    constexpr int NC = tile_cols(LMAX);
    if (s_blocks > 0) {
        void *ev = prof_begin(MODPP_KERNEL_SPLIT, st);
        group_split_kernel<LMAX, DB, NC><<<static_cast<unsigned>(s_blocks), 256, 0, st>>>(
            sjobs, sblock_job);
        prof_end(ev, st);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (gp.num_tiles == 0) return cudaSuccess;
    CUtensorMap dummy{};
    void *ev = prof_begin(MODPP_KERNEL_GEMM, st);
    const cudaError_t e = launch_gemm_kernel<LMAX, DB, NC, true>(dummy, dummy, gp, num_sms, st);
    prof_end(ev, st);
    return e;
}

template <int DB>
static cudaError_t launch_group_db(int lmax, const GroupSplitJob *sjobs, const int *sblock_job,
                                   int64_t s_blocks, const GemmParams &gp, int num_sms,
                                   cudaStream_t st) {
    switch (lmax) {
#define MODPP_CASE(LL) \
    case LL: return launch_group_kernels<LL, DB>(sjobs, sblock_job, s_blocks, gp, num_sms, st);
        MODPP_CASE(1)
        MODPP_CASE(2)
        MODPP_CASE(3)
        MODPP_CASE(4)
        MODPP_CASE(5)
        MODPP_CASE(6)
        MODPP_CASE(7)
        MODPP_CASE(8)
#undef MODPP_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace modpp

using namespace modpp;

namespace {

constexpr size_t kAlignG = 256;
size_t galign(size_t x) { return (x + kAlignG - 1) & ~(kAlignG - 1); }

struct ProblemCopy {
    modpp_problem p;
    std::vector<uint64_t> primes;
};

struct GroupLayout {
    int b = 0, lmax = 0;
    std::vector<int> Lp;                 // per problem
    std::vector<int> nc;                 // per problem: tile_cols(Lp)
    std::vector<int64_t> kp, n_blocks;   // per problem
    std::vector<size_t> off_u16, off_d;  // per problem
    int num_planes = 0;
    int64_t num_tiles = 0;               // GEMM tiles over all classes
    int64_t u_blocks = 0, s_blocks = 0;  // pre-pass blocks over all problems / classes
    size_t off_planes = 0, off_ujobs = 0, off_sjobs = 0, off_tiles = 0, off_ublk = 0, off_sblk = 0,
           off_maps = 0, total = 0;
};

GroupLayout group_layout(const std::vector<ProblemCopy> &probs, int b) {
    GroupLayout g;
    g.b = b;
    for (const auto &pc : probs) {
        int L = 0;
        for (uint64_t q : pc.primes) L = std::max(L, f16_digit_count(q, b));
        g.Lp.push_back(L);
        g.lmax = std::max(g.lmax, L);
        g.num_planes += pc.p.P;
    }
    for (int L : g.Lp) g.nc.push_back(tile_cols(L));
    for (size_t i = 0; i < probs.size(); ++i) {
        const modpp_problem &p = probs[i].p;
        if (p.d == 0 || p.n == 0 || p.k == 0) continue;
        const int64_t kp = (p.k + 7) / 8 * 8;
        const int64_t nbk = (p.n + g.nc[i] - 1) / g.nc[i];
        g.num_tiles += static_cast<int64_t>(p.P) * ((p.d + kBM - 1) / kBM) * nbk;
        g.u_blocks += (p.d * kp + kUElemsPerBlock - 1) / kUElemsPerBlock;
        g.s_blocks += static_cast<int64_t>(p.P) * ((kp + kSplitT - 1) / kSplitT) * nbk;
    }
    size_t off = 256;  // status word
    g.off_planes = off;
    off = galign(off + sizeof(GroupPlane) * g.num_planes);
    g.off_ujobs = off;
    off = galign(off + sizeof(GroupUJob) * probs.size());
    g.off_sjobs = off;
    off = galign(off + sizeof(GroupSplitJob) * g.num_planes);
    g.off_tiles = off;  // plane of every tile, class-relative (one int per tile)
    off = galign(off + sizeof(int) * static_cast<size_t>(g.num_tiles));
    g.off_ublk = off;   // U job of every U -> f16 block
    off = galign(off + sizeof(int) * static_cast<size_t>(g.u_blocks));
    g.off_sblk = off;   // split job of every split block, class-relative
    off = galign(off + sizeof(int) * static_cast<size_t>(g.s_blocks));
    g.off_maps = off;
    off = galign(off + 2 * sizeof(CUtensorMap) * probs.size());
    for (size_t i = 0; i < probs.size(); ++i) {
        const modpp_problem &p = probs[i].p;
        const int64_t kp = (p.k + 7) / 8 * 8;
        const int64_t nb = (p.n + g.nc[i] - 1) / g.nc[i];
        g.kp.push_back(kp);
        g.n_blocks.push_back(nb);
        g.off_u16.push_back(off);
        off = galign(off + static_cast<size_t>(p.d) * kp * 2);
        g.off_d.push_back(off);
        off = galign(off + static_cast<size_t>(p.P) * nb * g.Lp[i] * g.nc[i] * kp * 2);
    }
    g.total = off;
    return g;
}

int check_problem(const modpp_problem &p) {
    if (p.d < 0 || p.k < 0 || p.n < 0 || p.d >= (int64_t(1) << 31) ||
        p.n >= (int64_t(1) << 31) || p.k > (int64_t(1) << 20))
        return MODPP_ERR_ARG;
    if (p.P < 1 || p.P > kMaxPlanes || p.primes == nullptr) return MODPP_ERR_ARG;
    for (int j = 0; j < p.P; ++j) {
        const uint64_t q = p.primes[j];
        if (q < 3 || !(q & 1u) || q >= (uint64_t(1) << 62)) return MODPP_ERR_PRIME;
    }
    const bool work = p.d > 0 && p.n > 0;
    if (work && p.C == nullptr) return MODPP_ERR_ARG;
    if (work && p.k > 0 && (p.U == nullptr || p.A == nullptr)) return MODPP_ERR_ARG;
    if (p.ldu < p.k || p.lda < p.n || p.ldc < p.n) return MODPP_ERR_ARG;
    if (p.P > 1 && (p.strideA < p.k * p.lda || p.strideC < p.d * p.ldc)) return MODPP_ERR_ARG;
    return MODPP_OK;
}

using EncodeTiledFnG = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                    const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                    const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

bool encode_map(CUtensorMap *m, const void *base, uint64_t inner, uint64_t outer, uint32_t box_outer) {
    static EncodeTiledFnG fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult r{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &r) != cudaSuccess ||
            r != cudaDriverEntryPointSuccess)
            return static_cast<EncodeTiledFnG>(nullptr);
        return reinterpret_cast<EncodeTiledFnG>(p);
    }();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {inner * 2};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(kBK), box_outer};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(base), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              kRowBytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sms_of_current_device() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return v;
}

uint64_t group_wait_limit_ns() {
    const char *e = std::getenv("MODPP_WAIT_LIMIT_MS");
    long ms = e ? std::atol(e) : 2000;
    if (ms <= 0) ms = 2000;
    return static_cast<uint64_t>(ms) * 1000000ull;
}

// ------------------------------------------------------------ tuning cache
std::mutex g_tune_mu;
std::map<std::string, int> g_tune_cache;
bool g_tune_file_loaded = false;

std::string tune_signature(const std::vector<ProblemCopy> &probs) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, dev);
    std::string s = prop.name;
    for (char &c : s)
        if (c == ' ') c = '_';
    char buf[96];
    for (const auto &pc : probs) {
        int maxbits = 0;
        for (uint64_t q : pc.primes) maxbits = std::max(maxbits, bit_length(q - 1));
        std::snprintf(buf, sizeof buf, "|%lldx%lldx%lld:%dx%d", static_cast<long long>(pc.p.d),
                      static_cast<long long>(pc.p.k), static_cast<long long>(pc.p.n), pc.p.P,
                      maxbits);
        s += buf;
    }
    return s;
}

void tune_file_load() {
    if (g_tune_file_loaded) return;
    g_tune_file_loaded = true;
    const char *path = std::getenv("MODPP_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    std::vector<char> line(1 << 16);
    while (std::fgets(line.data(), static_cast<int>(line.size()), f)) {
        char *sp = std::strrchr(line.data(), ' ');
        if (!sp) continue;
        const int b = std::atoi(sp + 1);
        *sp = 0;
        if (b >= kMinDigitBits && b <= kMaxDigitBits) g_tune_cache[line.data()] = b;
    }
    std::fclose(f);
}

void tune_file_append(const std::string &sig, int b) {
    const char *path = std::getenv("MODPP_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d\n", sig.c_str(), b);
    std::fclose(f);
}

}  // namespace

struct GroupClass {
    int L = 0;
    int plane_begin = 0, plane_count = 0;
    int tiles = 0;
    int64_t tile_base = 0;  // first entry of the class in the tile -> plane table
    int64_t s_block_base = 0;  // first entry of the class in the split block -> job table
    int sjob_begin = 0, sjob_count = 0;
    int64_t s_blocks = 0;
};

struct modpp_group_plan {
    int device = 0;
    std::vector<GroupClass> classes;
    std::vector<ProblemCopy> probs;
    uint8_t *ws = nullptr;
    size_t ws_bytes = 0;
    GroupLayout lay;
    std::vector<uint8_t> staging;  // host image of the device tables (kept for async copies)
    GemmParams gp{};
    int n_ujobs = 0, n_sjobs = 0;
    int64_t u_blocks = 0;
    double tuned_ms[kMaxDigitBits + 1] = {0};
    int tuned = 0;  // 1 if the width came from timing, 2 from the cache
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
};

namespace {

// Builds the device tables for digit width b into the plan's workspace.
int plan_build(modpp_group_plan *pl, int b, cudaStream_t st) {
    pl->lay = group_layout(pl->probs, b);
    const GroupLayout &g = pl->lay;
    if (g.total > pl->ws_bytes) return MODPP_ERR_WORKSPACE;
    if (g.lmax < 1 || g.lmax > kMaxDigits) return MODPP_ERR_UNSUPPORTED;
    const size_t table_bytes = g.off_maps + 2 * sizeof(CUtensorMap) * pl->probs.size();
    pl->staging.assign(table_bytes, 0);
    uint8_t *h = pl->staging.data();
    uint8_t *w = pl->ws;
    auto *planes = reinterpret_cast<GroupPlane *>(h + g.off_planes);
    auto *ujobs = reinterpret_cast<GroupUJob *>(h + g.off_ujobs);
    auto *sjobs = reinterpret_cast<GroupSplitJob *>(h + g.off_sjobs);
    auto *maps = reinterpret_cast<CUtensorMap *>(h + g.off_maps);
    auto *tile_plane = reinterpret_cast<int *>(h + g.off_tiles);
    auto *ublock_job = reinterpret_cast<int *>(h + g.off_ublk);
    auto *sblock_job = reinterpret_cast<int *>(h + g.off_sblk);
    int64_t tile_base = 0, s_block_base = 0;
    const auto *dmaps = reinterpret_cast<const CUtensorMap *>(w + g.off_maps);

    // Classes of equal digit count; within a class the longest inner
    // dimension first (ties: larger output first).
    std::vector<int> order(pl->probs.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = static_cast<int>(i);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        if (g.Lp[a] != g.Lp[c]) return g.Lp[a] > g.Lp[c];
        const modpp_problem &pa = pl->probs[a].p, &pc = pl->probs[c].p;
        if (pa.k != pc.k) return pa.k > pc.k;
        return pa.d * pa.n > pc.d * pc.n;
    });

    pl->classes.clear();
    int np = 0, nu = 0, ns = 0;
    int64_t tiles = 0, ublocks = 0, sblocks = 0;
    for (int i : order) {
        const modpp_problem &p = pl->probs[i].p;
        if (p.d == 0 || p.n == 0 || p.k == 0) continue;  // zero-filled separately
        const int Lp = g.Lp[i];
        const int nc = g.nc[i];
        if (pl->classes.empty() || pl->classes.back().L != Lp) {
            if (!pl->classes.empty()) {
                tile_base += pl->classes.back().tiles;
                s_block_base += pl->classes.back().s_blocks;
            }
            GroupClass c;
            c.L = Lp;
            c.plane_begin = np;
            c.sjob_begin = ns;
            c.tile_base = tile_base;
            c.s_block_base = s_block_base;
            pl->classes.push_back(c);
            tiles = 0;
            sblocks = 0;
        }
        GroupClass &cls = pl->classes.back();
        __half *U16 = reinterpret_cast<__half *>(w + g.off_u16[i]);
        __half *D = reinterpret_cast<__half *>(w + g.off_d[i]);
        const int64_t kp = g.kp[i], nbk = g.n_blocks[i];
        const int64_t rows = static_cast<int64_t>(p.P) * nbk * Lp * nc;
        if (rows >= (int64_t(1) << 31)) return MODPP_ERR_UNSUPPORTED;
        if (!encode_map(&maps[2 * i], U16, kp, p.d, kBM) ||
            !encode_map(&maps[2 * i + 1], D, kp, rows, static_cast<uint32_t>(Lp * nc)))
            return MODPP_ERR_CUDA;
        ujobs[nu] = GroupUJob{static_cast<const int8_t *>(p.U), p.ldu, static_cast<int>(p.d),
                              static_cast<int>(p.k), static_cast<int>(kp), U16, ublocks};
        {
            const int64_t nub = (p.d * kp + kUElemsPerBlock - 1) / kUElemsPerBlock;
            if (ublocks + nub > g.u_blocks) return MODPP_ERR_UNSUPPORTED;
            for (int64_t t = 0; t < nub; ++t) ublock_job[ublocks + t] = nu;
            ublocks += nub;
        }
        ++nu;
        const int m_blocks = static_cast<int>((p.d + kBM - 1) / kBM);
        const int tblocks = static_cast<int>((kp + kSplitT - 1) / kSplitT);
        const uint64_t thresh = f16_lift_threshold(Lp, b);
        for (int j = 0; j < p.P; ++j) {
            const uint64_t q = pl->probs[i].primes[j];
            GroupPlane &gpl = planes[np];
            gpl.pc = make_plane_const(q, b, p.C + static_cast<int64_t>(j) * p.strideC, p.ldc);
            gpl.tmU = &dmaps[2 * i];
            gpl.tmD = &dmaps[2 * i + 1];
            gpl.d = static_cast<int>(p.d);
            gpl.n = static_cast<int>(p.n);
            gpl.kb_total = static_cast<int>((p.k + kBK - 1) / kBK);
            gpl.m_blocks = m_blocks;
            gpl.n_blocks = static_cast<int>(nbk);
            gpl.band_m = band_rows(m_blocks, kp);
            gpl.Lp = Lp;
            gpl.dplane = j;
            gpl.tile_begin = static_cast<int>(tiles);
            if (tile_base + tiles + static_cast<int64_t>(m_blocks) * nbk > g.num_tiles)
                return MODPP_ERR_UNSUPPORTED;
            for (int64_t t = 0; t < static_cast<int64_t>(m_blocks) * nbk; ++t)
                tile_plane[tile_base + tiles + t] = np - cls.plane_begin;
            tiles += static_cast<int64_t>(m_blocks) * nbk;
            ++np;
            sjobs[ns] = GroupSplitJob{p.A + static_cast<int64_t>(j) * p.strideA, p.lda, q, thresh,
                                      static_cast<int>(p.k), static_cast<int>(p.n),
                                      static_cast<int>(kp), static_cast<int>(nbk), tblocks, Lp,
                                      D + static_cast<int64_t>(j) * nbk * Lp * nc * kp, sblocks};
            {
                const int64_t nsb = static_cast<int64_t>(tblocks) * nbk;
                if (s_block_base + sblocks + nsb > g.s_blocks) return MODPP_ERR_UNSUPPORTED;
                for (int64_t t = 0; t < nsb; ++t)
                    sblock_job[s_block_base + sblocks + t] = ns - cls.sjob_begin;
                sblocks += nsb;
            }
            ++ns;
        }
        if (tiles >= (int64_t(1) << 31) || sblocks >= (int64_t(1) << 31))
            return MODPP_ERR_UNSUPPORTED;
        cls.plane_count = np - cls.plane_begin;
        cls.sjob_count = ns - cls.sjob_begin;
        cls.tiles = static_cast<int>(tiles);
        cls.s_blocks = sblocks;
    }
    if (ublocks >= (int64_t(1) << 31)) return MODPP_ERR_UNSUPPORTED;
    if (cudaMemcpyAsync(w, h, table_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return MODPP_ERR_CUDA;
    // The staging buffer must outlive the copy.
    if (cudaStreamSynchronize(st) != cudaSuccess) return MODPP_ERR_CUDA;

    GemmParams &gp = pl->gp;
    gp = GemmParams{};
    gp.num_tiles = 0;
    for (const auto &c : pl->classes) gp.num_tiles += c.tiles;
    gp.status = reinterpret_cast<int *>(w);
    gp.timeout_ns = group_wait_limit_ns();
    gp.gplanes = reinterpret_cast<const GroupPlane *>(w + g.off_planes);
    gp.num_gplanes = np;
    pl->n_ujobs = nu;
    pl->n_sjobs = ns;
    pl->u_blocks = ublocks;
    if (pl->gexec) {
        cudaGraphExecDestroy(pl->gexec);
        pl->gexec = nullptr;
    }
    if (pl->graph) {
        cudaGraphDestroy(pl->graph);
        pl->graph = nullptr;
    }
    return MODPP_OK;
}

int plan_enqueue(modpp_group_plan *pl, cudaStream_t st) {
    const GroupLayout &g = pl->lay;
    uint8_t *w = pl->ws;
    if (cudaMemsetAsync(w, 0, sizeof(int), st) != cudaSuccess) return MODPP_ERR_CUDA;
    for (const auto &pc : pl->probs) {  // k = 0: the product is zero
        const modpp_problem &p = pc.p;
        if (p.k != 0 || p.d == 0 || p.n == 0) continue;
        for (int j = 0; j < p.P; ++j)
            if (cudaMemset2DAsync(p.C + static_cast<int64_t>(j) * p.strideC,
                                  static_cast<size_t>(p.ldc) * 8, 0, static_cast<size_t>(p.n) * 8,
                                  static_cast<size_t>(p.d), st) != cudaSuccess)
                return MODPP_ERR_CUDA;
    }
    if (pl->u_blocks > 0) {
        void *ev = prof_begin(MODPP_KERNEL_U16, st);
        group_u_to_f16_kernel<<<static_cast<unsigned>(pl->u_blocks), 256, 0, st>>>(
            reinterpret_cast<const GroupUJob *>(w + g.off_ujobs),
            reinterpret_cast<const int *>(w + g.off_ublk));
        prof_end(ev, st);
        if (cudaGetLastError() != cudaSuccess) return MODPP_ERR_CUDA;
    }
    const int sms = sms_of_current_device();
    if (sms <= 0) return MODPP_ERR_CUDA;
    const auto *sjobs = reinterpret_cast<const GroupSplitJob *>(w + g.off_sjobs);
    for (const GroupClass &c : pl->classes) {
        GemmParams gp = pl->gp;
        gp.gplanes = pl->gp.gplanes + c.plane_begin;
        gp.num_gplanes = c.plane_count;
        gp.tile_plane = reinterpret_cast<const int *>(w + g.off_tiles) + c.tile_base;
        gp.num_tiles = c.tiles;
        const GroupSplitJob *cj = sjobs + c.sjob_begin;
        const int *sbj = reinterpret_cast<const int *>(w + g.off_sblk) + c.s_block_base;
        cudaError_t e;
        switch (g.b) {
            case 8: e = launch_group_db<8>(c.L, cj, sbj, c.s_blocks, gp, sms, st); break;
            case 9: e = launch_group_db<9>(c.L, cj, sbj, c.s_blocks, gp, sms, st); break;
            case 10: e = launch_group_db<10>(c.L, cj, sbj, c.s_blocks, gp, sms, st); break;
            default: return MODPP_ERR_ARG;
        }
        if (e != cudaSuccess) return MODPP_ERR_CUDA;
    }
    // Debug mode: every problem's residues A bounded by its primes (the
    // status word of the plan's workspace; in a captured graph the setting
    // at capture time holds).
    if (debug_checks_on()) {
        for (const auto &pc : pl->probs) {
            const modpp_problem &p = pc.p;
            if (p.k == 0 || p.d == 0 || p.n == 0) continue;
            if (range_planes(p.A, p.P, p.k, p.n, p.lda, p.strideA, pc.primes.data(), p.P,
                             reinterpret_cast<int *>(w), st) != cudaSuccess)
                return MODPP_ERR_CUDA;
        }
    }
    return MODPP_OK;
}

// Times one candidate width on the plan's own problems (median of 3 after a warm-up).
int plan_time(modpp_group_plan *pl, cudaStream_t st, double *ms_out) {
    cudaEvent_t a, c;
    if (cudaEventCreate(&a) != cudaSuccess) return MODPP_ERR_CUDA;
    if (cudaEventCreate(&c) != cudaSuccess) {
        cudaEventDestroy(a);
        return MODPP_ERR_CUDA;
    }
    int rc = plan_enqueue(pl, st);
    std::vector<float> t;
    for (int r = 0; rc == MODPP_OK && r < 3; ++r) {
        cudaEventRecord(a, st);
        rc = plan_enqueue(pl, st);
        cudaEventRecord(c, st);
        if (cudaEventSynchronize(c) != cudaSuccess) rc = MODPP_ERR_CUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, c);
        t.push_back(ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(c);
    if (rc == MODPP_OK) {
        std::sort(t.begin(), t.end());
        *ms_out = t[t.size() / 2];
    }
    return rc;
}

}  // namespace

extern "C" {

size_t modpp_group_workspace(const modpp_problem *probs, int count) {
    if (count < 1 || probs == nullptr) return 0;
    std::vector<ProblemCopy> pv;
    for (int i = 0; i < count; ++i) {
        if (check_problem(probs[i]) != MODPP_OK) return 0;
        pv.push_back(ProblemCopy{probs[i], std::vector<uint64_t>(probs[i].primes,
                                                                 probs[i].primes + probs[i].P)});
    }
    size_t best = 0;
    for (int b = kMinDigitBits; b <= kMaxDigitBits; ++b)
        best = std::max(best, group_layout(pv, b).total);
    return best;
}

int modpp_group_plan_create(const modpp_problem *probs, int count, void *ws, size_t ws_bytes,
                            int tune, void *stream, modpp_group_plan **out) {
    if (out == nullptr || probs == nullptr || count < 1 || count > 65536) return MODPP_ERR_ARG;
    *out = nullptr;
    if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & (kAlignG - 1)) != 0)
        return MODPP_ERR_WORKSPACE;
    auto *pl = new modpp_group_plan();
    for (int i = 0; i < count; ++i) {
        const int rc = check_problem(probs[i]);
        if (rc != MODPP_OK) {
            delete pl;
            return rc;
        }
        pl->probs.push_back(ProblemCopy{probs[i], std::vector<uint64_t>(
                                                      probs[i].primes, probs[i].primes + probs[i].P)});
        pl->probs.back().p.primes = pl->probs.back().primes.data();
    }
    pl->ws = static_cast<uint8_t *>(ws);
    pl->ws_bytes = ws_bytes;
    cudaGetDevice(&pl->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    int b = modpp_get_digit_bits();
    if (tune) {
        const std::string sig = tune_signature(pl->probs);
        int cached = 0;
        {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            tune_file_load();
            auto it = g_tune_cache.find(sig);
            if (it != g_tune_cache.end()) cached = it->second;
        }
        if (cached) {
            b = cached;
            pl->tuned = 2;
        } else {
            double best = 1e300;
            for (int cand = kMinDigitBits; cand <= kMaxDigitBits; ++cand) {
                int rc = plan_build(pl, cand, st);
                if (rc == MODPP_ERR_WORKSPACE || rc == MODPP_ERR_UNSUPPORTED) continue;
                double ms = 0;
                if (rc == MODPP_OK) rc = plan_time(pl, st, &ms);
                if (rc != MODPP_OK) {
                    delete pl;
                    return rc;
                }
                pl->tuned_ms[cand] = ms;
                if (ms < best) {
                    best = ms;
                    b = cand;
                }
            }
            pl->tuned = 1;
            std::lock_guard<std::mutex> lock(g_tune_mu);
            g_tune_cache[sig] = b;
            tune_file_append(sig, b);
        }
    }
    const int rc = plan_build(pl, b, st);
    if (rc != MODPP_OK) {
        delete pl;
        return rc;
    }
    *out = pl;
    return MODPP_OK;
}

int modpp_group_run(modpp_group_plan *plan, void *stream) {
    if (plan == nullptr) return MODPP_ERR_ARG;
    return plan_enqueue(plan, static_cast<cudaStream_t>(stream));
}

int modpp_group_run_graph(modpp_group_plan *plan, void *stream) {
    if (plan == nullptr) return MODPP_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (plan->gexec == nullptr) {
        // One eager run first sets the kernels' shared-memory attributes
        // outside the capture.
        int rc = plan_enqueue(plan, st);
        if (rc != MODPP_OK) return rc;
        cudaStream_t cap;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
            return MODPP_ERR_CUDA;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaStreamDestroy(cap);
            return MODPP_ERR_CUDA;
        }
        rc = plan_enqueue(plan, cap);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(cap, &graph);
        cudaStreamDestroy(cap);
        if (rc != MODPP_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return rc != MODPP_OK ? rc : MODPP_ERR_CUDA;
        }
        if (cudaGraphInstantiate(&plan->gexec, graph, 0) != cudaSuccess) {
            cudaGraphDestroy(graph);
            return MODPP_ERR_CUDA;
        }
        plan->graph = graph;
    }
    return cudaGraphLaunch(plan->gexec, st) == cudaSuccess ? MODPP_OK : MODPP_ERR_CUDA;
}

int modpp_group_plan_info(const modpp_group_plan *plan, int *digit_bits, int *tiles,
                          int *tuned, double *tuned_ms) {
    if (plan == nullptr) return MODPP_ERR_ARG;
    if (digit_bits) *digit_bits = plan->lay.b;
    if (tiles) *tiles = plan->gp.num_tiles;
    if (tuned) *tuned = plan->tuned;
    if (tuned_ms)
        for (int b = kMinDigitBits; b <= kMaxDigitBits; ++b)
            tuned_ms[b - kMinDigitBits] = plan->tuned_ms[b];
    return MODPP_OK;
}

void modpp_group_plan_destroy(modpp_group_plan *plan) {
    if (plan == nullptr) return;
    if (plan->gexec) cudaGraphExecDestroy(plan->gexec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    delete plan;
}

}  // extern "C"
