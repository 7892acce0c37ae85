// Exact Mod-PP-MM on the sm_103a tensor cores: the kernel template shared by
// the single-problem launch (gemm_f16.cu) and the grouped launch (grouped.cu).
//
// For one output plane (prime q, part A or B) the kernel computes
//   C[r][c] = sum_t U[r][t] * A[t][c]  mod q
// from balanced b-bit digits A = sum_l 2^(b l) D_l (|D_l| <= 2^(b-1), b = 8..10):
//   C = sum_l 2^(b l) * (U * D_l)  mod q.
// Every U * D_l runs on tcgen05.mma kind::f16 (f16 operands, FP32 accumulate
// in TMEM).  f16 holds U in [-128, 127] and D_l exactly, and the products
// are exact; the FP32 sums stay exact because the inner dimension is cut into
// chunks of 2^(18-b): |sum| <= 2^(18-b) * 128 * 2^(b-1) = 2^24, the largest
// range in which FP32 represents every integer.  After each chunk the
// epilogue warps move the chunk's sums out of TMEM into 64-bit integer
// registers; after the last chunk of a tile they recombine the digits modulo
// q (Barrett + Shoup) and store canonical residues.  This is the
// limb-splitting reduction of Sec. 6.1 (Lemma le:strategy1, exact chopping)
// with the digit base and chunk sized for FP32 tensor-core accumulation
// instead of binary64 BLAS.
//
// Tile: 128 output rows x NC output columns x Lp digits.  The Lp digit rows of
// the NC columns are adjacent in the digit matrix, so one UMMA of N = NC * Lp
// computes all digits of the tile and reuses the U tile Lp times.
//
// Warp roles (320 threads, one CTA per SM, persistent over tiles):
//   warp 0      TMA producer: U and digit tiles -> shared-memory ring
//   warp 1      TMEM owner and single-thread MMA issuer
//   warps 2-9   epilogue: TMEM -> registers, int64 accumulation of each
//               group of three digits (one IMAD.WIDE per value), modular
//               recombination at the end of the tile, global stores
// Two TMEM accumulators (columns 0.. and 256..) alternate between chunks, so
// the epilogue drains one while the tensor cores fill the other.
//
// CTAS = 2: a cluster of two CTAs computes tiles of 256 rows with
// tcgen05.mma.cta_group::2 (M = 256): each CTA loads its own 128 rows of U
// and half of the digit tile (N / 2 rows) into its shared memory, the even
// CTA (the leader) issues the MMAs, and each CTA's tensor memory receives
// the accumulators of its 128 rows.  Half of B per CTA means a stage of
// (128 + N/2) x 64 halves instead of (128 + N) x 64, so the ring holds more
// stages in flight.  TMA completions of both CTAs are counted on the
// leader's `full` barrier; MMA completions are multicast to both CTAs'
// `empty`, `tfull` and `drain` barriers; both CTAs' epilogue warps arrive on
// the leader's `tempty`.  Every wait stays bounded, and both CTAs meet at a
// cluster barrier before the tensor memory is released and the CTAs exit.
//
// GROUPED = false: one problem; all planes share U, the sizes and the digit
// count L, and the tensor maps are kernel parameters.  GROUPED = true: the
// tiles of many problems are concatenated; each tile looks up its plane's
// descriptor (sizes, digit count Lp <= L, tensor maps in global memory).
#pragma once
#include <cuda_fp16.h>

#include "modarith.cuh"
#include "modpp_internal.h"
#include "ptx_sm103.cuh"

namespace modpp {

template <int L, int NC, int CTAS = 1>
struct GemmCfg {
    static constexpr int BN = L * NC;  // largest UMMA N (all L digits)
    static constexpr int A_BYTES = kBM * kBK * 2;
    static constexpr int B_BYTES = BN / CTAS * kBK * 2;  // a CTA pair holds half of B each
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int SMEM_LIMIT = 232448;  // opt-in dynamic shared memory per CTA
    static constexpr int RESERVED = 1024 + 256;
    static constexpr int FIT = (SMEM_LIMIT - RESERVED) / STAGE_BYTES;
    static constexpr int STAGES = FIT > 8 ? 8 : FIT;
    static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + RESERVED;
    static constexpr uint32_t TMEM_COLS = 512;
    static constexpr uint32_t ACC_STRIDE = 256;
    static_assert(BN % (16 * CTAS) == 0 && BN <= 256, "UMMA N for M = 128 (one CTA) or 256 (pair)");
    static_assert(STAGES >= 2, "pipeline depth");
};

constexpr int kThreads = 320;
constexpr int kEpiWarps = 8;

// Everything the three roles need about one tile.
struct TileJob {
    const CUtensorMap *tmU;
    const CUtensorMap *tmD;
    const PlaneConst *pc;
    int mb, nb;       // 128-row block, column block
    int d, n;         // plane sizes (stores are bounded by them)
    int kb_total;     // inner dimension in 64-element blocks
    int by;           // first row of the tile's digits in the digit matrix
    int uy;           // first row of the plane's U in the U map (per-plane U, mode 1)
    int Lp;           // digits of this plane
};

// Position `local` of a plane's m_blocks x n_blocks tiles in band order:
// bands of `band` row blocks (the last may be shorter), row block fastest
// inside a band, then column block.
__device__ __forceinline__ void band_order(int local, int m_blocks, int n_blocks, int band,
                                           int &mb, int &nb) {
    if (band < 1) band = m_blocks;
    const int per_band = band * n_blocks;
    const int b = local / per_band;
    const int first = b * band;
    const int g = min(band, m_blocks - first);
    const int r = local - b * per_band;
    mb = first + r % g;
    nb = r / g;
}

template <int L, int NC, bool GROUPED>
__device__ __forceinline__ TileJob tile_job(int tile, const CUtensorMap *tmU,
                                            const CUtensorMap *tmD, const GemmParams &p) {
    TileJob j;
    if constexpr (!GROUPED) {
        // Row block fastest inside bands of p.band_m row blocks: the
        // concurrently running tiles share the digit tiles of a few column
        // blocks and the band's rows of U, which stay in L2.  Plane fastest,
        // for thin outputs with a large U: the planes of one row block run
        // together and read that block of U from HBM once.
        int plane;
        if (p.plane_fastest) {
            plane = tile % p.planes;
            const int rest = tile / p.planes;
            j.mb = rest % p.m_blocks;
            j.nb = rest / p.m_blocks;
        } else {
            const int per_plane = p.m_blocks * p.n_blocks;
            plane = tile / per_plane;
            band_order(tile - plane * per_plane, p.m_blocks, p.n_blocks, p.band_m, j.mb, j.nb);
        }
        j.tmU = tmU;
        j.tmD = tmD;
        j.pc = &p.pc[plane];
        j.d = p.d;
        j.n = p.n;
        j.kb_total = p.kb_total;
        j.by = (plane * p.n_blocks + j.nb) * L * NC;
        j.uy = p.u_per_plane ? plane * p.d : 0;
        j.Lp = L;
    } else {
        // One table entry per tile names its plane: one dependent load, so
        // short tiles do not wait on a search through the plane table.
        const GroupPlane &g = p.gplanes[p.tile_plane[tile]];
        band_order(tile - g.tile_begin, g.m_blocks, g.n_blocks, g.band_m, j.mb, j.nb);
        j.tmU = g.tmU;
        j.tmD = g.tmD;
        j.pc = &g.pc;
        j.d = g.d;
        j.n = g.n;
        j.kb_total = g.kb_total;
        j.by = (g.dplane * g.n_blocks + j.nb) * g.Lp * NC;
        j.uy = 0;
        j.Lp = g.Lp;
    }
    return j;
}

// MODE 0: digit products recombined modulo q (above).  MODE 1: one small
// prime per plane (L = 1): the plane's operands are residues modulo a prime
// p < 256 in balanced form, the host guarantees |sum| < 2^24 over the whole
// inner dimension (no chunks), and the epilogue stores the balanced residue
// of each output modulo p as int8 (the multi-modular products of
// rns_wide.cu).  Each plane then has its own U rows (p.u_per_plane).  With
// the plane's `accumulate` set, the residues already stored are added (the
// inner dimension in chunks).
template <int L, int DB, int NC, bool GROUPED, int MODE = 0, int CTAS = 1>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_f16_kernel(const __grid_constant__ CUtensorMap tmU_param,
                    const __grid_constant__ CUtensorMap tmD_param,
                    const __grid_constant__ GemmParams p) {
    static_assert(CTAS == 1 || (CTAS == 2 && MODE == 0 && !GROUPED), "pairs: single-problem digits");
    using Cfg = GemmCfg<L, NC, CTAS>;
    constexpr int STAGES = Cfg::STAGES;
    constexpr int kRowsPerTile = kBM * CTAS;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * Cfg::STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;
    uint64_t *tempty = tfull + 2;
    uint64_t *drain = tempty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *drain_abort = abort_flag + 1;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    // Pair: rank 0 leads; tiles are distributed over clusters.
    const uint32_t rank = CTAS == 2 ? cluster_ctarank() : 0u;
    const bool leader = rank == 0;
    const int tile0 = CTAS == 2 ? static_cast<int>(cluster_id_x()) : static_cast<int>(blockIdx.x);
    const int tstep = CTAS == 2 ? static_cast<int>(cluster_count_x()) : static_cast<int>(gridDim.x);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], kEpiWarps * CTAS);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        *drain_abort = 0;
        fence_mbar_init();
        if constexpr (!GROUPED) {
            tma_prefetch_desc(&tmU_param);
            tma_prefetch_desc(&tmD_param);
        }
    }
    if (warp == 1) {
        if constexpr (CTAS == 2) {
            tmem_alloc_pair(tmem_slot, Cfg::TMEM_COLS);
            tmem_relinquish_pair();
        } else {
            tmem_alloc(tmem_slot, Cfg::TMEM_COLS);
            tmem_relinquish();
        }
    }
    tc_fence_before();
    __syncthreads();
    // Pair: both CTAs' barriers initialised and tensor memory allocated
    // before either CTA signals the other.
    if constexpr (CTAS == 2) cluster_sync_all();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    constexpr int kChunkKB = MODE == 1 ? (1 << 20) / kBK : chunk_k(DB) / kBK;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            const CUtensorMap *last_map = nullptr;
            for (int tile = tile0; ok && tile < p.num_tiles; tile += tstep) {
                const TileJob j = tile_job<L, NC, GROUPED>(tile, &tmU_param, &tmD_param, p);
                if constexpr (GROUPED) {
                    if (j.tmD != last_map) {
                        // Tensor maps written to global memory before the launch.
                        tma_fence_acquire_desc(j.tmU);
                        tma_fence_acquire_desc(j.tmD);
                        last_map = j.tmD;
                    }
                }
                const int ay = j.uy + j.mb * kRowsPerTile + static_cast<int>(rank) * kBM;
                const int by = j.by + static_cast<int>(rank) * (j.Lp * NC / CTAS);
                const uint32_t bytes =
                    Cfg::A_BYTES + static_cast<uint32_t>(j.Lp * NC / CTAS * kBK * 2);
                for (int kb = 0; kb < j.kb_total; ++kb, ++it) {
                    const int s = static_cast<int>(it % STAGES);
                    const uint32_t ph = (it / STAGES) & 1u;
                    if (!mbar_wait_bounded(&empty[s], ph ^ 1u, abort_flag, p.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    uint8_t *sa = smem + s * Cfg::STAGE_BYTES;
                    if constexpr (CTAS == 2) {
                        // Both CTAs' loads complete on the leader's full[s],
                        // which expects the bytes of the pair.
                        if (leader) mbar_arrive_expect_tx(&full[s], bytes * CTAS);
                        const uint32_t fb = mapa_shared(&full[s], 0);
                        tma_load_2d_pair(sa, j.tmU, fb, kb * kBK, ay);
                        tma_load_2d_pair(sa + Cfg::A_BYTES, j.tmD, fb, kb * kBK, by);
                    } else {
                        mbar_arrive_expect_tx(&full[s], bytes);
                        tma_load_2d(sa, j.tmU, &full[s], kb * kBK, ay);
                        tma_load_2d(sa + Cfg::A_BYTES, j.tmD, &full[s], kb * kBK, by);
                    }
                }
            }
            // Every issued load must land before the CTA may exit.  A pair's
            // loads are counted on the leader's barriers: the leader drains
            // them, and the final cluster barrier holds the peer until then.
            if (leader)
                for (uint32_t q = it > static_cast<uint32_t>(STAGES) ? it - STAGES : 0u; q < it; ++q)
                    mbar_wait_bounded(&full[q % STAGES], (q / STAGES) & 1u, drain_abort,
                                      p.timeout_ns);
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0 && leader) {
            uint32_t it = 0, g = 0;
            bool ok = true;
            // Descriptors of stage 0's operand tiles; stage s adds
            // s * STAGE_BYTES and sub-block ks adds 32 bytes (the start address
            // field holds the address >> 4; shared addresses stay below 2^18, so
            // the additions never carry out of the field).
            const uint64_t adesc0 = sdesc_kmajor<kRowBytes>(smem_u32(smem));
            const uint64_t bdesc0 = sdesc_kmajor<kRowBytes>(smem_u32(smem) + Cfg::A_BYTES);
            for (int tile = tile0; ok && tile < p.num_tiles; tile += tstep) {
                const TileJob j = tile_job<L, NC, GROUPED>(tile, &tmU_param, &tmD_param, p);
                const uint32_t idesc = idesc_f16_f32(kRowsPerTile, j.Lp * NC);
                const int n_chunks = (j.kb_total + kChunkKB - 1) / kChunkKB;
                for (int ch = 0; ok && ch < n_chunks; ++ch, ++g) {
                    const uint32_t buf = g & 1u, use = g >> 1;
                    if (!mbar_wait_bounded(&tempty[buf], (use & 1u) ^ 1u, abort_flag,
                                           p.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dtm = tmem_base + buf * Cfg::ACC_STRIDE;
                    const int kb0 = ch * kChunkKB;
                    const int kb1 = min(kb0 + kChunkKB, j.kb_total);
                    for (int kb = kb0; kb < kb1; ++kb, ++it) {
                        const int s = static_cast<int>(it % STAGES);
                        const uint32_t ph = (it / STAGES) & 1u;
                        if (!mbar_wait_bounded(&full[s], ph, abort_flag, p.timeout_ns)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t soff = static_cast<uint64_t>(s) * (Cfg::STAGE_BYTES >> 4);
#pragma unroll
                        for (int ks = 0; ks < kBK / 16; ++ks) {
                            const uint64_t ad = adesc0 + soff + static_cast<uint64_t>(ks * 2);
                            const uint64_t bd = bdesc0 + soff + static_cast<uint64_t>(ks * 2);
                            const uint32_t acc = (kb > kb0 || ks > 0) ? 1u : 0u;
                            if constexpr (CTAS == 2)
                                umma_f16_ss_pair(dtm, ad, bd, idesc, acc);
                            else
                                umma_f16_ss(dtm, ad, bd, idesc, acc);
                        }
                        if constexpr (CTAS == 2)
                            umma_commit_pair_mc(&empty[s], 0x3);
                        else
                            umma_commit(&empty[s]);
                    }
                    if (!ok) break;
                    if constexpr (CTAS == 2)
                        umma_commit_pair_mc(&tfull[buf], 0x3);
                    else
                        umma_commit(&tfull[buf]);
                }
            }
            if constexpr (CTAS == 2)
                umma_commit_pair_mc(drain, 0x3);
            else
                umma_commit(drain);
            mbar_wait_bounded(drain, 0, drain_abort, p.timeout_ns);
        } else if (CTAS == 2 && lane == 0) {
            // The peer issues no MMAs: it waits until the leader's last ones
            // (which write its tensor memory and read its shared memory) are done.
            mbar_wait_bounded(drain, 0, drain_abort, p.timeout_ns);
        }
    } else {
        // ------------------------------------------------ epilogue warps
        constexpr int NCH = NC / 2;          // columns per epilogue warp
        if constexpr (MODE == 1) {
            const int ew = warp - 2;
            const int quarter = warp & 3;
            const int half = ew >> 2;
            const uint32_t lane_off = static_cast<uint32_t>(quarter * 32) << 16;
            uint32_t g = 0;
            for (int tile = blockIdx.x; tile < p.num_tiles; tile += gridDim.x, ++g) {
                const TileJob j = tile_job<L, NC, GROUPED>(tile, &tmU_param, &tmD_param, p);
                const uint32_t buf = g & 1u, use = g >> 1;
                const bool got = mbar_wait_bounded(&tfull[buf], use & 1u, abort_flag, p.timeout_ns);
                if (!__all_sync(0xffffffffu, got)) break;
                tc_fence_after();
                const uint32_t base = tmem_base + lane_off + buf * Cfg::ACC_STRIDE + half * NCH;
                const PlaneConst &pc = *j.pc;
                const int pr = static_cast<int>(pc.q);
                const float pinv = __uint_as_float(static_cast<uint32_t>(pc.mu));
                const int row = j.mb * kBM + quarter * 32 + lane;
                const int col0 = j.nb * NC + half * NCH;
                int8_t *out = reinterpret_cast<int8_t *>(pc.C) + static_cast<int64_t>(row) * pc.ldc +
                              col0;
                const bool vec = (reinterpret_cast<uintptr_t>(out) & 15u) == 0;
#pragma unroll 1
                for (int c0 = 0; c0 < NCH; c0 += 16) {
                    uint32_t r[16];
                    tmem_ld_cols<16>(base + c0, r);
                    tmem_wait_ld();
                    // balanced residue of an exact integer |v| < 2^24 modulo p:
                    // v - p * rint(v / p), corrected by at most one p
                    // accumulate: add the residues already stored (an earlier
                    // chunk of the inner dimension) and reduce again
                    uint32_t old[4] = {0, 0, 0, 0};
                    const bool acc = pc.accumulate && row < j.d;
                    if (acc) {
                        if (vec && col0 + c0 + 16 <= j.n) {
                            const uint4 o = *reinterpret_cast<const uint4 *>(out + c0);
                            old[0] = o.x;
                            old[1] = o.y;
                            old[2] = o.z;
                            old[3] = o.w;
                        } else {
#pragma unroll
                            for (int c = 0; c < 16; ++c)
                                if (col0 + c0 + c < j.n)
                                    old[c >> 2] |= (static_cast<uint32_t>(out[c0 + c]) & 0xffu)
                                                   << (8 * (c & 3));
                        }
                    }
                    uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        const float f = __uint_as_float(r[c]);
                        int x = __float2int_rn(f) - pr * __float2int_rn(f * pinv);
                        if (2 * x > pr) x -= pr;
                        if (2 * x < -pr) x += pr;
                        if (acc) {
                            x += static_cast<int8_t>((old[c >> 2] >> (8 * (c & 3))) & 0xffu);
                            if (2 * x > pr) x -= pr;
                            if (2 * x < -pr) x += pr;
                        }
                        w[c >> 2] |= (static_cast<uint32_t>(x) & 0xffu) << (8 * (c & 3));
                    }
                    if (row < j.d) {
                        if (vec && col0 + c0 + 16 <= j.n) {
                            *reinterpret_cast<uint4 *>(out + c0) = make_uint4(w[0], w[1], w[2], w[3]);
                        } else {
#pragma unroll
                            for (int c = 0; c < 16; ++c)
                                if (col0 + c0 + c < j.n)
                                    out[c0 + c] = static_cast<int8_t>((w[c >> 2] >> (8 * (c & 3))) & 0xffu);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[buf]);
            }
        } else {
        constexpr int G = (L + 2) / 3;       // digit groups: digits 3g, 3g+1, 3g+2
        // The TMEM round trips of a chunk's drain (load, then one wait) bound
        // it, not the conversions.  Two ways to batch the loads:
        //   by columns: all L digits of CW columns per wait, NCH / CW waits;
        //   by digits:  DPB digits of all NCH columns per wait, ceil(L / DPB)
        //               waits (DPB * NCH <= 64 registers; used with at most
        //               two digit groups, where the accumulators leave room).
        constexpr int CW = (L >= 7 || NCH % 8 != 0) ? 4 : 8;
        constexpr int DPB = NCH * 3 <= 64 ? 3 : (NCH * 2 <= 64 ? 2 : 1);
        // (load registers DPB * NCH plus int64 accumulators 2 * G * NCH kept
        // within 140 of the 168 a thread has: no spills)
        constexpr bool kByDigits =
            G <= 2 && (L + DPB - 1) / DPB < NCH / CW && DPB * NCH + 2 * G * NCH <= 140;
        constexpr int kDigitWeight[3] = {1, 1 << DB, 1 << (2 * DB)};
        const int ew = warp - 2;
        const int quarter = warp & 3;  // TMEM lane quarter this warp may access
        const int half = ew >> 2;      // which half of the tile's columns
        const uint32_t lane_off = static_cast<uint32_t>(quarter * 32) << 16;
        // grp[g][c] = sum over chunks of sum_{j<3} 2^(b j) * C_{3g+j}.  A chunk
        // adds at most 2^24 (1 + 2^b + 2^(2b)) < 2^(25+2b); with at most
        // 2^(2+b) chunks (k <= 2^20) the total stays below 2^(27+3b) <= 2^57.
        int64_t grp[G][NCH];
        uint32_t g = 0;
        bool ok = true;
        // Pair: both CTAs' epilogue warps release a drained accumulator on
        // the leader's tempty (which the leader's MMA thread waits on).
        const uint32_t tempty_leader0 = CTAS == 2 ? mapa_shared(&tempty[0], 0) : 0u;
        const uint32_t tempty_leader1 = CTAS == 2 ? mapa_shared(&tempty[1], 0) : 0u;
        for (int tile = tile0; ok && tile < p.num_tiles; tile += tstep) {
            const TileJob j = tile_job<L, NC, GROUPED>(tile, &tmU_param, &tmD_param, p);
            const int Lp = GROUPED ? j.Lp : L;
            const int n_chunks = (j.kb_total + kChunkKB - 1) / kChunkKB;
#pragma unroll
            for (int gi = 0; gi < G; ++gi)
#pragma unroll
                for (int c = 0; c < NCH; ++c) grp[gi][c] = 0;
            for (int ch = 0; ch < n_chunks; ++ch, ++g) {
                const uint32_t buf = g & 1u, use = g >> 1;
                const bool got = mbar_wait_bounded(&tfull[buf], use & 1u, abort_flag, p.timeout_ns);
                if (!__all_sync(0xffffffffu, got)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t base = tmem_base + lane_off + buf * Cfg::ACC_STRIDE + half * NCH;
                if constexpr (kByDigits) {
#pragma unroll
                    for (int l0 = 0; l0 < L; l0 += DPB) {
                        uint32_t r[DPB][NCH];
#pragma unroll
                        for (int j = 0; j < DPB; ++j)
                            if (l0 + j < L && l0 + j < Lp)
                                tmem_ld_cols<NCH>(base + (l0 + j) * NC, r[j]);
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < DPB; ++j) {
                            const int l = l0 + j;
                            if (l >= L || l >= Lp) continue;
#pragma unroll
                            for (int c = 0; c < NCH; ++c)
                                grp[l / 3][c] =
                                    mad_wide_s32(__float2int_rn(__uint_as_float(r[j][c])),
                                                 kDigitWeight[l % 3], grp[l / 3][c]);
                        }
                    }
                } else {
#pragma unroll
                    for (int c0 = 0; c0 < NCH; c0 += CW) {
                        uint32_t r[L][CW];
#pragma unroll
                        for (int l = 0; l < L; ++l)
                            if (l < Lp) tmem_ld_group<CW>(base + l * NC + c0, r[l]);
                        tmem_wait_ld();
#pragma unroll
                        for (int l = 0; l < L; ++l) {
                            if (l >= Lp) continue;
#pragma unroll
                            for (int c = 0; c < CW; ++c)
                                grp[l / 3][c0 + c] = mad_wide_s32(
                                    __float2int_rn(__uint_as_float(r[l][c])), kDigitWeight[l % 3],
                                    grp[l / 3][c0 + c]);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    if constexpr (CTAS == 2)
                        mbar_arrive_cluster(buf ? tempty_leader1 : tempty_leader0);
                    else
                        mbar_arrive(&tempty[buf]);
                }
            }
            if (!ok) break;
            // value = grp0 + 2^(3b) grp1 + 2^(6b) grp2  (mod q)
            const int row = j.mb * kRowsPerTile + static_cast<int>(rank) * kBM + quarter * 32 + lane;
            const int col0 = j.nb * NC + half * NCH;
            if (row < j.d) {
                const PlaneConst &pc = *j.pc;
                uint64_t *out = pc.C + static_cast<int64_t>(row) * pc.ldc + col0;
                // Whole 32-byte sectors per lane when the row segment is aligned
                // and inside the matrix; element stores otherwise.
                const bool vec =
                    (reinterpret_cast<uintptr_t>(out) & 31u) == 0 && col0 + NCH <= j.n;
#pragma unroll
                for (int c0 = 0; c0 < NCH; c0 += 4) {
                    uint64_t v[4];
#pragma unroll
                    for (int k4 = 0; k4 < 4; ++k4) {
                        const int c = c0 + k4;
                        // |grp| < 2^57: adding qoff (a multiple of q) makes each
                        // sum a non-negative word with the same residue, so one
                        // Barrett (group 0) or Shoup (groups 1, 2, times their
                        // weight) reduction needs no sign handling.  This
                        // per-tile reduction overlaps the next tile's MMAs only
                        // while it is shorter than about two K chunks, so its
                        // length shows in the GEMM time.
                        uint64_t x = barrett_u64(static_cast<uint64_t>(grp[0][c]) + pc.qoff,
                                                 pc.q, pc.mu);
                        if constexpr (G > 1)
                            x = add_mod(x, shoup_mulmod(static_cast<uint64_t>(grp[1][c]) + pc.qoff,
                                                        pc.wg1, pc.wg1s, pc.q),
                                        pc.q);
                        if constexpr (G > 2)
                            x = add_mod(x, shoup_mulmod(static_cast<uint64_t>(grp[2][c]) + pc.qoff,
                                                        pc.wg2, pc.wg2s, pc.q),
                                        pc.q);
                        if (pc.accumulate) {  // C <- C + wout * x (wide products), or
                            x = shoup_mulmod(x, pc.wout, pc.wouts, pc.q);  // wout * x (2)
                            if (pc.accumulate == 1 && col0 + c < j.n) x = add_mod(x, out[c], pc.q);
                        }
                        v[k4] = x;
                    }
                    if (vec) {
                        st_global_v4_u64(out + c0, v[0], v[1], v[2], v[3]);
                    } else {
#pragma unroll
                        for (int k4 = 0; k4 < 4; ++k4)
                            if (col0 + c0 + k4 < j.n) out[c0 + k4] = v[k4];
                    }
                }
            }
        }
        }  // MODE 0
    }

    tc_fence_before();
    __syncthreads();
    // Pair: neither CTA releases its tensor memory or exits while the other
    // may still signal its barriers or have the leader's MMAs use its memory.
    if constexpr (CTAS == 2) cluster_sync_all();
    if (warp == 1) {
        tc_fence_after();
        if constexpr (CTAS == 2)
            tmem_dealloc_pair(tmem_base, Cfg::TMEM_COLS);
        else
            tmem_dealloc(tmem_base, Cfg::TMEM_COLS);
    }
    if (threadIdx.x == 0 && (*abort_flag || *drain_abort)) atomicExch(p.status, -7);
}

template <int L, int DB, int NC, bool GROUPED, int MODE = 0>
cudaError_t launch_gemm_kernel(const CUtensorMap &tmU, const CUtensorMap &tmD, const GemmParams &p,
                               int num_sms, cudaStream_t s) {
    using Cfg = GemmCfg<L, NC>;
    static std::atomic<unsigned long long> smem_set{0};
    cudaError_t e = set_smem_limit_once(
        reinterpret_cast<const void *>(gemm_f16_kernel<L, DB, NC, GROUPED, MODE>), Cfg::SMEM_BYTES,
        smem_set);
    if (e != cudaSuccess) return e;
    const int grid = p.num_tiles < num_sms ? p.num_tiles : num_sms;
    gemm_f16_kernel<L, DB, NC, GROUPED, MODE><<<grid, kThreads, Cfg::SMEM_BYTES, s>>>(tmU, tmD, p);
    return cudaGetLastError();
}

}  // namespace modpp
