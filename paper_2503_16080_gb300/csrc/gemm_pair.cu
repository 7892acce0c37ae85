// Launch of the CTA-pair form of the tensor-core Mod-PP-MM kernel
// (gemm_f16_kernel.cuh with CTAS = 2): clusters of two CTAs, each pair
// computing tiles of 256 rows with tcgen05.mma.cta_group::2.
#include "gemm_f16_kernel.cuh"

namespace modpp {
namespace {

template <int L, int DB>
cudaError_t launch_pair(const CUtensorMap &tmU, const CUtensorMap &tmD, const GemmParams &p,
                        cudaStream_t s) {
    constexpr int NC = pair_tile_cols(L);
    using Cfg = GemmCfg<L, NC, 2>;
    auto kern = gemm_f16_kernel<L, DB, NC, false, 0, 2>;
    static std::atomic<unsigned long long> smem_set{0};
    cudaError_t e =
        set_smem_limit_once(reinterpret_cast<const void *>(kern), Cfg::SMEM_BYTES, smem_set);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = Cfg::SMEM_BYTES;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // Persistent clusters: as many as can be resident together (one CTA per
    // SM), queried once per instantiation.
    static int max_clusters = 0;
    if (max_clusters == 0) {
        cfg.gridDim = dim3(2, 1, 1);
        int m = 0;
        e = cudaOccupancyMaxActiveClusters(&m, kern, &cfg);
        if (e != cudaSuccess) return e;
        if (m < 1) return cudaErrorInvalidConfiguration;
        max_clusters = m;
    }
    const int clusters = p.num_tiles < max_clusters ? p.num_tiles : max_clusters;
    cfg.gridDim = dim3(2 * clusters, 1, 1);
    e = cudaLaunchKernelEx(&cfg, kern, tmU, tmD, p);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int DB>
cudaError_t launch_pair_db(const CUtensorMap &tmU, const CUtensorMap &tmD, const GemmParams &p,
                           int digits, cudaStream_t s) {
    switch (digits) {
        case 1: return launch_pair<1, DB>(tmU, tmD, p, s);
        case 2: return launch_pair<2, DB>(tmU, tmD, p, s);
        case 3: return launch_pair<3, DB>(tmU, tmD, p, s);
        case 4: return launch_pair<4, DB>(tmU, tmD, p, s);
        case 5: return launch_pair<5, DB>(tmU, tmD, p, s);
        case 6: return launch_pair<6, DB>(tmU, tmD, p, s);
        case 7: return launch_pair<7, DB>(tmU, tmD, p, s);
        case 8: return launch_pair<8, DB>(tmU, tmD, p, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_gemm_f16_pair(const CUtensorMap &tmU, const CUtensorMap &tmD,
                                 const GemmParams &p, int digits, int digit_bits, cudaStream_t s) {
    if (p.num_tiles == 0) return cudaSuccess;
    switch (digit_bits) {
        case 8: return launch_pair_db<8>(tmU, tmD, p, digits, s);
        case 9: return launch_pair_db<9>(tmU, tmD, p, digits, s);
        case 10: return launch_pair_db<10>(tmU, tmD, p, digits, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace modpp
