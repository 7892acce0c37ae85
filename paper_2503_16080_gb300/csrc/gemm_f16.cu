// Single-problem launch of the tensor-core Mod-PP-MM kernel
// (gemm_f16_kernel.cuh): every plane of one modpp_mm / pc_mm call shares U,
// the sizes and the digit count.
#include "gemm_f16_kernel.cuh"

namespace modpp {

template <int DB>
static cudaError_t launch_gemm_db(const CUtensorMap &tmU, const CUtensorMap &tmD,
                                  const GemmParams &p, int digits, int num_sms, cudaStream_t s,
                                  int nc) {
    if (nc == 32 && digits == 5) return launch_gemm_kernel<5, DB, 32, false>(tmU, tmD, p, num_sms, s);
    if (nc == 32 && digits == 6) return launch_gemm_kernel<6, DB, 32, false>(tmU, tmD, p, num_sms, s);
    if (nc != 0 && nc != tile_cols(digits)) return cudaErrorInvalidValue;
    switch (digits) {
#define MODPP_CASE(LL) \
    case LL: return launch_gemm_kernel<LL, DB, tile_cols(LL), false>(tmU, tmD, p, num_sms, s);
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

cudaError_t launch_gemm_f16(const CUtensorMap &tmU, const CUtensorMap &tmD, const GemmParams &p,
                            int digits, int digit_bits, int num_sms, cudaStream_t s, int nc) {
    if (p.num_tiles == 0) return cudaSuccess;
    switch (digit_bits) {
        case 8: return launch_gemm_db<8>(tmU, tmD, p, digits, num_sms, s, nc);
        case 9: return launch_gemm_db<9>(tmU, tmD, p, digits, num_sms, s, nc);
        case 10: return launch_gemm_db<10>(tmU, tmD, p, digits, num_sms, s, nc);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace modpp
